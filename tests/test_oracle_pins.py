"""Pins of the CPU oracle to facts that do not come from the oracle itself.

The oracle restates the Raubold-Lynch phase-space generator of Hydra §4.2 (F. James,
CERN 68-15).  These tests check it against: published Philox known-answer vectors,
exact conservation laws, the two-body closed form, invariant masses of the subsystems,
Kallen's lambda in exact rational arithmetic, the closed-form massless N-body volume,
massive volumes by numerical quadrature (3 and 4 bodies), the flat Dalitz density of
3-body phase space, a Dalitz matrix-element integral by 2-D quadrature, isotropy, and
the oracle's own rounding error (double vs long double build).
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads
from conftest import load_kat
from refmath import (R3_quad, R_recursive, dalitz_me_integral_quad, dalitz_s23_range,
                     massless_volume, minkowski2, two_body_p)

TWO32 = 2 ** 32


# ----------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    for row in load_kat("philox4x32_10_kat.txt"):
        ctr, key, want = row[0:4], row[4:6], tuple(row[6:10])
        assert oracle.philox4x32_10(ctr, key) == want


def test_draw_mapping_is_counter_based():
    # draw d of event e is word d%4 of Philox(counter=(e_lo, e_hi, d//4, 0), key=(seed_lo, seed_hi))
    seed, event = 0x0123456789ABCDEF, 0xFEDCBA9876543210
    for d in range(26):
        blk = oracle.philox4x32_10([event & 0xFFFFFFFF, event >> 32, d // 4, 0],
                                   [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle.draw(seed, event, d) == blk[d % 4]


# ----------------------------------------------------------------------------- two-body
@pytest.mark.parametrize("M,m1,m2", [(10.0, 0.0, 0.0), (5.2795, 3.0969, 0.4937),
                                     (1.0, 0.3, 0.6999), (3.0, 0.0, 1.2)])
def test_two_body_closed_form(M, m1, m2):
    p, w = oracle.generate(M, (m1, m2), 2000, seed=3)
    pstar = two_body_p(M, m1, m2)
    E1 = (M * M + m1 * m1 - m2 * m2) / (2 * M)
    E2 = (M * M + m2 * m2 - m1 * m1) / (2 * M)
    mom1 = np.sqrt(p[0, 1] ** 2 + p[0, 2] ** 2 + p[0, 3] ** 2)
    np.testing.assert_allclose(mom1, pstar, rtol=1e-12, atol=1e-14 * M)
    np.testing.assert_allclose(p[0, 0], E1, rtol=1e-13)
    np.testing.assert_allclose(p[1, 0], E2, rtol=1e-13)
    # two-body weight: R_2 = pi p* / M exactly (C_2 = pi / M)
    np.testing.assert_allclose(w, math.pi * pstar / M, rtol=1e-12)
    # back to back
    np.testing.assert_allclose(p[0, 1:] + p[1, 1:], 0.0, atol=1e-14 * M)


# ----------------------------------------------------------------------------- conservation
@pytest.mark.parametrize("n", range(2, 11))
def test_conservation_and_on_shell(n):
    rng = np.random.default_rng(100 + n)
    for trial in range(3):
        M, masses = workloads.random_decay(rng, n)
        p, w = oracle.generate(M, masses, 3000, seed=trial + 11 * n)
        tot = p.sum(axis=0)
        np.testing.assert_allclose(tot[0], M, rtol=0, atol=1e-13 * M)
        np.testing.assert_allclose(tot[1:], 0.0, rtol=0, atol=1e-13 * M)
        for i, m in enumerate(masses):
            np.testing.assert_allclose(minkowski2(p[i].T), m * m, rtol=0, atol=1e-12 * M * M)
            assert np.all(p[i, 0] >= m * (1 - 1e-14))
        assert np.all(w >= 0) and np.all(np.isfinite(w))


@pytest.mark.parametrize("n", range(3, 11))
def test_subsystem_invariant_masses(n):
    """(p_1 + ... + p_k)^2 = M_k^2 with M_k = m_1+...+m_k + r_{k-1} T (sorted uniforms)."""
    rng = np.random.default_rng(7 + n)
    M, masses = workloads.random_decay(rng, n)
    seed, nev = 99, 40
    p, _ = oracle.generate(M, masses, nev, seed=seed)
    T = M - sum(masses)
    for e in range(nev):
        x = oracle.draws(seed, e, n)
        y = sorted(int(v) for v in x[: n - 2])
        r = [0.0] + [(v + 0.5) / TWO32 for v in y] + [1.0]
        cum = p[:, :, e].cumsum(axis=0)
        for k in range(2, n):
            Mk = sum(masses[:k]) + r[k - 1] * T
            got = math.sqrt(max(minkowski2(cum[k - 1]), 0.0))
            assert got == pytest.approx(Mk, rel=1e-12, abs=1e-12 * M)


@pytest.mark.parametrize("n", range(2, 11))
def test_weight_is_product_of_two_body_momenta(n):
    """w = C_n prod_k p*(M_{k+1}; M_k, m_{k+1}), masses taken from the output 4-vectors and
    lambda evaluated in exact rationals (not the factorised form the oracle uses)."""
    rng = np.random.default_rng(50 + n)
    M, masses = workloads.random_decay(rng, n)
    p, w = oracle.generate(M, masses, 30, seed=5)
    C = oracle.volume_factor(M, masses)
    T = M - sum(masses)
    assert C == pytest.approx(math.pi ** (n - 1) * (2 * T) ** (n - 2) / math.factorial(n - 2) / M,
                              rel=1e-14)
    for e in range(p.shape[2]):
        cum = p[:, :, e].cumsum(axis=0)
        Mk = [None] + [math.sqrt(max(minkowski2(cum[k - 1]), 0.0)) for k in range(1, n)] + [M]
        Mk[1] = masses[0]
        prod = 1.0
        for k in range(1, n):
            prod *= two_body_p(Mk[k + 1], Mk[k], masses[k])
        assert w[e] == pytest.approx(C * prod, rel=1e-9, abs=1e-12 * C * (M ** (n - 1)))


# ----------------------------------------------------------------------------- volumes
@pytest.mark.parametrize("n", range(2, 11))
def test_massless_volume_closed_form(n):
    M = workloads.SWEEP_M
    nev = 200_000
    _, w = oracle.generate(M, workloads.sweep_masses(n, massive=False), nev, seed=1234 + n)
    R = massless_volume(n, M)
    if n == 2:
        np.testing.assert_allclose(w, R, rtol=1e-14)
        return
    mean, sem = w.mean(), w.std(ddof=1) / math.sqrt(nev)
    assert abs(mean - R) < 4.0 * sem, (mean, R, sem)


def test_massless_three_body_exact_moment():
    """For 3 massless daughters w = C_3 p_1 p_2 and E[p_1 p_2] = M^2/16 exactly,
    so E[w] = pi^2 M^2 / 8; checked with the MC error."""
    M = 3.0
    _, w = oracle.generate(M, (0.0, 0.0, 0.0), 400_000, seed=77)
    R = math.pi ** 2 * M * M / 8
    assert R == pytest.approx(massless_volume(3, M), rel=1e-15)
    assert abs(w.mean() - R) < 4 * w.std(ddof=1) / math.sqrt(len(w))


def test_massive_three_body_volume_quadrature():
    cfg = workloads.B_TO_JPSI_K_PI
    R = R3_quad(cfg["M"], cfg["masses"])
    assert R == pytest.approx(R_recursive(cfg["M"], list(cfg["masses"]), epsrel=1e-10), rel=1e-8)
    _, w = oracle.generate(cfg["M"], cfg["masses"], cfg["nevents"] * 4, seed=cfg["seed"])
    sem = w.std(ddof=1) / math.sqrt(len(w))
    assert abs(w.mean() - R) < 4 * sem, (w.mean(), R, sem)


def test_massive_four_body_volume_nested_quadrature():
    M = 4.0
    masses = [0.3, 0.5, 0.1, 0.7]
    R = R_recursive(M, masses, epsrel=1e-6)
    nev = 300_000
    _, w = oracle.generate(M, masses, nev, seed=4)
    sem = w.std(ddof=1) / math.sqrt(nev)
    assert abs(w.mean() - R) < 4 * sem, (w.mean(), R, sem)


@pytest.mark.parametrize("n", [3, 4])
def test_massive_sweep_volumes_by_quadrature(n):
    """The N-body sweep's massive decays for N = 3, 4 against nested quadrature."""
    masses = workloads.sweep_masses(n, massive=True)
    R = R_recursive(workloads.SWEEP_M, list(masses), epsrel=1e-5)
    nev = 200_000
    _, w = oracle.generate(workloads.SWEEP_M, masses, nev, seed=10 + n)
    sem = w.std(ddof=1) / math.sqrt(nev)
    assert abs(w.mean() - R) < 4 * sem, (n, w.mean(), R, sem)


# ----------------------------------------------------------------------------- Dalitz density
def test_dalitz_density_is_flat():
    """3-body phase space is uniform in (s12, s23): the expected sum of weights in a bin
    fully inside the Dalitz boundary is n pi^2/(4M^2) * area; chi^2 over such bins."""
    cfg = workloads.B_TO_JPSI_K_PI
    M, (m1, m2, m3) = cfg["M"], cfg["masses"]
    nev = 1_000_000
    p, w = oracle.generate(M, cfg["masses"], nev, seed=cfg["seed"])
    s12 = minkowski2((p[0] + p[1]).T)
    s23 = minkowski2((p[1] + p[2]).T)
    lo12, hi12 = (m1 + m2) ** 2, (M - m3) ** 2
    lo23, hi23 = (m2 + m3) ** 2, (M - m1) ** 2
    nb = 24
    e12 = np.linspace(lo12, hi12, nb + 1)
    e23 = np.linspace(lo23, hi23, nb + 1)

    def inside(a, b):
        if a <= lo12 or a >= hi12:
            return False
        lo, hi = dalitz_s23_range(M, m1, m2, m3, a)
        return lo < b < hi

    sw, _, _ = np.histogram2d(s12, s23, bins=[e12, e23], weights=w)
    sw2, _, _ = np.histogram2d(s12, s23, bins=[e12, e23], weights=w * w)
    area = (e12[1] - e12[0]) * (e23[1] - e23[0])
    expect = nev * math.pi ** 2 / (4 * M * M) * area
    chi2, dof = 0.0, 0
    for i in range(nb):
        for j in range(nb):
            corners = [(e12[i + a], e23[j + b]) for a in (0, 1) for b in (0, 1)]
            if all(inside(a, b) for a, b in corners):
                chi2 += (sw[i, j] - expect) ** 2 / sw2[i, j]
                dof += 1
    assert dof > 100
    pval = stats.chi2.sf(chi2, dof)
    assert pval > 1e-3, (chi2, dof, pval)


def test_dalitz_matrix_element_integral_quadrature():
    """Int |ME|^2 dR_3 = pi^2/(4M^2) Int Int |ME|^2 ds12 ds23 (2-D quadrature, with the
    resonance poles as break points) against the oracle's weighted MC mean."""
    cfg = workloads.D0_DALITZ
    M = cfg["M"]
    exact, me2 = dalitz_me_integral_quad(M, cfg["masses"], cfg["params"])
    # the oracle's ME at a few points (complex-number form written independently here)
    for s12, s23 in [(0.8, 1.0), (0.9, 1.04), (0.5, 0.7)]:
        assert oracle.me_dalitz_2bw(s12, s23, cfg["params"]) == pytest.approx(me2(s12, s23), rel=1e-13)
    res = oracle.integrate(M, cfg["masses"], 2_000_000, seed=cfg["seed"], me=1, params=cfg["params"])
    sigma = math.sqrt(res["var_mean"])
    assert abs(res["mean"] - exact) < 4 * sigma, (res["mean"], exact, sigma)
    # flat matrix element: the integral is the volume
    flat = oracle.integrate(M, cfg["masses"], 400_000, seed=3)
    assert abs(flat["mean"] - R3_quad(M, cfg["masses"])) < 4 * math.sqrt(flat["var_mean"])
    assert flat["sum_f"] == flat["sum_w"]


# ----------------------------------------------------------------------------- isotropy
@pytest.mark.parametrize("n", [2, 3, 6, 10])
def test_isotropy_of_last_daughter(n):
    M = 10.0
    masses = workloads.sweep_masses(n, massive=True)
    p, _ = oracle.generate(M, masses, 50_000, seed=21)
    d = p[n - 1]
    mom = np.sqrt(d[1] ** 2 + d[2] ** 2 + d[3] ** 2)
    cos_t = d[3] / mom
    phi = np.arctan2(d[2], d[1])
    assert stats.kstest(cos_t, "uniform", args=(-1, 2)).pvalue > 1e-3
    assert stats.kstest(phi, "uniform", args=(-math.pi, 2 * math.pi)).pvalue > 1e-3


# ----------------------------------------------------------------------------- reproducibility
def test_event_offset_reproduces_one_call():
    M, masses = 7.0, (0.1, 0.2, 0.3, 0.4, 0.5)
    a, wa = oracle.generate(M, masses, 1000, seed=9)
    b1, wb1 = oracle.generate(M, masses, 300, seed=9)
    b2, wb2 = oracle.generate(M, masses, 700, seed=9, event_offset=300)
    assert np.array_equal(a, np.concatenate([b1, b2], axis=2))
    assert np.array_equal(wa, np.concatenate([wb1, wb2]))


# ----------------------------------------------------------------------------- own error
@pytest.mark.parametrize("n", range(2, 11))
def test_oracle_rounding_error_vs_long_double(n):
    """The FP64 oracle against its own long double build, at the event scale max(M, E_i)."""
    M = 10.0
    masses = workloads.sweep_masses(n, massive=True)
    p64, w64 = oracle.generate(M, masses, 10_000, seed=17)
    pld, wld = oracle.generate(M, masses, 10_000, seed=17, kind="ld")
    scale = np.maximum(M, pld[:, 0, :].max(axis=0).astype(np.float64))
    err_p = (np.abs(p64 - pld.astype(np.float64)) / scale).max()
    err_w = (np.abs(w64 - wld.astype(np.float64)) / np.abs(wld.astype(np.float64))).max()
    assert err_p < 2e-14, err_p
    assert err_w < 5e-14, err_w


def test_threshold_and_invalid_inputs():
    with pytest.raises(oracle.OracleError):
        oracle.generate(1.0, (0.5, 0.5), 10, seed=1)          # sum m == M
    with pytest.raises(oracle.OracleError):
        oracle.generate(1.0, (0.6, 0.5), 10, seed=1)          # below threshold
    with pytest.raises(oracle.OracleError):
        oracle.generate(1.0, (0.1,) * 11, 10, seed=1)         # n > 10
    with pytest.raises(oracle.OracleError):
        oracle.generate(-1.0, (0.1, 0.1), 10, seed=1)


def test_near_threshold_stays_physical():
    for n in (3, 5, 10):
        M, masses = workloads.near_threshold_decay(n, rel_gap=1e-7)
        p, w = oracle.generate(M, masses, 2000, seed=8)
        assert np.all(np.isfinite(p)) and np.all(w >= 0)
        tot = p.sum(axis=0)
        np.testing.assert_allclose(tot[0], M, atol=1e-13 * M)
        for i, m in enumerate(masses):
            np.testing.assert_allclose(minkowski2(p[i].T), m * m, rtol=0, atol=1e-12 * M * M)


# ----------------------------------------------------------------------------- moving mother
def lorentz_matrix(P, M):
    """4x4 matrix of the pure boost that takes the rest frame of mass M to 4-momentum P
    (Lambda^0_0 = gamma, Lambda^0_i = gamma beta_i, Lambda^i_j = delta_ij + (gamma-1) b_i b_j)."""
    gamma = P[0] / M
    beta = np.asarray(P[1:]) / P[0]
    b2 = beta @ beta
    L = np.eye(4)
    L[0, 0] = gamma
    L[0, 1:] = L[1:, 0] = gamma * beta
    if b2 > 0:
        L[1:, 1:] += (gamma - 1.0) * np.outer(beta, beta) / b2
    return L


@pytest.mark.parametrize("n", [2, 3, 6, 10])
def test_boosted_events_are_the_rest_frame_events_boosted(n):
    rng = np.random.default_rng(300 + n)
    M, masses = workloads.random_decay(rng, n)
    mother = (1.3 * M, -0.7 * M, 2.1 * M)
    P = np.array([math.sqrt(M * M + sum(v * v for v in mother)), *mother])
    lab, w_lab = oracle.generate_boosted(M, masses, 200, seed=5, mother=mother)
    rest, w_rest = oracle.generate(M, masses, 200, seed=5)
    assert np.array_equal(w_lab, w_rest)  # weights are Lorentz invariant
    Linv = lorentz_matrix(np.array([P[0], *(-P[1:])]), M)  # inverse boost
    back = np.einsum("ab,ibe->iae", Linv, lab)
    np.testing.assert_allclose(back, rest, rtol=0, atol=1e-12 * P[0])
    tot = lab.sum(axis=0)
    np.testing.assert_allclose(tot, np.broadcast_to(P[:, None], tot.shape), rtol=0, atol=1e-12 * P[0])
    for i in range(n):
        np.testing.assert_allclose(minkowski2(lab[i].T), masses[i] ** 2, rtol=0, atol=1e-10 * P[0] ** 2)
    s_lab = minkowski2((lab[0] + lab[-1]).T)
    s_rest = minkowski2((rest[0] + rest[-1]).T)
    np.testing.assert_allclose(s_lab, s_rest, rtol=0, atol=1e-10 * P[0] ** 2)


def test_per_event_mothers():
    M, masses = 3.0, (0.2, 0.3, 0.4, 0.5)
    rng = np.random.default_rng(9)
    moms = rng.normal(0.0, 5.0, size=(3, 300))
    lab, _ = oracle.generate_boosted(M, masses, 300, seed=2, mothers=moms)
    tot = lab.sum(axis=0)
    E = np.sqrt(M * M + (moms ** 2).sum(axis=0))
    np.testing.assert_allclose(tot[0], E, rtol=1e-13)
    np.testing.assert_allclose(tot[1:], moms, rtol=0, atol=1e-12 * E.max())
    # one event equals the uniform-mother call with that event's momentum
    one, _ = oracle.generate_boosted(M, masses, 1, seed=2, mother=tuple(moms[:, 7]), event_offset=7)
    np.testing.assert_allclose(one[:, :, 0], lab[:, :, 7], rtol=0, atol=1e-13 * E[7])


# ----------------------------------------------------------------------------- unweighting
def test_unweighting_acceptance_rate_and_flat_dalitz_density():
    """Accept-reject against w_max keeps each event with probability w/w_max: the accepted
    fraction is E[w]/w_max, and the accepted (unweighted) 3-body events are uniform in the
    Dalitz plane (chi^2 of counts against bin area, bins inside the boundary)."""
    cfg = workloads.B_TO_JPSI_K_PI
    M, (m1, m2, m3) = cfg["M"], cfg["masses"]
    nev = 600_000
    p, w = oracle.generate(M, cfg["masses"], nev, seed=11)
    w_max = float(w.max()) * 1.0001
    acc = oracle.unweight(M, cfg["masses"], nev, seed=11, w_max=w_max)
    rate = w.mean() / w_max
    k = acc.sum()
    assert abs(k - nev * rate) < 5 * math.sqrt(nev * rate * (1 - rate)), (k, nev * rate)
    s12 = minkowski2((p[0] + p[1]).T)[acc]
    s23 = minkowski2((p[1] + p[2]).T)[acc]
    lo12, hi12 = (m1 + m2) ** 2, (M - m3) ** 2
    lo23, hi23 = (m2 + m3) ** 2, (M - m1) ** 2
    nb = 16
    e12, e23 = np.linspace(lo12, hi12, nb + 1), np.linspace(lo23, hi23, nb + 1)
    cnt, _, _ = np.histogram2d(s12, s23, bins=[e12, e23])
    area_tot = R3_quad(M, cfg["masses"]) * 4 * M * M / math.pi ** 2
    area = (e12[1] - e12[0]) * (e23[1] - e23[0])
    expect = k * area / area_tot

    def inside(a, b):
        lo, hi = dalitz_s23_range(M, m1, m2, m3, a)
        return lo12 < a < hi12 and lo < b < hi

    chi2, dof = 0.0, 0
    for i in range(nb):
        for j in range(nb):
            if all(inside(e12[i + a], e23[j + b]) for a in (0, 1) for b in (0, 1)):
                chi2 += (cnt[i, j] - expect) ** 2 / expect
                dof += 1
    assert dof > 50 and stats.chi2.sf(chi2, dof) > 1e-3, (chi2, dof)


def test_evaluate_on_stored_events_equals_integrate():
    """Evaluating the matrix element on stored events reproduces the integral over the same
    generated events, and the flat matrix element returns the weights."""
    d = workloads.D0_DALITZ
    p, w = oracle.generate(d["M"], d["masses"], 20_000, seed=4)
    vals, sums = oracle.evaluate(p, w, me=1, params=d["params"])
    ref = oracle.integrate_sums(d["M"], d["masses"], 20_000, seed=4, me=1, params=d["params"])
    np.testing.assert_allclose(sums, ref, rtol=1e-13)
    flat, fs = oracle.evaluate(p, w)
    assert np.array_equal(flat, w)
    s12 = minkowski2((p[0] + p[1]).T)
    s23 = minkowski2((p[1] + p[2]).T)
    for e in (0, 17, 19_999):
        assert vals[e] == pytest.approx(w[e] * oracle.me_dalitz_2bw(s12[e], s23[e], d["params"]), rel=1e-12)


def test_sequential_decay_composition():
    """A two-stage decay (daughter 2 of a 3-body decay decays to 2 bodies): the stage-2
    particles are the decay of the stage-1 daughter in its own frame, so their total
    4-momentum equals it, their invariant mass is its mass, and all final particles
    conserve the parent's 4-momentum."""
    M, m = 5.0, (0.5, 1.2, 0.3)
    sub = (0.4, 0.6)
    p1, _ = oracle.generate(M, m, 500, seed=1)
    moms = p1[1, 1:4, :]  # daughter 2's momenta
    p2, _ = oracle.generate_boosted(m[1], sub, 500, seed=2, mothers=moms)
    np.testing.assert_allclose(p2.sum(axis=0), p1[1], rtol=0, atol=1e-12 * M)
    np.testing.assert_allclose(np.sqrt(minkowski2(p2.sum(axis=0).T)), m[1], rtol=1e-12)
    final = p1[0] + p1[2] + p2[0] + p2[1]
    np.testing.assert_allclose(final[0], M, atol=1e-12 * M)
    np.testing.assert_allclose(final[1:], 0.0, atol=1e-12 * M)


# ----------------------------------------------------------------------------- VEGAS
def test_vegas_against_quadrature_and_plain():
    """VEGAS (importance sampling over the 3n-4 phase-space variables) of the Dalitz matrix
    element and of the flat one agrees with 2-D quadrature within 4 sigma; one bin per
    dimension (plain MC) too; grids stay ordered from 0 to 1."""
    d = workloads.D0_DALITZ
    exact, _ = dalitz_me_integral_quad(d["M"], d["masses"], d["params"])
    for bins in (50, 1):
        r = oracle.vegas(d["M"], d["masses"], 3, 60_000, 6, bins=bins, me=1, params=d["params"])
        assert abs(r["mean"] - exact) < 4 * r["sigma"], (bins, r["mean"], exact, r["sigma"])
        assert r["chi2_dof"] < 4.0
        g = r["grid"]
        assert np.all(g[:, 0] == 0.0) and np.all(g[:, -1] == 1.0) and np.all(np.diff(g, axis=1) > 0)
    flat = oracle.vegas(d["M"], d["masses"], 4, 40_000, 4, bins=20)
    assert abs(flat["mean"] - R3_quad(d["M"], d["masses"])) < 4 * flat["sigma"]


def test_vegas_adapts_to_a_separable_peak():
    """With only the K*(892) term and a narrow width, the peak sits at a fixed value of the
    intermediate-mass variable u0 = (0.892 - m1 - m2)/T: the refined grid puts its narrowest
    bin there, the per-iteration error falls by more than 10x, and the result matches
    quadrature."""
    d = workloads.D0_DALITZ
    par = (0.892, 0.005, 1.02, 0.004, 0.0, 1.2)
    r = oracle.vegas(d["M"], d["masses"], 1, 60_000, 8, bins=50, me=1, params=par)
    sig = np.sqrt(r["var"])
    assert sig[-1] < sig[0] / 10
    m1, m2, _ = d["masses"]
    u0 = (0.892 - m1 - m2) / (d["M"] - sum(d["masses"]))
    g0 = r["grid"][0]
    k = int(np.argmin(np.diff(g0)))
    assert g0[k] - 0.002 <= u0 <= g0[k + 1] + 0.002
    exact, _ = dalitz_me_integral_quad(d["M"], d["masses"], par)
    assert abs(r["mean"] - exact) < 4 * r["sigma"], (r["mean"], exact, r["sigma"])
