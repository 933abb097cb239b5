"""Mistakes planted in a copy of the oracle source must fail at least one pin.

Each mutation below is a plausible slip (a dropped term, a wrong sign or index, a transposed
operand, a wrong constant); the mutated oracle is compiled on the CPU and run through a fast
subset of the pins of test_oracle_pins.py.  The unmutated source passes every one of them.
(Pure conventions that physics cannot see -- which Philox word feeds cos(theta), the sign
convention of phi -- are pinned by the GPU parity tests instead.)
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from conftest import load_kat
from refmath import R3_quad, massless_volume, minkowski2, two_body_p

MUTATIONS = {
    "lambda_drops_term": ("(g + (real)2 * a + (real)2 * b)", "(g + (real)2 * a)"),
    "subsystem_sign": ("real sub[4] = {sqrt(q * q + Mk[k] * Mk[k]), q * dir[0],",
                       "real sub[4] = {sqrt(q * q + Mk[k] * Mk[k]), -q * dir[0],"),
    "mass_index": ("Mk[k] = D->mu[k - 1] + r[k - 1] * D->T;", "Mk[k] = D->mu[k - 1] + r[k] * D->T;"),
    "boost_operand": ("real f = qp / (mq * (q[0] + mq)) + v[0] / mq;",
                      "real f = qp / (mq * (q[0] + mq)) + q[0] / mq;"),
    "gap_formula": ("gap[k] = D->T * (r[k] - r[k - 1]);", "gap[k] = D->T * r[k];"),
    "weight_constant": ("for (int i = 0; i < n - 2; ++i) c *= (real)2 * T;",
                        "for (int i = 0; i < n - 2; ++i) c *= T;"),
    "philox_word": ("uint32_t n0 = hi1 ^ c[1] ^ k[0];", "uint32_t n0 = hi0 ^ c[1] ^ k[0];"),
    "sort_order": ("while (i > 0 && y[i - 1] > v)", "while (i > 0 && y[i - 1] < v)"),
    "two_body_mass": ("pk[k] = sqrt(lam) / ((real)2 * Mk[k + 1]);", "pk[k] = sqrt(lam) / ((real)2 * Mk[k]);"),
    "cos_theta": ("real c = (real)2 * u[n - 2 + 2 * j] - (real)1;", "real c = u[n - 2 + 2 * j] - (real)1;"),
    "bw_width": ("real xb = m0b * m0b - s23, yb = m0b * Gb", "real xb = m0b * m0b - s23, yb = m0b * Ga"),
    "dalitz_pair": ("dalitz_2bw(invariant_mass2(p[0], p[1]), invariant_mass2(p[1], p[2]), params);\n        real f = w * me2;",
                    "dalitz_2bw(invariant_mass2(p[0], p[1]), invariant_mass2(p[0], p[2]), params);\n        real f = w * me2;"),
}


def _pin_philox():
    return all(oracle.philox4x32_10(r[0:4], r[4:6]) == tuple(r[6:10]) for r in load_kat("philox4x32_10_kat.txt"))


def _pin_two_body():
    M, m1, m2 = 5.2795, 3.0969, 0.4937
    p, w = oracle.generate(M, (m1, m2), 50, seed=3)
    pst = two_body_p(M, m1, m2)
    return bool(np.allclose(np.sqrt((p[0, 1:] ** 2).sum(axis=0)), pst, rtol=1e-12)
                and np.allclose(w, math.pi * pst / M, rtol=1e-12))


def _events(n):
    rng = np.random.default_rng(n)
    Md, masses = workloads.random_decay(rng, n)
    p, w = oracle.generate(Md, masses, 300, seed=n)
    return Md, masses, p, w


def _pin_conservation(n):
    Md, masses, p, _ = _events(n)
    tot = p.sum(axis=0)
    return bool(np.allclose(tot[0], Md, rtol=0, atol=1e-12 * Md) and np.allclose(tot[1:], 0, rtol=0, atol=1e-12 * Md))


def _pin_on_shell(n):
    Md, masses, p, _ = _events(n)
    return all(np.allclose(minkowski2(p[i].T), masses[i] ** 2, rtol=0, atol=1e-10 * Md * Md) for i in range(n))


def _pin_weight_lambda(n):
    Md, masses, p, w = _events(n)
    C = math.pi ** (n - 1) * (2 * (Md - sum(masses))) ** (n - 2) / math.factorial(n - 2) / Md
    for e in range(0, 300, 37):
        cum = p[:, :, e].cumsum(axis=0)
        Mk = [None, masses[0]] + [math.sqrt(max(minkowski2(cum[k - 1]), 0.0)) for k in range(2, n)] + [Md]
        prod = 1.0
        for k in range(1, n):
            prod *= two_body_p(Mk[k + 1], Mk[k], masses[k])
        if not abs(w[e] - C * prod) <= 1e-9 * abs(C * prod) + 1e-300:
            return False
    return True


def _pin_massless_volume(n):
    _, w = oracle.generate(10.0, (0.0,) * n, 60_000, seed=7 + n)
    return bool(abs(w.mean() - massless_volume(n, 10.0)) < 4 * w.std(ddof=1) / math.sqrt(len(w)))


def _pin_isotropy():
    from scipy import stats
    p, _ = oracle.generate(10.0, (0.1, 0.2, 0.3), 40_000, seed=2)
    d = p[2]
    cz = d[3] / np.sqrt(d[1] ** 2 + d[2] ** 2 + d[3] ** 2)
    return bool(stats.kstest(cz, "uniform", args=(-1, 2)).pvalue > 1e-3)


def _pin_massive_volume():
    cfg = workloads.B_TO_JPSI_K_PI
    _, w = oracle.generate(cfg["M"], cfg["masses"], 100_000, seed=5)
    return bool(abs(w.mean() - R3_quad(cfg["M"], cfg["masses"])) < 4 * w.std(ddof=1) / math.sqrt(len(w)))


def _pin_dalitz_me():
    dz = workloads.D0_DALITZ
    pz, wz = oracle.generate(dz["M"], dz["masses"], 20_000, seed=4)
    s12 = minkowski2((pz[0] + pz[1]).T)
    s23 = minkowski2((pz[1] + pz[2]).T)
    m0a, Ga, m0b, Gb, cm, ca = dz["params"]
    c = cm * complex(math.cos(ca), math.sin(ca))
    me2 = np.abs(1 / (m0a ** 2 - s12 - 1j * m0a * Ga) + c / (m0b ** 2 - s23 - 1j * m0b * Gb)) ** 2
    sums = oracle.integrate_sums(dz["M"], dz["masses"], 20_000, seed=4, me=1, params=dz["params"])
    return bool(abs(sums[0] - float((wz * me2).sum())) <= 1e-10 * abs(sums[0]))


PINS = {"philox_kat": _pin_philox, "two_body": _pin_two_body, "isotropy": _pin_isotropy,
        "massive_volume": _pin_massive_volume, "dalitz_me": _pin_dalitz_me}
for _n in (3, 5, 8):
    PINS[f"conservation_{_n}"] = (lambda n: lambda: _pin_conservation(n))(_n)
    PINS[f"on_shell_{_n}"] = (lambda n: lambda: _pin_on_shell(n))(_n)
    PINS[f"weight_lambda_{_n}"] = (lambda n: lambda: _pin_weight_lambda(n))(_n)
for _n in (3, 5):
    PINS[f"massless_volume_{_n}"] = (lambda n: lambda: _pin_massless_volume(n))(_n)


def pins() -> list[str]:
    """Run the fast pins against the current oracle library; return the names that fail (a
    pin that raises -- NaN, division by zero -- has caught the mistake too)."""
    failed = []
    with np.errstate(all="ignore"):
        for name, fn in PINS.items():
            try:
                ok = fn()
            except (ArithmeticError, ValueError, FloatingPointError):
                ok = False
            if not ok:
                failed.append(name)
    return failed


def test_unmutated_oracle_passes_the_fast_pins():
    assert pins() == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = oracle.source()
    assert src.count(old) == 1, name
    so = oracle.compile_variant(src.replace(old, new), str(tmp_path / f"mut_{name}.so"))
    with oracle.variant(so):
        failed = pins()
    assert failed, f"mutation {name} passed every pin"
