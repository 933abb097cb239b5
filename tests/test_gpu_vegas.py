"""VEGAS over the Raubold-Lynch variables (section 3, self-adaptive importance sampling;
section 4.1) on the GPU against the oracle's VEGAS, same seeds, same draws, in both FP64
arithmetics of the library (double-float, the default, and native FP64).

The first iteration uses the uniform grid on both sides, so its estimate and variance agree to
FP64 reduction-order rounding.  Later iterations sample through refined grids; the GPU's bin
sums of f^2 are 64-bit fixed point relative to the iteration's largest f^2 (about 2^-40 of it
per point), so its grid differs from the oracle's by that much and the later estimates by a
comparable relative amount: the tolerances below allow 1e-8 (1e-7 for the narrow peak)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1711_05683_b300 as hp  # noqa: E402
import workloads  # noqa: E402
from refmath import R3_quad, dalitz_me_integral_quad  # noqa: E402

pytestmark = pytest.mark.gpu
D0 = workloads.D0_DALITZ
NARROW = (0.892, 0.005, 1.02, 0.004, 0.0, 1.2)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_05683_b300 import build as hp_build
    hp_build.build()
    torch.cuda.set_device(0)


def _case(name):
    rng = np.random.default_rng(77)
    if name == "dalitz":
        return D0["M"], D0["masses"], dict(me=1, params=D0["params"]), 20_011, 4, 50, 1e-8
    if name == "narrow_peak":
        return D0["M"], D0["masses"], dict(me=1, params=NARROW), 30_001, 5, 50, 1e-7
    if name == "plain_mc":
        return D0["M"], D0["masses"], dict(me=1, params=D0["params"]), 6_145, 3, 1, 1e-12
    if name == "flat_n5":
        M, m = workloads.random_decay(rng, 5)
        return M, m, {}, 9_000, 3, 16, 1e-8
    if name == "flat_n10":
        M, m = workloads.random_decay(rng, 10)
        return M, m, {}, 4_100, 3, 8, 1e-8
    raise KeyError(name)


@pytest.fixture(params=["df", "native"])
def arith(request):
    saved = hp.get_fp64_arith()
    hp.set_fp64_arith(hp.FP64_NATIVE if request.param == "native" else hp.FP64_DOUBLE_FLOAT)
    yield request.param
    hp.set_fp64_arith(saved)


@pytest.mark.parametrize("name", ["dalitz", "narrow_peak", "plain_mc", "flat_n5", "flat_n10"])
def test_vegas_matches_oracle(name, arith):
    M, m, me, calls, iters, bins, tol = _case(name)
    g = hp.vegas(M, m, 11, calls, iters, bins=bins, **me)
    r = oracle.vegas(M, m, 11, calls, iters, bins=bins, **me)
    np.testing.assert_allclose(g["est"][0], r["est"][0], rtol=1e-12)
    np.testing.assert_allclose(g["var"][0], r["var"][0], rtol=1e-9)
    np.testing.assert_allclose(g["est"], r["est"], rtol=tol)
    np.testing.assert_allclose(g["var"], r["var"], rtol=100 * tol)
    np.testing.assert_allclose(g["grid"], r["grid"], rtol=0, atol=tol)
    np.testing.assert_allclose(g["mean"], r["mean"], rtol=tol)
    np.testing.assert_allclose(g["sigma"], r["sigma"], rtol=100 * tol)
    assert np.all(g["grid"][:, 0] == 0.0) and np.all(g["grid"][:, -1] == 1.0)
    assert np.all(np.diff(g["grid"], axis=1) > 0)


def test_vegas_two_body_is_exact(arith):
    """n = 2: F is the constant R_2 = pi p*/M on the (cos theta, phi) square.  With one bin
    (J = 1) every iteration returns it to rounding; with a grid the first (uniform) one does,
    and the later ones average J = prod K (g[b+1] - g[b]), whose mean is 1."""
    M, m = 3.0, (0.5, 1.1)
    pstar = math.sqrt((M * M - (m[0] + m[1]) ** 2) * (M * M - (m[0] - m[1]) ** 2)) / (2 * M)
    plain = hp.vegas(M, m, 5, 5_000, 3, bins=1)
    np.testing.assert_allclose(plain["est"], math.pi * pstar / M, rtol=1e-13)
    g = hp.vegas(M, m, 5, 5_000, 3, bins=10)
    np.testing.assert_allclose(g["est"][0], math.pi * pstar / M, rtol=1e-13)
    r = oracle.vegas(M, m, 5, 5_000, 3, bins=10)
    np.testing.assert_allclose(g["est"], r["est"], rtol=1e-8)


def test_vegas_is_deterministic(arith):
    a = hp.vegas(D0["M"], D0["masses"], 3, 50_000, 3, bins=40, me=1, params=D0["params"])
    b = hp.vegas(D0["M"], D0["masses"], 3, 50_000, 3, bins=40, me=1, params=D0["params"])
    assert np.array_equal(a["est"], b["est"]) and np.array_equal(a["var"], b["var"])
    assert np.array_equal(a["grid"], b["grid"])


def test_vegas_large_sample_against_quadrature(arith):
    """2^24 + 3 points per iteration (32769 warp tiles of 512 points, 33 segments, a ragged
    last tile): the first iteration equals
    the oracle's on the same draws; the combined result matches quadrature of the Dalitz
    integral within 5 sigma and the narrow peak's per-iteration error drops by 10x."""
    calls = (1 << 24) + 3
    g = hp.vegas(D0["M"], D0["masses"], 21, calls, 5, bins=64, me=1, params=D0["params"])
    exact, _ = dalitz_me_integral_quad(D0["M"], D0["masses"], D0["params"])
    assert abs(g["mean"] - exact) < 5 * g["sigma"], (g["mean"], exact, g["sigma"])
    assert g["chi2_dof"] < 5.0
    r1 = oracle.vegas(D0["M"], D0["masses"], 21, calls, 1, bins=64, me=1, params=D0["params"])
    np.testing.assert_allclose(g["est"][0], r1["est"][0], rtol=1e-12)
    np.testing.assert_allclose(g["var"][0], r1["var"][0], rtol=1e-9)
    n = hp.vegas(D0["M"], D0["masses"], 22, 1 << 22, 6, bins=100, me=1, params=NARROW)
    assert math.sqrt(n["var"][-1]) < math.sqrt(n["var"][0]) / 10
    exact_n, _ = dalitz_me_integral_quad(D0["M"], D0["masses"], NARROW)
    assert abs(n["mean"] - exact_n) < 5 * n["sigma"]
    f = hp.vegas(D0["M"], D0["masses"], 23, 1 << 22, 3, bins=32)
    assert abs(f["mean"] - R3_quad(D0["M"], D0["masses"])) < 5 * f["sigma"]


@pytest.mark.parametrize("kw", [dict(bins=0), dict(bins=257), dict(calls=1), dict(skip=3),
                                dict(iterations=0), dict(alpha=-1.0), dict(n10_bins=256)])
def test_vegas_rejects_bad_arguments(kw):
    kw = dict(kw)
    M, m = D0["M"], D0["masses"]
    args = dict(calls=1000, iterations=3, bins=10, alpha=1.5, skip=1)
    if "n10_bins" in kw:
        M, m = workloads.random_decay(np.random.default_rng(1), 10)
        args["bins"] = kw.pop("n10_bins")  # (3n-4)(bins+1) = 26 * 257 > 6144 edges
    args.update(kw)
    calls, iters = args.pop("calls"), args.pop("iterations")
    with pytest.raises(hp.HydraError, match="INVALID_ARG"):
        hp.vegas(M, m, 1, calls, iters, **args)
