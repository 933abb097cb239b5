"""Unit tier for the double-float device primitives of the FP64 path (phsp_df.cuh), run by a
test probe on the GPU and compared with exact values: the integer-to-double-float conversions
exactly (edge inputs 0, 255, 256, 2^31 - 1, 2^31, 2^32 - 1 and random ones), sin/cos of
2 pi (x + 1/2) 2^-32 to 4e-14 absolute (double-float precision, ~2^-46, the product and sum
of the angle-addition step) against 30-digit values (table edges, octant and quadrant
boundaries), v 2^-64 to 2^-46 relative, the weight product (mantissa and binary exponent)
to 1e-14 relative, including factors at the FP32 range limits, a subnormal one and zero, and
the double-float to double conversions (the nearest double for normal parts; zeros exact in
the weight's conversion, within 2^-125 in the stored kinematics')."""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mpmath = pytest.importorskip("mpmath")

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    so = tmp_path_factory.mktemp("probe") / "df_probe.so"
    src = os.path.join(ROOT, "tests", "gpu_probes", "df_primitives_probe.cu")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-fmad=false",
                           "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
                           "-I", os.path.join(ROOT, "paper_1711_05683_b300", "csrc"),
                           "-I", os.path.join(ROOT, "include"), "-o", str(so), src])
    return ctypes.CDLL(str(so))


EDGES32 = [0, 1, 2, 255, 256, 257, (1 << 21) - 1, 1 << 21, (1 << 29) - 1, 1 << 29, (1 << 30) - 1, 1 << 30,
           (1 << 31) - 1, 1 << 31, (1 << 31) + 1, 3 << 30, (1 << 32) - 2, (1 << 32) - 1]


def _u32_inputs():
    rng = np.random.default_rng(17)
    return EDGES32 + [int(v) for v in rng.integers(0, 1 << 32, size=2000, dtype=np.uint64)]


def _run_u32(probe, op, xs):
    x = (ctypes.c_uint32 * len(xs))(*xs)
    out = (ctypes.c_double * (2 * len(xs)))()
    assert probe.probe_df_u32(op, x, len(xs), out) == 0
    return [Fraction(out[2 * i]) + Fraction(out[2 * i + 1]) for i in range(len(xs))]


def test_integer_conversions_are_exact(probe):
    xs = _u32_inputs()
    half = Fraction(1, 2)
    assert _run_u32(probe, 0, xs) == [(x + half) / 2 ** 31 for x in xs]          # 1 + cos(theta)
    assert _run_u32(probe, 1, xs) == [(x - 2 ** 31 + half) / 2 ** 31 for x in xs]  # cos(theta)
    assert _run_u32(probe, 2, xs) == [Fraction(x) for x in xs]
    assert _run_u32(probe, 3, xs) == [x + half for x in xs]


def test_sincos_of_the_phi_draw(probe):
    xs = _u32_inputs()
    # every table entry's first and last argument
    xs += [k << 21 for k in range(0, 2048, 7)] + [(k << 21) - 1 for k in range(1, 2048, 7)]
    x = (ctypes.c_uint32 * len(xs))(*xs)
    out = (ctypes.c_double * (4 * len(xs)))()
    assert probe.probe_df_sincos(x, len(xs), out) == 0
    mpmath.mp.dps = 30
    worst = 0.0
    for i, v in enumerate(xs):
        phi = 2 * mpmath.pi * (mpmath.mpf(v) + mpmath.mpf(0.5)) / 2 ** 32
        s = mpmath.mpf(out[4 * i]) + mpmath.mpf(out[4 * i + 1])
        c = mpmath.mpf(out[4 * i + 2]) + mpmath.mpf(out[4 * i + 3])
        worst = max(worst, float(abs(s - mpmath.sin(phi))), float(abs(c - mpmath.cos(phi))))
    assert worst < 4e-14, worst


def test_fixed_point_fraction(probe):
    rng = np.random.default_rng(3)
    vs = [0, 1, 2, (1 << 16) - 1, 1 << 40, (1 << 63) - 1, 1 << 63, (1 << 64) - 1]
    vs += [int(v) for v in rng.integers(0, 1 << 63, size=500, dtype=np.uint64)]
    vs += [int(v) >> int(k) for v, k in zip(rng.integers(1 << 40, 1 << 62, size=200, dtype=np.uint64),
                                               rng.integers(0, 60, size=200))]
    arr = (ctypes.c_uint64 * len(vs))(*vs)
    out = (ctypes.c_double * (2 * len(vs)))()
    assert probe.probe_df_frac64(arr, len(vs), out) == 0
    for i, v in enumerate(vs):
        got = Fraction(out[2 * i]) + Fraction(out[2 * i + 1])
        exact = Fraction(v, 1 << 64)
        if v == 0:
            assert got == 0
        else:
            assert abs(got - exact) <= exact * Fraction(1, 1 << 46), v
            assert got <= exact  # truncation, never above


def _df_split(x: float):
    hi = np.float32(x)
    lo = np.float32(x - float(hi))
    return float(hi), float(lo)


@pytest.mark.parametrize("factors", [
    [0.37, 1.9, 2.5e-3, 4.4, 0.91, 1.2e-2, 7.0, 0.5, 3.3],
    [1e-12, 3e-11, 5e-13, 2e-12, 8e-12, 1e-10, 4e-13, 6e-12, 1e-11],  # product ~1e-104: below FP32
    [3.0e37, 2.5, 1.0e-37, 4.0],                                        # FP32 range ends
    [0.5, 0.0, 3.0],                                                    # a tie in the mass draws: zero
    [1.0e-40, 2.0],                                                     # an FP32 subnormal factor
])
def test_weight_product(probe, factors):
    pairs = [_df_split(f) for f in factors]
    p = (ctypes.c_float * (2 * len(pairs)))(*[v for pr in pairs for v in pr])
    out = (ctypes.c_double * 1)()
    c = 0.123456789
    assert probe.probe_df_weight(p, len(pairs), ctypes.c_double(c), out) == 0
    exact = Fraction(c)
    for hi, lo in pairs:
        exact *= Fraction(hi) + Fraction(lo)
    if exact == 0:
        assert out[0] == 0.0
    else:
        assert abs(Fraction(out[0]) - exact) <= abs(exact) * Fraction(1, 10 ** 14)



def _normal_or_zero(v: float) -> bool:
    return v == 0.0 or abs(v) >= 2.0 ** -126


def test_double_float_to_double(probe):
    rng = np.random.default_rng(29)
    pairs = [_df_split(float(v)) for v in rng.standard_normal(3000) * 10.0 ** rng.integers(-30, 30, size=3000)]
    # low parts at the edge of the pair's range, exact halfway cases of the FP64 rounding, and
    # powers of two with a negative low part (the sum drops below the binade of hi)
    for hi in (1.0, -3.0, 2.0 ** 100, 0.75, 5.9e-36):
        u = float(np.spacing(np.float32(hi)))
        pairs += [(hi, u / 2), (hi, -u / 2), (hi, u / 4), (hi, -u / 4), (hi, u * 2.0 ** -29), (hi, -u * 2.0 ** -30)]
    zeros = [(0.0, 0.0), (-0.0, 0.0), (0.0, -0.0), (-0.0, -0.0), (1.0e-39, 0.0)]
    pairs += zeros + [(3.0, 0.0), (-7.5, -0.0)]
    pairs = [(float(np.float32(h)), float(np.float32(l))) for h, l in pairs]
    p = (ctypes.c_float * (2 * len(pairs)))(*[v for pr in pairs for v in pr])
    out = (ctypes.c_double * (2 * len(pairs)))()
    assert probe.probe_df_to_double(p, len(pairs), out) == 0
    for i, (hi, lo) in enumerate(pairs):
        exact = Fraction(hi) + Fraction(lo)
        fast, exact_conv = out[2 * i], out[2 * i + 1]
        bound = Fraction(2.0 ** -125) + abs(exact) * Fraction(1, 1 << 53)
        if _normal_or_zero(hi) and _normal_or_zero(lo):
            assert exact_conv == float(exact), (hi, lo)  # float(Fraction) is the nearest double
        else:
            assert abs(Fraction(exact_conv) - exact) <= bound, (hi, lo)  # FP32 subnormal parts flush
        if hi != 0.0 and lo != 0.0 and _normal_or_zero(hi) and _normal_or_zero(lo):
            assert fast == float(exact), (hi, lo)
        else:
            assert abs(Fraction(fast) - exact) <= bound, (hi, lo, fast)  # zero / subnormal parts
    for i in range(len(pairs) - len(zeros) - 2, len(pairs) - 2):
        assert out[2 * i + 1] == 0.0  # the weight's conversion keeps a zero exact
