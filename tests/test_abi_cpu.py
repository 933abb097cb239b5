"""The C ABI without a GPU: the library loads, exports every declared symbol, and rejects
bad arguments with the documented status codes before touching the device."""
import ctypes
import math

import numpy as np

import pytest

import oracle
import paper_1711_05683_b300 as hp
from paper_1711_05683_b300 import build as hp_build


@pytest.fixture(scope="module")
def L():
    hp_build.build()
    return hp.lib()


def _dbl(v):
    return (ctypes.c_double * len(v))(*v)


def test_exports_every_declared_symbol(L):
    names = hp.header_functions()
    assert "hydra_phsp_generate" in names and "hydra_phsp_integrate" in names
    for name in names:
        assert hasattr(L, name), name


def test_status_strings(L):
    for code, name in hp.STATUS.items():
        assert L.hydra_status_string(code).decode() == name


def test_volume_factor_matches_oracle(L):
    for M, masses in [(10.0, (0.0,) * 10), (5.2795, (3.0969, 0.4937, 0.1396)), (2.0, (0.1, 0.2))]:
        assert hp.volume_factor(M, masses) == pytest.approx(oracle.volume_factor(M, masses), rel=1e-15)


def _gen(L, M=5.0, n=3, masses=None, nevents=8, seed=1, offset=0, dtype=0, out=16, ld=8, w=16):
    masses = masses if masses is not None else [0.1] * n
    return L.hydra_phsp_generate(M, n, _dbl(masses) if masses else None, nevents, seed, offset,
                                 dtype, ctypes.c_void_p(out) if out is not None else None, ld,
                                 ctypes.c_void_p(w) if w is not None else None, None)


@pytest.mark.parametrize("kwargs,status", [
    (dict(n=1, masses=[0.1]), "HYDRA_ERR_UNSUPPORTED_N"),
    (dict(n=11, masses=[0.1] * 11), "HYDRA_ERR_UNSUPPORTED_N"),
    (dict(M=0.0), "HYDRA_ERR_INVALID_ARG"),
    (dict(M=-1.0), "HYDRA_ERR_INVALID_ARG"),
    (dict(M=math.inf), "HYDRA_ERR_INVALID_ARG"),
    (dict(M=math.nan), "HYDRA_ERR_INVALID_ARG"),
    (dict(masses=[0.1, -0.1, 0.1]), "HYDRA_ERR_INVALID_ARG"),
    (dict(masses=[0.1, math.nan, 0.1]), "HYDRA_ERR_INVALID_ARG"),
    (dict(M=0.3, masses=[0.1, 0.1, 0.1]), "HYDRA_ERR_BELOW_THRESHOLD"),
    (dict(M=0.2, masses=[0.1, 0.1, 0.1]), "HYDRA_ERR_BELOW_THRESHOLD"),
    (dict(dtype=7), "HYDRA_ERR_INVALID_ARG"),
    (dict(out=None), "HYDRA_ERR_INVALID_ARG"),
    (dict(w=None), "HYDRA_ERR_INVALID_ARG"),
    (dict(ld=4), "HYDRA_ERR_INVALID_ARG"),
    (dict(out=20), "HYDRA_ERR_MISALIGNED"),
    (dict(w=24), "HYDRA_ERR_MISALIGNED"),
    (dict(ld=10), "HYDRA_ERR_MISALIGNED"),
    (dict(offset=2 ** 64 - 4), "HYDRA_ERR_INVALID_ARG"),
])
def test_generate_rejects(L, kwargs, status):
    rc = _gen(L, **kwargs)
    assert hp.STATUS[rc] == status, L.hydra_last_error()
    assert L.hydra_last_error().decode() != ""


def test_generate_zero_events_is_noop(L):
    assert _gen(L, nevents=0, out=None, w=None, ld=0) == 0


def test_integrate_rejects(L):
    res = hp.Integral()
    par = _dbl([0.892, 0.05, 1.02, 0.004, 0.5, 1.2])
    cases = [
        (dict(n=4, masses=[0.1] * 4, me=1, npar=6), "HYDRA_ERR_UNSUPPORTED_N"),
        (dict(me=1, npar=5), "HYDRA_ERR_INVALID_ARG"),
        (dict(me=9), "HYDRA_ERR_INVALID_ARG"),
        (dict(nevents=0), "HYDRA_ERR_INVALID_ARG"),
        (dict(M=0.25), "HYDRA_ERR_BELOW_THRESHOLD"),
        (dict(dtype=3), "HYDRA_ERR_INVALID_ARG"),
    ]
    for kw, status in cases:
        n = kw.get("n", 3)
        masses = kw.get("masses", [0.1] * n)
        rc = L.hydra_phsp_integrate(kw.get("M", 2.0), n, _dbl(masses), kw.get("nevents", 100), 1, 0,
                                    kw.get("dtype", 0), kw.get("me", 0), par, kw.get("npar", 0),
                                    ctypes.byref(res), None)
        assert hp.STATUS[rc] == status, (kw, L.hydra_last_error())
    rc = L.hydra_phsp_integrate(2.0, 3, _dbl([0.1] * 3), 100, 1, 0, 0, 0, par, 0, None, None)
    assert hp.STATUS[rc] == "HYDRA_ERR_INVALID_ARG"


def test_draws_rejects(L):
    assert hp.STATUS[L.hydra_phsp_draws(11, 10, 1, 0, ctypes.c_void_p(16), 16, None)] == "HYDRA_ERR_UNSUPPORTED_N"
    assert hp.STATUS[L.hydra_phsp_draws(3, 10, 1, 0, None, 16, None)] == "HYDRA_ERR_INVALID_ARG"
    assert hp.STATUS[L.hydra_phsp_draws(3, 10, 1, 0, ctypes.c_void_p(16), 8, None)] == "HYDRA_ERR_INVALID_ARG"
    assert L.hydra_phsp_draws(3, 0, 1, 0, None, 0, None) == 0


def test_launch_config_validation(L):
    b, e = ctypes.c_int(), ctypes.c_int()
    assert L.hydra_get_launch_config(0, 3, 0, ctypes.byref(b), ctypes.byref(e)) == 0
    assert b.value % 32 == 0 and e.value in (1, 2, 4)
    bad = [(2, 3, 0, 256, 1, "HYDRA_ERR_INVALID_ARG"), (0, 11, 0, 256, 1, "HYDRA_ERR_UNSUPPORTED_N"),
           (0, 3, 5, 256, 1, "HYDRA_ERR_INVALID_ARG"), (0, 3, 0, 100, 1, "HYDRA_ERR_INVALID_ARG"),
           (0, 3, 0, 1024, 1, "HYDRA_ERR_INVALID_ARG"), (1, 3, 1, 256, 3, "HYDRA_ERR_INVALID_ARG")]
    for kind, n, dt, block, ept, status in bad:
        assert hp.STATUS[L.hydra_set_launch_config(kind, n, dt, block, ept)] == status
    assert L.hydra_set_launch_config(1, 5, 1, 128, 2) == 0
    assert L.hydra_get_launch_config(1, 5, 1, ctypes.byref(b), ctypes.byref(e)) == 0
    assert (b.value, e.value) == (128, 2)


def test_fp64_arith_switch(L):
    assert L.hydra_get_fp64_arith() == 1
    assert hp.STATUS[L.hydra_set_fp64_arith(7)] == "HYDRA_ERR_INVALID_ARG"
    assert L.hydra_set_fp64_arith(0) == 0 and L.hydra_get_fp64_arith() == 0
    assert L.hydra_set_fp64_arith(1) == 0 and L.hydra_get_fp64_arith() == 1


def test_fp32_lambda_switch(L):
    assert L.hydra_get_fp32_lambda() == 0
    assert hp.STATUS[L.hydra_set_fp32_lambda(2)] == "HYDRA_ERR_INVALID_ARG"
    assert L.hydra_set_fp32_lambda(1) == 0 and L.hydra_get_fp32_lambda() == 1
    assert L.hydra_set_fp32_lambda(0) == 0 and L.hydra_get_fp32_lambda() == 0


def test_batch_shape_validation(L):
    block, ept = hp.get_batch_shape("f32")
    assert block == 256 and ept[2:] == [2, 4, 4, 4, 4, 2, 2, 2, 2]
    with pytest.raises(hp.HydraError):
        hp.set_batch_shape("f32", 384, ept)            # block not offered
    with pytest.raises(hp.HydraError):
        hp.set_batch_shape("f32", 256, [4] * 11)       # four events per thread only up to n = 6
    with pytest.raises(hp.HydraError):
        hp.set_batch_shape("f64", 256, [1] * 11)       # FP64 tiles take two
    hp.set_batch_shape("f32", 512, [1] * 11)
    assert hp.get_batch_shape("f32") == (512, [2, 2] + [1] * 9)
    hp.set_batch_shape("f32", block, ept)
    assert hp.get_batch_shape("f64") == (256, [2] * 11)


def test_batch_run_validates_before_any_launch(L):
    """Errors found on the host, each request's status set; no CUDA call is needed to reach
    them (this runs without a GPU)."""
    class _E(Exception):
        pass

    class hp_:  # the C ABI directly, on the legacy default stream (no torch CUDA state here)
        HydraError = _E

        @staticmethod
        def batch_run(t, budget):
            rc = L.hydra_phsp_batch_run(ctypes.c_void_p(t.ctypes.data if len(t) else None), len(t), budget, None)
            if rc:
                raise _E(f"{hp.STATUS[rc]}: {L.hydra_last_error().decode()}")
    t = np.zeros(3, dtype=hp.batch_request_dtype())
    for i in range(3):
        t[i]["kind"], t[i]["n"], t[i]["M"], t[i]["nevents"], t[i]["seed"] = hp.REQ_GENERATE, 3, 5.0, 100, i
        t[i]["masses"][:3] = (0.1, 0.2, 0.3)
    t[1]["masses"][:3] = (2.0, 2.0, 2.0)  # below threshold
    with pytest.raises(hp_.HydraError) as e:
        hp_.batch_run(t, 1 << 30)
    assert "request 1" in str(e.value) and list(t["status"]) == [0, 2, 0]
    t[1]["masses"][:3] = (0.1, 0.2, 0.3)
    t[2]["dtype"] = hp.F64
    with pytest.raises(hp_.HydraError):
        hp_.batch_run(t, 1 << 30)            # mixed precisions
    assert t["status"][2] == 1
    t[2]["dtype"] = hp.F32
    t[0]["dest"] = hp.DEST_DEVICE             # device destination without buffers
    with pytest.raises(hp_.HydraError):
        hp_.batch_run(t, 1 << 30)
    t[0]["dest"] = hp.DEST_NONE
    t[2]["kind"], t[2]["me"] = hp.REQ_INTEGRATE, hp.ME_DALITZ_2BW  # Dalitz needs its 6 params finite: zeros are fine
    t[2]["params"][:6] = (0.892, 0.05, 1.02, 0.004, 0.5, float("nan"))
    with pytest.raises(hp_.HydraError):
        hp_.batch_run(t, 1 << 30)
    t[2]["params"][5] = 1.2
    with pytest.raises(hp_.HydraError) as e:
        hp_.batch_run(t, 1 << 20)            # budget below what the runner needs
    assert "budget" in str(e.value)
    with pytest.raises(hp_.HydraError):
        hp_.batch_run(t[:0], 1 << 30)        # no requests


def test_op_rate_probe_rejects_bad_arguments(L):
    """Host-side checks of hydra_probe_op_rate (no GPU needed to reach them)."""
    r = ctypes.c_double()
    assert hp.STATUS[L.hydra_probe_op_rate(0, 0, 0, ctypes.byref(r), None)] == "HYDRA_ERR_INVALID_ARG"  # iterations
    assert hp.STATUS[L.hydra_probe_op_rate(0, 0, 10, None, None)] == "HYDRA_ERR_INVALID_ARG"            # no output
    assert hp.STATUS[L.hydra_probe_op_rate(7, 0, 10, ctypes.byref(r), None)] == "HYDRA_ERR_INVALID_ARG"  # arithmetic
