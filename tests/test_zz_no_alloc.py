"""The integral entry point that allocates no memory, through the C ABI.

hydra_phsp_integrate_noalloc serves callers that cannot call cudaMalloc (processes that
forbid device allocation after start-up, plug-ins whose host owns all device memory, loops
where an allocation's device-wide synchronization would stall other streams).  Its scratch
is a fixed static device array inside the library.  This test calls it twice in a row on
several workloads and checks each result against the allocating hydra_phsp_integrate, with
the tolerance the parity tests use for FP64 sums (1e-12 relative); the two share kernels
and reduction order, so in practice they agree bit for bit.  The file is named to be
collected last.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")

import paper_1711_05683_b300 as hp  # noqa: E402
import workloads  # noqa: E402

pytestmark = pytest.mark.gpu

REL = 1e-12


def _call(fn, M, masses, nev, seed, kin, me, params, offset=0):
    res = hp.Integral()
    m = (ctypes.c_double * len(masses))(*masses)
    par = (ctypes.c_double * max(1, len(params)))(*params)
    rc = fn(float(M), len(masses), m, nev, seed, offset, kin, me, par, len(params), ctypes.byref(res),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, res


def _close(a, b):
    return abs(a - b) <= REL * max(abs(a), abs(b))


def test_noalloc_integral_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_05683_b300 import build as hp_build
    hp_build.build()
    torch.cuda.set_device(0)
    L = hp.lib()
    d = workloads.D0_DALITZ
    cases = [
        (d["M"], d["masses"], 5_000_000, d["seed"], hp.F32, hp.ME_DALITZ_2BW, d["params"], 0),
        (d["M"], d["masses"], 123_457, 11, hp.F64, hp.ME_DALITZ_2BW, d["params"], 2 ** 32 - 10),
        (10.0, workloads.sweep_masses(5, True), 1_000_003, 3, hp.F64, hp.ME_FLAT, (), 0),
        (10.0, workloads.sweep_masses(9, False), 2 ** 26 + 4099, 5, hp.F32, hp.ME_FLAT, (), 0),
    ]
    for _ in range(2):  # two calls in a row: the shared static scratch keeps the last contents
        for M, masses, nev, seed, kin, me, params, off in cases:
            rc_a, ref = _call(L.hydra_phsp_integrate, M, masses, nev, seed, kin, me, params, off)
            rc_b, got = _call(L.hydra_phsp_integrate_noalloc, M, masses, nev, seed, kin, me, params, off)
            assert rc_a == 0 and rc_b == 0, L.hydra_last_error()
            assert got.n == ref.n == nev
            for field in ("mean", "var_mean", "sum_f", "sum_f2", "sum_w", "sum_w2"):
                assert _close(getattr(got, field), getattr(ref, field)), (field, nev, got.as_dict(),
                                                                          ref.as_dict())


def test_noalloc_rejects_counts_beyond_its_fixed_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = hp.lib()
    d = workloads.D0_DALITZ
    rc, _ = _call(L.hydra_phsp_integrate_noalloc, d["M"], d["masses"], 2 ** 32 + 1, 1, hp.F32,
                  hp.ME_DALITZ_2BW, d["params"])
    assert hp.STATUS[rc] == "HYDRA_ERR_INVALID_ARG"
    assert "2^32" in L.hydra_last_error().decode()
