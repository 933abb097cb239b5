"""B300-native phase-space Monte Carlo (Hydra, arXiv:1711.05683, section 4.2).

Thin Python binding of the C ABI in ``include/hydra_phsp.h``: it marshals arguments,
allocates outputs with PyTorch on the current CUDA device and passes the current stream.
Every step of the generator and of the integral runs in the CUDA kernels of
``libhydra_phsp.so``; there is no other implementation here.  If the library is missing
the import fails.

    import paper_1711_05683_b300 as hp
    p, w = hp.generate(5.2795, (3.0969, 0.4937, 0.1396), 100_000, seed=42, dtype="f64")
    # p: [3, 4, ld] (E, px, py, pz) per daughter on the GPU; w: [nevents] weights
    res = hp.integrate(1.865, (0.4937, 0.1396, 0.4937), 10**9, seed=7,
                       me=hp.ME_DALITZ_2BW, params=(0.892, 0.05, 1.02, 0.004, 0.5, 1.2))
"""
from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhydra_phsp.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "hydra_phsp.h")

F32, F64 = 0, 1
ME_FLAT, ME_DALITZ_2BW = 0, 1
KERNEL_GENERATE, KERNEL_INTEGRATE = 0, 1

STATUS = {0: "HYDRA_OK", 1: "HYDRA_ERR_INVALID_ARG", 2: "HYDRA_ERR_BELOW_THRESHOLD",
          3: "HYDRA_ERR_UNSUPPORTED_N", 4: "HYDRA_ERR_MISALIGNED", 5: "HYDRA_ERR_OOM",
          6: "HYDRA_ERR_CUDA", 7: "HYDRA_ERR_TIMEOUT", 8: "HYDRA_ERR_BUSY"}


class HydraError(RuntimeError):
    """A non-OK hydra_status from the C ABI."""

    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Integral(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double), ("var_mean", ctypes.c_double),
                ("sum_f", ctypes.c_double), ("sum_f2", ctypes.c_double),
                ("sum_w", ctypes.c_double), ("sum_w2", ctypes.c_double),
                ("n", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded C library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_1711_05683_b300.build` "
                              "(nvcc, sm_103a) first; there is no fallback implementation")
        L = ctypes.CDLL(LIB_PATH)
        d, i, u64, vp = ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        L.hydra_last_error.restype = ctypes.c_char_p
        L.hydra_status_string.restype = ctypes.c_char_p
        L.hydra_status_string.argtypes = [i]
        L.hydra_phsp_volume_factor.argtypes = [d, i, dp, dp]
        L.hydra_phsp_generate.argtypes = [d, i, dp, u64, u64, u64, i, vp, u64, vp, vp]
        L.hydra_phsp_integrate.argtypes = [d, i, dp, u64, u64, u64, i, i, dp, i,
                                           ctypes.POINTER(Integral), vp]
        L.hydra_phsp_draws.argtypes = [i, u64, u64, u64, vp, u64, vp]
        L.hydra_phsp_generate_host.argtypes = [d, i, dp, u64, u64, u64, i, vp, u64, vp, vp]
        L.hydra_phsp_integrate_noalloc.argtypes = L.hydra_phsp_integrate.argtypes
        L.hydra_set_launch_config.argtypes = [i, i, i, i, i]
        L.hydra_set_fp64_arith.argtypes = [i]
        L.hydra_phsp_generate_boosted.argtypes = [d, i, dp, u64, u64, u64, i, dp, vp, u64, vp, u64, vp, vp]
        L.hydra_phsp_unweight.argtypes = [i, u64, u64, u64, i, vp, d, vp, ctypes.POINTER(u64), dp, vp]
        L.hydra_phsp_gather.argtypes = [i, i, vp, u64, vp, vp, u64, vp, u64, vp, vp]
        L.hydra_phsp_evaluate.argtypes = [i, u64, i, i, dp, i, vp, u64, vp, vp, ctypes.POINTER(Integral), vp]
        L.hydra_phsp_vegas.argtypes = [d, i, dp, u64, i, dp, i, u64, i, i, d, i, dp, dp, dp, dp, vp]
        L.hydra_probe_fma_rate.argtypes = [i, i, dp, vp]
        L.hydra_probe_write_bandwidth.argtypes = [vp, u64, i, dp, vp]
        L.hydra_probe_op_rate.argtypes = [i, i, i, dp, vp]
        L.hydra_get_fp64_arith.restype = i
        L.hydra_set_fp32_lambda.argtypes = [i]
        L.hydra_get_fp32_lambda.restype = i
        L.hydra_batch_create.argtypes = [i, u64, ctypes.POINTER(vp)]
        L.hydra_batch_run.argtypes = [vp, vp, i, i, vp]
        L.hydra_batch_result.argtypes = [vp, i, ctypes.POINTER(Integral)]
        L.hydra_batch_destroy.argtypes = [vp]
        L.hydra_get_launch_config.argtypes = [i, i, i, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.hydra_set_batch_shape.argtypes = [i, i, vp]
        L.hydra_get_batch_shape.argtypes = [i, ctypes.POINTER(i), vp]
        L.hydra_phsp_batch_run.argtypes = [vp, i, ctypes.c_size_t, vp]
        L.hydra_phsp_batch_stats.argtypes = [ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.hydra_server_create.argtypes = [u64, vp, u64, i, i, u64, i, ctypes.POINTER(vp)]
        L.hydra_server_run.argtypes = [vp, vp, i, d, vp, dp, ctypes.POINTER(u64)]
        L.hydra_server_destroy.argtypes = [vp]
        L.hydra_server_set_deadline.argtypes = [vp, d]
        L.hydra_server_start.argtypes = [vp]
        L.hydra_server_submit.argtypes = [vp, vp, ctypes.POINTER(u64)]
        L.hydra_server_poll.argtypes = [vp, u64, d, vp]
        L.hydra_server_stop.argtypes = [vp, d]
        for name in ("hydra_phsp_volume_factor", "hydra_phsp_generate", "hydra_phsp_integrate",
                     "hydra_phsp_draws", "hydra_phsp_generate_host", "hydra_phsp_integrate_noalloc",
                     "hydra_set_launch_config", "hydra_get_launch_config", "hydra_set_fp64_arith",
                     "hydra_phsp_generate_boosted", "hydra_phsp_unweight", "hydra_phsp_gather",
                     "hydra_phsp_evaluate",
                     "hydra_batch_create",
                     "hydra_batch_run", "hydra_batch_result", "hydra_batch_destroy", "hydra_shutdown",
                     "hydra_server_create", "hydra_server_run", "hydra_server_destroy",
                     "hydra_probe_fma_rate", "hydra_probe_write_bandwidth", "hydra_probe_op_rate",
                     "hydra_set_fp32_lambda", "hydra_set_batch_shape", "hydra_get_batch_shape",
                     "hydra_phsp_batch_run", "hydra_phsp_batch_stats", "hydra_server_set_deadline",
                     "hydra_server_start", "hydra_server_submit", "hydra_server_poll", "hydra_server_stop"):
            getattr(L, name).restype = i
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/hydra_phsp.h."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(hydra_\w+)\s*\(", text, re.M)))


def _check(status: int) -> None:
    if status != 0:
        raise HydraError(status, lib().hydra_last_error().decode())


def _dbl(values) -> ctypes.Array:
    vals = [float(v) for v in values]
    return (ctypes.c_double * max(1, len(vals)))(*vals)


def _dtype_code(dtype) -> int:
    if dtype in (F32, "f32", "float32"):
        return F32
    if dtype in (F64, "f64", "float64"):
        return F64
    raise ValueError(f"dtype must be 'f32' or 'f64', got {dtype!r}")


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def volume_factor(M: float, masses) -> float:
    """C_n = pi^(n-1) 2^(n-2) T^(n-2) / ((n-2)! M) (host only)."""
    out = ctypes.c_double()
    _check(lib().hydra_phsp_volume_factor(float(M), len(masses), _dbl(masses), ctypes.byref(out)))
    return out.value


def padded_ld(nevents: int) -> int:
    """Smallest leading dimension >= nevents accepted by generate (a multiple of 4)."""
    return max(4, (int(nevents) + 3) // 4 * 4)


def generate_into(M: float, masses, nevents: int, seed: int, out, weights, *, dtype="f32",
                  event_offset: int = 0, stream=None) -> None:
    """hydra_phsp_generate into caller tensors: out [n, 4, ld] and weights [>= nevents]."""
    code = _dtype_code(dtype)
    ld = int(out.shape[-1]) if nevents else 0
    _check(lib().hydra_phsp_generate(float(M), len(masses), _dbl(masses), int(nevents), int(seed),
                                     int(event_offset), code, ctypes.c_void_p(out.data_ptr()),
                                     ld, ctypes.c_void_p(weights.data_ptr()),
                                     _stream_handle(stream)))


def generate_host_into(M: float, masses, nevents: int, seed: int, out, weights, *, dtype="f32",
                       event_offset: int = 0, stream=None) -> None:
    """hydra_phsp_generate_host into host (CPU, ideally pinned) tensors out [n, 4, ld] and
    weights [>= nevents]; blocks until the events are in host memory."""
    ld = int(out.shape[-1]) if nevents else 0
    _check(lib().hydra_phsp_generate_host(float(M), len(masses), _dbl(masses), int(nevents),
                                          int(seed), int(event_offset), _dtype_code(dtype),
                                          ctypes.c_void_p(out.data_ptr()), ld,
                                          ctypes.c_void_p(weights.data_ptr()),
                                          _stream_handle(stream)))


def generate(M: float, masses, nevents: int, seed: int, *, dtype="f32", event_offset: int = 0,
             stream=None, device=None):
    """Generate nevents weighted phase-space events on the GPU (section 4.2, Listing 4).

    Returns (p, w): p is a [n, 4, ld] tensor (ld = nevents rounded up to a multiple of 4)
    with p[i, c, e] the component c of (E, px, py, pz) of daughter i in event e, and w
    the [nevents] event weights.  Asynchronous on the current stream."""
    import torch
    tdt = torch.float32 if _dtype_code(dtype) == F32 else torch.float64
    ld = padded_ld(nevents)
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    out = torch.empty((len(masses), 4, ld), dtype=tdt, device=dev)
    w = torch.empty((ld,), dtype=tdt, device=dev)
    generate_into(M, masses, nevents, seed, out, w, dtype=dtype, event_offset=event_offset,
                  stream=stream)
    return out, w[:nevents]


def generate_boosted(M: float, masses, nevents: int, seed: int, *, mother=None, mothers=None,
                     dtype="f32", event_offset: int = 0, stream=None):
    """Events of a moving parent (Listing 4, Generate(Mother, ...)): `mother` is one momentum
    (px, py, pz) for all events, or `mothers` a device tensor [3, >= nevents] of per-event
    momenta in the output dtype.  Returns (p, w) like generate()."""
    import torch
    code = _dtype_code(dtype)
    tdt = torch.float32 if code == F32 else torch.float64
    ld = padded_ld(nevents)
    out = torch.empty((len(masses), 4, ld), dtype=tdt, device="cuda")
    w = torch.empty((ld,), dtype=tdt, device="cuda")
    mp = (ctypes.c_double * 3)(*[float(v) for v in mother]) if mother is not None else None
    mptr = ctypes.c_void_p(mothers.data_ptr()) if mothers is not None else None
    mld = int(mothers.shape[-1]) if mothers is not None else 0
    _check(lib().hydra_phsp_generate_boosted(float(M), len(masses), _dbl(masses), int(nevents), int(seed),
                                             int(event_offset), code, mp, mptr, mld,
                                             ctypes.c_void_p(out.data_ptr()), ld,
                                             ctypes.c_void_p(w.data_ptr()), _stream_handle(stream)))
    return out, w[:nevents]


def unweight(n: int, weights, seed: int, *, w_max: float = 0.0, dtype="f32", event_offset: int = 0,
             stream=None):
    """Accept-reject unweighting of the events whose weights are `weights` (device tensor):
    returns (indices of kept events as an int64 device tensor, w_max used)."""
    import torch
    nev = int(weights.shape[0])
    idx = torch.empty(max(1, nev), dtype=torch.int64, device="cuda")
    cnt = ctypes.c_uint64()
    used = ctypes.c_double()
    _check(lib().hydra_phsp_unweight(int(n), nev, int(seed), int(event_offset), _dtype_code(dtype),
                                     ctypes.c_void_p(weights.data_ptr()), float(w_max),
                                     ctypes.c_void_p(idx.data_ptr()), ctypes.byref(cnt), ctypes.byref(used),
                                     _stream_handle(stream)))
    return idx[: cnt.value], used.value


def gather(p, w, indices, *, dtype="f32", stream=None):
    """Compact events p[:, :, indices] (and w[indices]) with the library's gather kernel."""
    import torch
    n, cnt = int(p.shape[0]), int(indices.shape[0])
    ld = padded_ld(cnt)
    dst = torch.empty((n, 4, ld), dtype=p.dtype, device="cuda")
    dw = torch.empty(ld, dtype=p.dtype, device="cuda")
    _check(lib().hydra_phsp_gather(n, _dtype_code(dtype), ctypes.c_void_p(p.data_ptr()), int(p.shape[-1]),
                                   ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(indices.data_ptr()), cnt,
                                   ctypes.c_void_p(dst.data_ptr()), ld, ctypes.c_void_p(dw.data_ptr()),
                                   _stream_handle(stream)))
    return dst[:, :, :cnt], dw[:cnt]


def evaluate(p, w, nevents: int | None = None, *, me: int = ME_FLAT, params=(), dtype="f32",
             want_values: bool = False, stream=None):
    """f = w |ME|^2 on stored events p [n, 4, ld] with weights w (device tensors); returns
    (integral dict, values tensor or None)."""
    import torch
    nev = int(w.shape[0]) if nevents is None else int(nevents)
    n = int(p.shape[0])
    vals = torch.empty(nev, dtype=w.dtype, device="cuda") if want_values else None
    res = Integral()
    _check(lib().hydra_phsp_evaluate(n, nev, _dtype_code(dtype), int(me), _dbl(params), len(params),
                                     ctypes.c_void_p(p.data_ptr()), int(p.shape[-1]),
                                     ctypes.c_void_p(w.data_ptr()),
                                     ctypes.c_void_p(vals.data_ptr()) if vals is not None else None,
                                     ctypes.byref(res), _stream_handle(stream)))
    return res.as_dict(), vals


def vegas(M: float, masses, seed: int, calls: int, iterations: int, *, bins: int = 50, alpha: float = 1.5,
          skip: int = 1, me: int = ME_FLAT, params=(), stream=None):
    """VEGAS estimate of Int |ME|^2 dR_n (section 3, self-adaptive importance sampling) over the
    3n-4 Raubold-Lynch variables, all iterations on the GPU in FP64.  Returns a dict with the
    per-iteration estimates ``est`` and variances ``var``, the combined ``mean``, ``sigma``,
    ``chi2_dof`` and the final ``grid`` [(3n-4), bins+1]."""
    import numpy as np
    n = len(masses)
    D = 3 * n - 4
    est = np.zeros(iterations)
    var = np.zeros(iterations)
    res = np.zeros(3)
    grid = np.zeros((D, bins + 1))
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().hydra_phsp_vegas(float(M), n, _dbl(masses), int(seed), int(me), _dbl(params), len(params),
                                  int(calls), int(iterations), int(bins), float(alpha), int(skip),
                                  est.ctypes.data_as(dp), var.ctypes.data_as(dp), res.ctypes.data_as(dp),
                                  grid.ctypes.data_as(dp), _stream_handle(stream)))
    return {"est": est, "var": var, "mean": float(res[0]), "sigma": float(res[1]), "chi2_dof": float(res[2]),
            "grid": grid}


def probe_fma_rate(dtype="f32", iterations: int = 100_000, stream=None) -> float:
    """Measured fused multiply-add rate of the device (FMA instructions per second)."""
    r = ctypes.c_double()
    _check(lib().hydra_probe_fma_rate(_dtype_code(dtype), int(iterations), ctypes.byref(r), _stream_handle(stream)))
    return r.value


ARITH = {"f32": 0, "df": 1, "f64": 2}
OPS = {"add": 0, "mul": 1, "fma": 2, "sqrt": 3, "rcp": 4}


def probe_op_rate(arith: str, op: str, iterations: int = 20_000, stream=None) -> float:
    """Measured rate (operations per second) of one arithmetic operation: arith "f32" (the FP32
    kernels' arithmetic, hardware sqrt/rcp approximations), "df" (double-float pairs, the FP64
    generator's default) or "f64" (FP64 instructions); op one of OPS."""
    r = ctypes.c_double()
    _check(lib().hydra_probe_op_rate(ARITH[arith], OPS[op], int(iterations), ctypes.byref(r),
                                     _stream_handle(stream)))
    return r.value


def probe_write_bandwidth(buffer, reps: int = 5, stream=None) -> float:
    """Measured write-only bandwidth (GB/s) over a device tensor (16-byte stores)."""
    r = ctypes.c_double()
    nbytes = buffer.numel() * buffer.element_size()
    _check(lib().hydra_probe_write_bandwidth(ctypes.c_void_p(buffer.data_ptr()), int(nbytes), int(reps),
                                             ctypes.byref(r), _stream_handle(stream)))
    return r.value


def generate_sequential(M: float, masses, i: int, sub_masses, nevents: int, seed: int, sub_seed: int, *,
                        dtype="f32", stream=None):
    """Sequential decay (section 4.2): the n-body decay of M, then daughter i (mass masses[i])
    decays to len(sub_masses) bodies in its own frame.  Stage 2 uses the per-event parent
    momenta read straight from stage 1's SoA rows (px, py, pz of daughter i) and its own key
    `sub_seed`.  Returns (p1, w1, p2, w2); the event weight is w1 * w2."""
    p1, w1 = generate(M, masses, nevents, seed, dtype=dtype, stream=stream)
    moms = p1[i, 1:4]  # [3, ld] view: rows px, py, pz of daughter i, leading dimension ld
    p2, w2 = generate_boosted(masses[i], sub_masses, nevents, sub_seed, mothers=moms, dtype=dtype,
                              stream=stream)
    return p1, w1, p2, w2


def integrate(M: float, masses, nevents: int, seed: int, *, kin_dtype="f32", me: int = ME_FLAT,
              params=(), event_offset: int = 0, stream=None) -> dict:
    """Phase-space MC integral of f = w |ME|^2 over nevents events (blocking).

    Returns dict(mean, var_mean, sum_f, sum_f2, sum_w, sum_w2, n)."""
    res = Integral()
    _check(lib().hydra_phsp_integrate(float(M), len(masses), _dbl(masses), int(nevents), int(seed),
                                      int(event_offset), _dtype_code(kin_dtype), int(me),
                                      _dbl(params), len(params), ctypes.byref(res),
                                      _stream_handle(stream)))
    return res.as_dict()


def draws(n: int, nevents: int, seed: int, *, event_offset: int = 0, stream=None):
    """The raw 3n-4 Philox draws per event as an int64 tensor [3n-4, nevents] (uint32 values)."""
    import torch
    ld = padded_ld(nevents)
    out = torch.empty((3 * n - 4, ld), dtype=torch.int32, device="cuda")
    _check(lib().hydra_phsp_draws(int(n), int(nevents), int(seed), int(event_offset),
                                  ctypes.c_void_p(out.data_ptr()), ld, _stream_handle(stream)))
    return out[:, :nevents].to(torch.int64) & 0xFFFFFFFF


def set_launch_config(kind: int, n: int, dtype, block: int, events_per_thread: int) -> None:
    """Threads per block and events per thread of a kernel (kind: KERNEL_GENERATE or
    KERNEL_INTEGRATE) for n daughters in a precision; results do not depend on it."""
    _check(lib().hydra_set_launch_config(int(kind), int(n), _dtype_code(dtype), int(block),
                                         int(events_per_thread)))


FP64_NATIVE, FP64_DOUBLE_FLOAT = 0, 1


def set_fp64_arith(arith: int) -> None:
    """Arithmetic of FP64 generation: FP64_DOUBLE_FLOAT (default) or FP64_NATIVE."""
    _check(lib().hydra_set_fp64_arith(int(arith)))


def get_fp64_arith() -> int:
    return int(lib().hydra_get_fp64_arith())


LAMBDA_FACTORED_F32, LAMBDA_F64 = 0, 1


def set_fp32_lambda(arith: int) -> None:
    """Arithmetic of Kallen's lambda in FP32 generation: LAMBDA_FACTORED_F32 (default: the four
    gap factors multiplied in FP32) or LAMBDA_F64 (the same factors multiplied in FP64)."""
    _check(lib().hydra_set_fp32_lambda(int(arith)))


def get_fp32_lambda() -> int:
    return int(lib().hydra_get_fp32_lambda())


def get_launch_config(kind: int, n: int, dtype) -> tuple[int, int]:
    b, e = ctypes.c_int(), ctypes.c_int()
    _check(lib().hydra_get_launch_config(int(kind), int(n), _dtype_code(dtype), ctypes.byref(b),
                                         ctypes.byref(e)))
    return b.value, e.value


# ----------------------------------------------------------------------------- batches
REQ_GENERATE, REQ_INTEGRATE = 0, 1
SEGMENT_EVENTS = 1 << 21  # integral slices start on (and, unless last, hold) multiples of this


def request_dtype():
    """numpy record type with the layout of the C struct hydra_request (224 bytes)."""
    import numpy as np
    dt = np.dtype([("kind", "<i4"), ("n", "<i4"), ("dtype", "<i4"), ("me", "<i4"), ("M", "<f8"),
                   ("masses", "<f8", (10,)), ("params", "<f8", (6,)), ("seed", "<u8"),
                   ("event_offset", "<u8"), ("first", "<u8"), ("count", "<u8"), ("out", "<u8"),
                   ("ld", "<u8"), ("weights", "<u8"), ("total", "<u8"), ("seg_partials", "<u8")],
                  align=True)
    assert dt.itemsize == 224
    return dt


def batch_request_dtype():
    """numpy record type with the layout of the C struct hydra_batch_request (264 bytes)."""
    import numpy as np
    dt = np.dtype([("kind", "<i4"), ("n", "<i4"), ("dtype", "<i4"), ("me", "<i4"), ("M", "<f8"),
                   ("masses", "<f8", (10,)), ("params", "<f8", (6,)), ("seed", "<u8"), ("event_offset", "<u8"),
                   ("nevents", "<u8"), ("dest", "<i4"), ("status", "<i4"), ("out", "<u8"), ("ld", "<u8"),
                   ("weights", "<u8"),
                   ("result", [(k, "<f8") for k in ("mean", "var_mean", "sum_f", "sum_f2", "sum_w", "sum_w2")]
                    + [("n", "<u8")])], align=True)
    assert dt.itemsize == 264
    return dt


DEST_NONE, DEST_HOST, DEST_DEVICE = 0, 1, 2


def batch_run(table, budget_bytes: int, stream=None) -> None:
    """hydra_phsp_batch_run over a batch_request_dtype() array (in place: each record's status
    and, for integrals, result are written); blocks until every output has landed."""
    _check(lib().hydra_phsp_batch_run(ctypes.c_void_p(table.ctypes.data), len(table), int(budget_bytes),
                                      _stream_handle(stream)))


def batch_stats() -> tuple[int, int]:
    """(waves, slices) of this thread's latest successful batch_run."""
    w, s = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().hydra_phsp_batch_stats(ctypes.byref(w), ctypes.byref(s)))
    return w.value, s.value


def set_batch_shape(dtype, block: int, ept_by_n) -> None:
    """Launch shape of the persistent batch kernel: threads per block (FP32 runs) and events per
    thread of generation tiles for n = 2..10 (a mapping n -> ept or a sequence indexed by n)."""
    arr = (ctypes.c_int32 * 11)(*([2] * 11))
    for n in range(2, 11):
        arr[n] = int(ept_by_n[n])
    _check(lib().hydra_set_batch_shape(_dtype_code(dtype), int(block), ctypes.cast(arr, ctypes.c_void_p)))


def get_batch_shape(dtype) -> tuple[int, list]:
    arr = (ctypes.c_int32 * 11)()
    b = ctypes.c_int()
    _check(lib().hydra_get_batch_shape(_dtype_code(dtype), ctypes.byref(b), ctypes.cast(arr, ctypes.c_void_p)))
    return b.value, list(arr)


def serve_request_dtype():
    """numpy record type with the layout of the C struct hydra_serve_request (184 bytes)."""
    import numpy as np
    dt = np.dtype([("arrival", "<f8"), ("kind", "<i4"), ("n", "<i4"), ("M", "<f8"), ("masses", "<f8", (10,)),
                   ("nevents", "<u8"), ("seed", "<u8"), ("me", "<i4"), ("reserved", "<i4"), ("params", "<f8", (6,)),
                   ("withdraw", "<f8")])
    assert dt.itemsize == 184
    return dt


def serve_outcome_dtype():
    """numpy record type with the layout of the C struct hydra_serve_outcome (88 bytes)."""
    import numpy as np
    dt = np.dtype([("latency", "<f8"), ("host_offset", "<u8"), ("ld", "<u8"),
                   ("result", [(k, "<f8") for k in ("mean", "var_mean", "sum_f", "sum_f2", "sum_w", "sum_w2")]
                    + [("n", "<u8")]), ("status", "<i4"), ("reserved", "<i4")])
    assert dt.itemsize == 88
    return dt


SERVE_DONE, SERVE_REFUSED, SERVE_WITHDRAWN, SERVE_INVALID, SERVE_TIMED_OUT = 0, 1, 2, 3, 4


def segments(total: int) -> int:
    """Segments of 2^21 events in an integral request (size of its seg_partials / 8)."""
    return (int(total) + SEGMENT_EVENTS - 1) // SEGMENT_EVENTS


class Batch:
    """Runner for many uneven request slices in one persistent launch (hydra_batch_*)."""

    def __init__(self, max_requests: int = 4096, max_integrate_tiles: int = 1 << 20):
        h = ctypes.c_void_p()
        _check(lib().hydra_batch_create(int(max_requests), int(max_integrate_tiles), ctypes.byref(h)))
        self._h = h
        self.max_requests = max_requests

    def run(self, table, nreq: int | None = None, *, use_graph: bool = True, stream=None) -> None:
        """Enqueue a run of the first nreq records of `table` (a request_dtype() array)."""
        n = len(table) if nreq is None else int(nreq)
        _check(lib().hydra_batch_run(self._h, ctypes.c_void_p(table.ctypes.data), n, int(use_graph),
                                     _stream_handle(stream)))

    def result(self, i: int) -> dict:
        res = Integral()
        _check(lib().hydra_batch_result(self._h, int(i), ctypes.byref(res)))
        return res.as_dict()

    def close(self) -> None:
        if self._h:
            lib().hydra_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def shutdown() -> None:
    _check(lib().hydra_shutdown())
