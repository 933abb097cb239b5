"""CPU oracle for the phase-space Monte Carlo -- TEST INFRASTRUCTURE ONLY.

Python access (ctypes + numpy) to ``phsp_oracle.c``, a plain single-threaded FP64 C
implementation of the Raubold-Lynch generator and of the weighted phase-space integral
(Hydra §4.2, after F. James, CERN 68-15).  A second build in ``long double`` states the
oracle's own rounding error.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU baseline and
its ``--impl reference`` arm) may import this package.  The product library
(``paper_1711_05683_b300``) never imports it, and it never imports the product library.

Every public function cites the step of the method it exposes; the arithmetic itself is in
``phsp_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phsp_oracle.c")
_LIB64 = os.path.join(_HERE, "liboracle_f64.so")
_LIBLD = os.path.join(_HERE, "liboracle_f80.so")
_CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared"]

_lock = threading.Lock()
_libs: dict[str, ctypes.CDLL] = {}


def build(force: bool = False) -> None:
    """Compile the oracle (double and long double builds) with gcc."""
    for out, extra in ((_LIB64, []), (_LIBLD, ["-DORACLE_LD"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
            tmp = out + ".tmp"
            subprocess.check_call(["gcc", *_CFLAGS, *extra, "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, out)


def _lib(kind: str = "f64") -> ctypes.CDLL:
    with _lock:
        if kind not in _libs:
            build()
            lib = ctypes.CDLL(_LIB64 if kind == "f64" else _LIBLD)
            pfx = "oracle_" if kind == "f64" else "oracle_ld_"
            real = ctypes.c_double if kind == "f64" else ctypes.c_longdouble
            u32p, dp = ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_double)
            rp = ctypes.POINTER(real)
            getattr(lib, pfx + "philox4x32_10").argtypes = [u32p, u32p, u32p]
            getattr(lib, pfx + "draw").argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
            getattr(lib, pfx + "draw").restype = ctypes.c_uint32
            getattr(lib, pfx + "volume_factor").argtypes = [ctypes.c_double, ctypes.c_int, dp]
            getattr(lib, pfx + "volume_factor").restype = ctypes.c_double
            getattr(lib, pfx + "generate").argtypes = [ctypes.c_double, ctypes.c_int, dp,
                                                       ctypes.c_uint64, ctypes.c_uint64,
                                                       ctypes.c_uint64, rp, rp]
            getattr(lib, pfx + "generate").restype = ctypes.c_int
            getattr(lib, pfx + "integrate").argtypes = [ctypes.c_double, ctypes.c_int, dp,
                                                        ctypes.c_uint64, ctypes.c_uint64,
                                                        ctypes.c_uint64, ctypes.c_int, dp,
                                                        ctypes.c_int, dp]
            getattr(lib, pfx + "integrate").restype = ctypes.c_int
            getattr(lib, pfx + "generate_boosted").argtypes = [ctypes.c_double, ctypes.c_int, dp,
                                                               ctypes.c_uint64, ctypes.c_uint64,
                                                               ctypes.c_uint64, dp, dp, ctypes.c_uint64,
                                                               rp, rp]
            getattr(lib, pfx + "generate_boosted").restype = ctypes.c_int
            getattr(lib, pfx + "unweight").argtypes = [ctypes.c_double, ctypes.c_int, dp, ctypes.c_uint64,
                                                       ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                                       ctypes.POINTER(ctypes.c_ubyte)]
            getattr(lib, pfx + "unweight").restype = ctypes.c_int
            getattr(lib, pfx + "evaluate").argtypes = [ctypes.c_int, ctypes.c_uint64, dp, ctypes.c_uint64, dp,
                                                       ctypes.c_int, dp, ctypes.c_int, dp, dp]
            getattr(lib, pfx + "evaluate").restype = ctypes.c_int
            getattr(lib, pfx + "vegas").argtypes = [ctypes.c_double, ctypes.c_int, dp, ctypes.c_uint64, ctypes.c_int,
                                                    dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_double, ctypes.c_int, dp, dp, dp, dp]
            getattr(lib, pfx + "vegas").restype = ctypes.c_int
            getattr(lib, pfx + "me_dalitz_2bw").argtypes = [ctypes.c_double, ctypes.c_double, dp]
            getattr(lib, pfx + "me_dalitz_2bw").restype = ctypes.c_double
            _libs[kind] = lib
        return _libs[kind]


class variant:
    """Context manager that makes the f64 oracle functions use another build of the oracle
    source (used by the tests that plant mistakes in a copy of the source)."""

    def __init__(self, so_path: str):
        self.path = so_path
        self.saved = None

    def __enter__(self):
        lib = _lib("f64")  # ensure the normal library is set up, then swap
        with _lock:
            self.saved = _libs["f64"]
            new = ctypes.CDLL(self.path)
            for attr in ("philox4x32_10", "draw", "volume_factor", "generate", "integrate", "me_dalitz_2bw",
                         "generate_boosted", "unweight", "evaluate", "vegas"):
                src = getattr(lib, "oracle_" + attr)
                dst = getattr(new, "oracle_" + attr)
                dst.argtypes, dst.restype = src.argtypes, src.restype
            _libs["f64"] = new
        return self

    def __exit__(self, *exc):
        with _lock:
            _libs["f64"] = self.saved
        return False


def compile_variant(source_text: str, out_path: str) -> str:
    """Compile oracle source text (FP64 build) to a shared library at out_path."""
    src = out_path + ".c"
    with open(src, "w") as fh:
        fh.write(source_text)
    subprocess.check_call(["gcc", *_CFLAGS, "-o", out_path, src, "-lm"])
    return out_path


def source() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _pfx(kind: str) -> str:
    return "oracle_" if kind == "f64" else "oracle_ld_"


def _masses(masses) -> ctypes.Array:
    arr = (ctypes.c_double * len(masses))(*[float(m) for m in masses])
    return arr


class OracleError(ValueError):
    pass


def philox4x32_10(ctr, key) -> tuple[int, int, int, int]:
    """Philox4x32-10 block function (Salmon et al., SC'11): counter (4 words), key (2 words)."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    getattr(_lib(), "oracle_philox4x32_10")(c, k, o)
    return tuple(int(v) for v in o)


def draw(seed: int, event: int, d: int) -> int:
    """Draw d of event `event` under `seed` (word d%4 of counter (event, d/4, 0))."""
    return int(getattr(_lib(), "oracle_draw")(seed, event, d))


def draws(seed: int, event: int, n: int) -> np.ndarray:
    """All 3n-4 draws of one event, in draw order."""
    return np.array([draw(seed, event, d) for d in range(3 * n - 4)], dtype=np.uint64)


def volume_factor(M: float, masses) -> float:
    """Weight constant C_n = pi^(n-1) 2^(n-2) T^(n-2) / ((n-2)! M)."""
    v = getattr(_lib(), "oracle_volume_factor")(float(M), len(masses), _masses(masses))
    if v < 0:
        raise OracleError("invalid decay")
    return float(v)


def generate(M: float, masses, nevents: int, seed: int, event_offset: int = 0,
             kind: str = "f64") -> tuple[np.ndarray, np.ndarray]:
    """Raubold-Lynch events: returns (p[n, 4, nevents] as (E, px, py, pz), w[nevents])."""
    n = len(masses)
    dt = np.float64 if kind == "f64" else np.longdouble
    out = np.empty((n, 4, nevents), dtype=dt)
    w = np.empty(nevents, dtype=dt)
    real = ctypes.c_double if kind == "f64" else ctypes.c_longdouble
    rp = ctypes.POINTER(real)
    rc = getattr(_lib(kind), _pfx(kind) + "generate")(
        float(M), n, _masses(masses), nevents, seed, event_offset,
        out.ctypes.data_as(rp), w.ctypes.data_as(rp))
    if rc == -2:
        raise OracleError("below threshold")
    if rc != 0:
        raise OracleError("invalid decay")
    return out, w


def generate_boosted(M: float, masses, nevents: int, seed: int, mother=None, mothers=None,
                     event_offset: int = 0, kind: str = "f64") -> tuple[np.ndarray, np.ndarray]:
    """Events of a moving parent: generated at rest, then every daughter boosted to the frame
    where the parent has momentum `mother` (3 values) or mothers[:, e] (array [3, nevents])."""
    n = len(masses)
    dt = np.float64 if kind == "f64" else np.longdouble
    out = np.empty((n, 4, nevents), dtype=dt)
    w = np.empty(nevents, dtype=dt)
    real = ctypes.c_double if kind == "f64" else ctypes.c_longdouble
    rp, dp = ctypes.POINTER(real), ctypes.POINTER(ctypes.c_double)
    if mothers is not None:
        mo = np.ascontiguousarray(mothers, dtype=np.float64)
        mp, mptr, mld = None, mo.ctypes.data_as(dp), mo.shape[1]
    else:
        mo = None
        mp, mptr, mld = (ctypes.c_double * 3)(*[float(v) for v in mother]), None, 0
    rc = getattr(_lib(kind), _pfx(kind) + "generate_boosted")(
        float(M), n, _masses(masses), nevents, seed, event_offset, mp, mptr, mld,
        out.ctypes.data_as(rp), w.ctypes.data_as(rp))
    if rc != 0:
        raise OracleError("invalid decay")
    return out, w


def unweight(M: float, masses, nevents: int, seed: int, w_max: float, event_offset: int = 0) -> np.ndarray:
    """Accept flags of accept-reject unweighting: keep e when u_e w_max < w_e (u_e = draw 3n-4)."""
    acc = np.zeros(nevents, dtype=np.uint8)
    rc = getattr(_lib(), "oracle_unweight")(float(M), len(masses), _masses(masses), nevents, seed,
                                             event_offset, float(w_max),
                                             acc.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    if rc != 0:
        raise OracleError("invalid arguments")
    return acc.astype(bool)


def integrate_sums(M: float, masses, nevents: int, seed: int, me: int = 0, params=(),
                   event_offset: int = 0, kind: str = "f64") -> np.ndarray:
    """(sum f, sum f^2, sum w, sum w^2) with f = w |ME|^2 over the given events."""
    sums = (ctypes.c_double * 4)()
    par = (ctypes.c_double * max(1, len(params)))(*[float(p) for p in params])
    rc = getattr(_lib(kind), _pfx(kind) + "integrate")(
        float(M), len(masses), _masses(masses), nevents, seed, event_offset, me, par,
        len(params), sums)
    if rc == -2:
        raise OracleError("below threshold")
    if rc != 0:
        raise OracleError("invalid arguments")
    return np.array(list(sums), dtype=np.float64)


def integrate(M: float, masses, nevents: int, seed: int, me: int = 0, params=(),
              event_offset: int = 0, kind: str = "f64") -> dict:
    """Mean of f = w |ME|^2 and the variance of that mean, (<f^2> - <f>^2) / (n - 1)."""
    s = integrate_sums(M, masses, nevents, seed, me, params, event_offset, kind)
    n = float(nevents)
    mean = s[0] / n
    var_mean = (s[1] / n - mean * mean) / (n - 1.0) if nevents > 1 else float("nan")
    return dict(mean=mean, var_mean=var_mean, sum_f=s[0], sum_f2=s[1], sum_w=s[2],
                sum_w2=s[3], n=nevents)


def evaluate(events: np.ndarray, weights: np.ndarray, me: int = 0, params=()) -> tuple[np.ndarray, np.ndarray]:
    """f_e = w_e |ME|^2 on stored events events[n, 4, nevents] (FP64); returns (values, sums)."""
    ev = np.ascontiguousarray(events, dtype=np.float64)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    n, _, nev = ev.shape
    vals = np.empty(nev, dtype=np.float64)
    sums = (ctypes.c_double * 4)()
    par = (ctypes.c_double * max(1, len(params)))(*[float(p) for p in params])
    dp = ctypes.POINTER(ctypes.c_double)
    rc = getattr(_lib(), "oracle_evaluate")(n, nev, ev.ctypes.data_as(dp), nev, w.ctypes.data_as(dp), me,
                                            par, len(params), vals.ctypes.data_as(dp), sums)
    if rc != 0:
        raise OracleError("invalid arguments")
    return vals, np.array(list(sums))


def vegas(M: float, masses, seed: int, calls: int, iterations: int, bins: int = 50, alpha: float = 1.5,
          skip: int = 1, me: int = 0, params=()) -> dict:
    """VEGAS (importance sampling, GSL structure) of |ME|^2 over the Raubold-Lynch variables:
    per-iteration estimates and variances, the combined result, sigma, chi2/dof, final grid."""
    n = len(masses)
    D = 3 * n - 4
    est = np.zeros(iterations)
    var = np.zeros(iterations)
    res = np.zeros(3)
    grid = np.zeros((D, bins + 1))
    dp = ctypes.POINTER(ctypes.c_double)
    par = (ctypes.c_double * max(1, len(params)))(*[float(p) for p in params])
    rc = getattr(_lib(), "oracle_vegas")(float(M), n, _masses(masses), seed, me, par, len(params), calls,
                                         iterations, bins, float(alpha), skip, est.ctypes.data_as(dp),
                                         var.ctypes.data_as(dp), res.ctypes.data_as(dp), grid.ctypes.data_as(dp))
    if rc != 0:
        raise OracleError("invalid arguments")
    return {"est": est, "var": var, "mean": res[0], "sigma": res[1], "chi2_dof": res[2], "grid": grid}


def me_dalitz_2bw(s12: float, s23: float, params) -> float:
    """|BW(s12; m0a, Ga) + |c| e^{i arg c} BW(s23; m0b, Gb)|^2, BW(s) = 1/(m0^2 - s - i m0 G)."""
    par = (ctypes.c_double * 6)(*[float(p) for p in params])
    return float(getattr(_lib(), "oracle_me_dalitz_2bw")(float(s12), float(s23), par))
