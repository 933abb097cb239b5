"""Autotuner for the launch shape (threads per block, events per thread) of the kernels.

For each (kernel, n, precision) it times every candidate shape through the C ABI with CUDA
events on the current stream and installs the fastest with hydra_set_launch_config.  The
results are cached as JSON keyed by GPU name, so a process can apply a previous tuning
without re-measuring.  Shapes never change results (every event's arithmetic is the same and
integrals use a fixed reduction tree), so tuning is purely a speed decision.
"""
from __future__ import annotations

import json
import os

import paper_1711_05683_b300 as hp

BLOCKS = (128, 256, 512)
EPTS = (1, 2, 4)
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def _time(fn, reps: int) -> float:
    import torch
    s = torch.cuda.current_stream()
    fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_generate(n: int, dtype: str, masses, M: float = 10.0, nevents: int = 1 << 24,
                  reps: int = 3, buf=None) -> dict:
    """Best (block, ept) for hydra_phsp_generate at n daughters; returns the timing table."""
    import torch
    tdt = torch.float32 if dtype == "f32" else torch.float64
    if buf is None:
        buf = torch.empty((4 * n + 1) * nevents, dtype=tdt, device="cuda")
    out = buf[: 4 * n * nevents].view(n, 4, nevents)
    w = buf[4 * n * nevents: (4 * n + 1) * nevents]
    table = {}
    for block in BLOCKS:
        for ept in EPTS:
            hp.set_launch_config(hp.KERNEL_GENERATE, n, dtype, block, ept)
            table[f"{block}x{ept}"] = _time(lambda: hp.generate_into(M, masses, nevents, 1, out, w,
                                                                     dtype=dtype), reps)
    best = min(table, key=table.get)
    block, ept = (int(v) for v in best.split("x"))
    hp.set_launch_config(hp.KERNEL_GENERATE, n, dtype, block, ept)
    return {"block": block, "ept": ept, "ms": table[best], "table": table, "nevents": nevents}


def tune_integrate(n: int, dtype: str, masses, M: float, me: int = hp.ME_FLAT, params=(),
                   nevents: int = 1 << 25, reps: int = 3) -> dict:
    table = {}
    for block in BLOCKS:
        for ept in EPTS:
            hp.set_launch_config(hp.KERNEL_INTEGRATE, n, dtype, block, ept)
            table[f"{block}x{ept}"] = _time(lambda: hp.integrate(M, masses, nevents, 1, kin_dtype=dtype,
                                                                 me=me, params=params), reps)
    best = min(table, key=table.get)
    block, ept = (int(v) for v in best.split("x"))
    hp.set_launch_config(hp.KERNEL_INTEGRATE, n, dtype, block, ept)
    return {"block": block, "ept": ept, "ms": table[best], "table": table, "nevents": nevents}


def tune_all(ns=range(2, 11), dtypes=("f32", "f64"), gen_events: int = 1 << 24,
             int_events: int = 1 << 25, integrate_cases=None) -> dict:
    """Tune generate for every (n, dtype) with massive daughters m_i = M/(4n), and integrate
    for the given (n, dtype, M, masses, me, params) cases."""
    import torch
    res = {"gpu": _gpu_name(), "generate": {}, "integrate": {}}
    buf = torch.empty((4 * max(ns) + 1) * gen_events, dtype=torch.float64, device="cuda")
    for dtype in dtypes:
        view = buf if dtype == "f64" else buf.view(torch.float32)
        for n in ns:
            masses = tuple(10.0 / (4 * n) for _ in range(n))
            res["generate"][f"{n}/{dtype}"] = tune_generate(n, dtype, masses, nevents=gen_events, buf=view)
    del buf
    for case in integrate_cases or ():
        n, dtype, M, masses, me, params = case
        res["integrate"][f"{n}/{dtype}"] = tune_integrate(n, dtype, masses, M, me, params, int_events)
    return res


def apply(res: dict) -> None:
    for key, v in res.get("generate", {}).items():
        n, dtype = key.split("/")
        hp.set_launch_config(hp.KERNEL_GENERATE, int(n), dtype, v["block"], v["ept"])
    for key, v in res.get("integrate", {}).items():
        n, dtype = key.split("/")
        hp.set_launch_config(hp.KERNEL_INTEGRATE, int(n), dtype, v["block"], v["ept"])


def load_or_tune(path: str = CACHE, **kw) -> dict:
    """Apply the cached tuning for this GPU, or tune now and cache it."""
    name = _gpu_name()
    if os.path.exists(path):
        with open(path) as fh:
            cache = json.load(fh)
        if cache.get("gpu") == name:
            apply(cache)
            cache["source"] = "cache"
            return cache
    res = tune_all(**kw)
    with open(path, "w") as fh:
        json.dump(res, fh, indent=1)
    res["source"] = "tuned"
    return res
