"""Autotuner for the launch shape (threads per block, events per thread) of the kernels.

For each (kernel, n, precision) it times every candidate shape through the C ABI with CUDA
events on the current stream and installs the fastest with hydra_set_launch_config; for the
persistent batch kernel (FP32 runs) it picks the events per thread of each n and the block
size (tune_batch, installed with hydra_set_batch_shape).  The
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


def _gen_table(reqs, arena_ptr: int, arena_bytes: int):
    """Waves of request records (hydra_request) for FP32 generate requests (M, masses, nevents,
    seed) packed in order into an arena: [4n+1][ld] floats each, ld rounded up to 4."""
    import numpy as np
    waves, cur, off = [], [], 0
    for M, masses, nev, seed in reqs:
        n = len(masses)
        ld = (nev + 3) // 4 * 4
        nbytes = ((4 * n + 1) * ld * 4 + 255) // 256 * 256
        if cur and off + nbytes > arena_bytes:
            waves.append(cur)
            cur, off = [], 0
        cur.append((M, masses, nev, seed, off, ld))
        off += nbytes
    if cur:
        waves.append(cur)
    tables = []
    for wave in waves:
        t = np.zeros(len(wave), dtype=hp.request_dtype())
        for i, (M, masses, nev, seed, off, ld) in enumerate(wave):
            n = len(masses)
            t[i]["kind"], t[i]["n"], t[i]["dtype"], t[i]["M"] = hp.REQ_GENERATE, n, hp.F32, M
            t[i]["masses"][:n] = masses
            t[i]["seed"], t[i]["count"], t[i]["ld"] = seed, nev, ld
            t[i]["out"] = arena_ptr + off
            t[i]["weights"] = arena_ptr + off + 4 * n * ld * 4
        tables.append(t)
    return tables


def batch_ept_choices(n: int) -> tuple:
    return (1, 2, 4) if n <= 6 else (1, 2)


def tune_batch(mix=None, homogeneous_events: int = 1 << 20, nreq: int = 32, reps: int = 3,
               arena_bytes: int = 8 << 30) -> dict:
    """Launch shape of the FP32 persistent batch kernel: for each block size, the events per
    thread of each n that run a homogeneous batch (nreq requests of homogeneous_events events,
    masses M/(4n)) fastest; then the block size whose choice runs the uneven request mix fastest
    (default: 256 requests of the C4 mix, outputs in an arena of arena_bytes, overwritten wave to
    wave).  Installs the winner with hydra_set_batch_shape; returns the timing tables."""
    import torch
    import workloads
    if mix is None:
        mix = [(r.M, r.masses, r.nevents, r.seed) for r in workloads.batch_requests(256)]
    arena = torch.empty(arena_bytes // 4, dtype=torch.float32, device="cuda")
    ptr = arena.data_ptr()
    stream = torch.cuda.current_stream()
    res = {"blocks": {}, "nevents_homogeneous": homogeneous_events, "nreq_homogeneous": nreq,
           "mix_requests": len(mix)}
    _, default_ept = hp.get_batch_shape("f32")
    best_block, best_ms = None, float("inf")
    for block in BLOCKS:
        ept = list(default_ept)
        hp.set_batch_shape("f32", block, ept)
        batch = hp.Batch(max(nreq, len(mix)), 1)
        per_n = {}
        for n in range(2, 11):
            masses = tuple(10.0 / (4 * n) for _ in range(n))
            (table,) = _gen_table([(10.0, masses, homogeneous_events, 7 + i) for i in range(nreq)], ptr, arena_bytes)
            times = {}
            for e in batch_ept_choices(n):
                ept[n] = e
                hp.set_batch_shape("f32", block, ept)
                times[e] = _time(lambda: batch.run(table, stream=stream), reps)
            ept[n] = min(times, key=times.get)
            per_n[n] = {"ept": ept[n], "ms": times}
        hp.set_batch_shape("f32", block, ept)
        tables = _gen_table(mix, ptr, arena_bytes)
        mix_ms = _time(lambda: [batch.run(t, stream=stream) for t in tables], reps)
        batch.close()
        res["blocks"][block] = {"ept": list(ept), "per_n": per_n, "mix_ms": mix_ms}
        if mix_ms < best_ms:
            best_block, best_ms = block, mix_ms
    res["block"] = best_block
    res["ept"] = res["blocks"][best_block]["ept"]
    hp.set_batch_shape("f32", best_block, res["ept"])
    del arena
    torch.cuda.empty_cache()
    return res


def apply(res: dict) -> None:
    for key, v in res.get("generate", {}).items():
        n, dtype = key.split("/")
        hp.set_launch_config(hp.KERNEL_GENERATE, int(n), dtype, v["block"], v["ept"])
    for key, v in res.get("integrate", {}).items():
        n, dtype = key.split("/")
        hp.set_launch_config(hp.KERNEL_INTEGRATE, int(n), dtype, v["block"], v["ept"])
    if "batch" in res:
        hp.set_batch_shape("f32", res["batch"]["block"], res["batch"]["ept"])


def load_or_tune(path: str = CACHE, **kw) -> dict:
    """Apply the cached tuning for this GPU, or tune now and cache it."""
    name = _gpu_name()
    if os.path.exists(path):
        with open(path) as fh:
            cache = json.load(fh)
        if cache.get("gpu") == name and ("batch" in cache or not kw.get("batch", True)):
            apply(cache)
            cache["source"] = "cache"
            return cache
    batch = kw.pop("batch", True)
    res = tune_all(**kw)
    if batch:
        res["batch"] = tune_batch()
    with open(path, "w") as fh:
        json.dump(res, fh, indent=1)
    res["source"] = "tuned"
    return res
