"""Benchmark: phase-space events/s on B300 for the N-body generator sweep and the Dalitz integral.

One step = one pass of the whole hot path over the synthetic workload:
  * generate: N = 2..10 daughters, massless and massive (m_i ~ U[0, M/(2N)], seeded),
    M = 10 GeV, 1e8 events per (N, masses, precision), FP32 and FP64 kinematics and
    outputs (structure of arrays (E, px, py, pz) per daughter + weight), 36 launches;
  * integrate: the 3-body Dalitz matrix element |BW(m12) + 0.5 e^{1.2i} BW(m23)|^2 over
    1e9 events (M = 1.865 GeV), FP32 kinematics, FP64 compensated sums, no event storage.
value = (events generated + events integrated) / step time, timed with CUDA events on the
launching stream; outputs (5-33 GB per launch) are far larger than L2, so no L2 flush is
needed.  `e2e` times the same step through the host-output C-ABI entry point (every event
copied to pinned host memory inside the timed region).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) each rank runs the same per-rank workload on disjoint counter-event
ranges (weak scaling, no data-path collective); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "phase-space events/s (N=3..10, FP32/FP64) vs roofline; served p50/p99 latency"
GEN_N = workloads.SWEEP_N
GEN_EVENTS = workloads.SWEEP_NEVENTS
INT_CFG = workloads.D0_DALITZ


# Thread instructions issued per event by the generator kernels at their tuned launch shapes
# (ncu smsp__inst_executed.sum x 32 / events on a 4e6-event launch of each kernel, one capture
# of a single generator kernel per row).  They explain the issue-bound double-float generator
# (issue_frac in the per-launch breakdown); the roofline itself counts method operations.
INSTR_PER_EVENT = {
    ("f32", 2): 80, ("f32", 3): 198, ("f32", 4): 280, ("f32", 5): 399, ("f32", 6): 512,
    ("f32", 7): 632, ("f32", 8): 718, ("f32", 9): 880, ("f32", 10): 996,
    ("f64", 2): 336, ("f64", 3): 848, ("f64", 4): 1314, ("f64", 5): 1773, ("f64", 6): 2310,
    ("f64", 7): 2803, ("f64", 8): 3252, ("f64", 9): 3743, ("f64", 10): 4229,
    # the double-float variant for all-massless decays (no square root per two-body momentum)
    ("f64", 2, "massless"): 260, ("f64", 3, "massless"): 736, ("f64", 4, "massless"): 1175,
    ("f64", 5, "massless"): 1602, ("f64", 6, "massless"): 2099, ("f64", 7, "massless"): 2537,
    ("f64", 8, "massless"): 2950, ("f64", 9, "massless"): 3403, ("f64", 10, "massless"): 3841,
}


# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) per launch of the dominant
# kernel family, averaged over its 18 launches: captured on 4e6-event launches (one kernel,
# two launches per capture) and scaled by 25 to the benchmark's 1e8 events.  The captures
# leave ~64 MB of written lines dirty in L2 when a launch ends, so the scaled figure sits that
# much per 4e6 events (1.6 GB per scaled launch) below the 20.0 GB of outputs; None until
# captured for the kernels as they stand.
TRAFFIC_GB_PER_LAUNCH = {"f64": 18.49, "f32": None}


def emit_detail(detail: dict, path: str | None) -> None:
    """The per-launch breakdown, measured ceilings, batch, serving and extension figures: one
    JSON line on stderr (stdout carries only the result line), and to `path` if given."""
    text = json.dumps(detail)
    print("bench detail: " + text, file=sys.stderr, flush=True)
    if path:
        with open(path, "w") as fh:
            fh.write(text + "\n")


def method_ops(n: int, massless: bool = False) -> dict:
    """Algorithmic floating-point operations of one Raubold-Lynch event by kind (an add,
    multiply or fused multiply-add counts 1; a square root, reciprocal, division or sin/cos
    pair counts 1 each).  A boosted two-body step (massive daughters) takes 48: the
    intermediate mass r T + mu (mul, add), the gap (mul), lambda's four factors and their
    product (2 M_k, 2 m by scaling; 3 adds, 3 muls), 1/M_{k+1} (rcp), p = sqrt(lambda) / (2 M_{k+1})
    (sqrt, 2 muls), the weight factor (mul), cos theta, 1 -+ cos theta (3 adds), sin theta
    (mul, sqrt), sin/cos phi (1), the 3-momentum (4 muls), the rest-frame energy M_k +
    Delta (Delta + 2 m) / (2 M_{k+1}) (fma), Q.p (3 muls, 2 adds), the boosted energy (2 muls,
    add), the boost factor (2 adds, div), the boosted 3-momentum (3 muls, 3 adds) and the
    daughter by subtraction (4 adds); the parent's decay has no boost (31).  For all-massless
    daughters lambda = (Delta (Delta + 2 M_k))^2 and the momentum needs 4 operations instead
    of 10 (43 per boosted step, 26 for the parent).  Plus the constant C_n (mul)."""
    k = n - 2  # boosted steps
    ops = {"add": 19 * k + 11, "mul": 23 * k + 15 + 1, "fma": n - 1, "sqrt": 2 * (n - 1),
           "rcp": n - 1, "div": k, "sincos": n - 1}
    if massless:  # per step: 2 adds, 2 muls and the square root of lambda fewer
        ops["add"] -= 2 * (n - 1)
        ops["mul"] -= 2 * (n - 1)
        ops["sqrt"] -= n - 1
    return ops


def fp_ops_per_event(n: int, massless: bool = False) -> int:
    return sum(method_ops(n, massless).values())


def fp_seconds_per_event(ops: dict, rates: dict) -> float:
    """Time of one event's method operations at the measured rates of the arithmetic the
    kernel runs.  A division counts as a reciprocal and a product; a sin/cos pair as one
    square root (a generous ceiling: the kernels spend more on it)."""
    t = ops["add"] / rates["add"] + ops["mul"] / rates["mul"] + ops["fma"] / rates["fma"]
    t += ops["sqrt"] / rates["sqrt"] + ops["rcp"] / rates["rcp"]
    t += ops["div"] * (1.0 / rates["rcp"] + 1.0 / rates["mul"]) + ops["sincos"] / rates["sqrt"]
    return t


def measure_op_rates(hp) -> dict:
    """Rates (operations/s) of add, mul, fma, sqrt and rcp in FP32 (the FP32 kernels'
    arithmetic) and in double-float (the FP64 generator's), from the library's probe."""
    out = {}
    for arith, iters in (("f32", 100_000), ("df", 20_000)):
        out[arith] = {op: hp.probe_op_rate(arith, op, iters) for op in ("add", "mul", "fma", "sqrt", "rcp")}
    return out


def instr_per_event(dtype: str, n: int, massive: bool) -> int:
    """Thread instructions per event of the generator kernel a launch runs."""
    return INSTR_PER_EVENT.get((dtype, n) if massive else (dtype, n, "massless"), INSTR_PER_EVENT[(dtype, n)])


def bytes_per_event(n: int, dtype: str) -> int:
    """Algorithmic output bytes per generated event: 4n components + 1 weight."""
    return (4 * n + 1) * (4 if dtype == "f32" else 8)


def sweep_items():
    items = []
    for dtype in ("f32", "f64"):
        for massive in (False, True):
            for n in GEN_N:
                items.append((dtype, massive, n))
    return items


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return {"hbm_gbs": float(pk["hbm_gbs"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6400.0, "src": "fallback"}


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.rows: list[list[str]] = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- our arm
def run_ours(args) -> None:
    import torch
    import paper_1711_05683_b300 as hp
    from paper_1711_05683_b300 import build as hp_build

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        hp_build.build()
    if world > 1:
        dist.barrier()
    hp.lib()
    # launch shapes: the autotuner's cached choice for this GPU, or a fresh tuning (untimed)
    from paper_1711_05683_b300 import autotune
    cases = [(3, "f32", INT_CFG["M"], INT_CFG["masses"], hp.ME_DALITZ_2BW, INT_CFG["params"])]
    if rank == 0:  # rank 0 tunes (or loads) and writes the cache; the others then load it
        tuning = autotune.load_or_tune(integrate_cases=cases)
    if world > 1:
        dist.barrier()
    if rank != 0:
        tuning = autotune.load_or_tune(integrate_cases=cases)

    nev = args.events
    int_events = args.int_events
    items = sweep_items()
    max_elems = max((4 * n + 1) for n in GEN_N) * nev
    buf64 = torch.empty(max_elems, dtype=torch.float64, device="cuda")  # reused by every launch
    buf32 = buf64.view(torch.float32)
    stream = torch.cuda.current_stream()
    from paper_1711_05683_b300 import shard
    base_offset = shard.rank_event_offset(rank, nev + int_events)  # disjoint counter-event ranges

    def views(n, dtype):
        ld = nev
        b = buf32 if dtype == "f32" else buf64
        out = b[: 4 * n * ld].view(n, 4, ld)
        w = b[4 * n * ld: (4 * n + 1) * ld]
        return out, w

    ev_pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(len(items) + 1)]

    def step(record: bool):
        for k, (dtype, massive, n) in enumerate(items):
            out, w = views(n, dtype)
            masses = workloads.sweep_masses(n, massive)
            if record:
                ev_pairs[k][0].record(stream)
            hp.generate_into(workloads.SWEEP_M, masses, nev, 1000 + n, out, w, dtype=dtype,
                             event_offset=base_offset)
            if record:
                ev_pairs[k][1].record(stream)
        if record:
            ev_pairs[-1][0].record(stream)
        res = hp.integrate(INT_CFG["M"], INT_CFG["masses"], int_events, INT_CFG["seed"],
                           kin_dtype="f32", me=hp.ME_DALITZ_2BW, params=INT_CFG["params"],
                           event_offset=base_offset)
        if record:
            ev_pairs[-1][1].record(stream)
        return res

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # Measured device ceilings (outside the timed region): FP32 / FP64 FMA rates and the
    # write-only HBM bandwidth of 16-byte stores over 4 GB.
    probe_buf = torch.empty(1 << 32, dtype=torch.uint8, device="cuda")
    fma32 = hp.probe_fma_rate("f32", 200_000)
    fma64 = hp.probe_fma_rate("f64", 4_000)
    measured = {"fp32_fma_per_s": fma32, "fp32_tflops": round(2 * fma32 / 1e12, 2),
                "fp64_fma_per_s": fma64, "fp64_tflops": round(2 * fma64 / 1e12, 3),
                "hbm_write_gbs": round(hp.probe_write_bandwidth(probe_buf, 5), 1),
                "src": "hydra_probe_fma_rate (8 independent FMA chains per thread, all SMs) and "
                       "hydra_probe_write_bandwidth (16-byte stores over 4 GB), this run"}
    op_rates = measure_op_rates(hp)
    measured["op_rates"] = {a: {k: round(v / 1e12, 3) for k, v in r.items()} for a, r in op_rates.items()}
    measured["op_rates_unit"] = "T operations/s (hydra_probe_op_rate: 8 independent chains per thread, all SMs)"
    del probe_buf
    torch.cuda.empty_cache()

    for _ in range(args.warmup):
        step(False)
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    per_launch_ms = [0.0] * (len(items) + 1)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    barrier()
    t0.record(stream)
    for _ in range(args.steps):
        res = step(True)
        torch.cuda.synchronize()
        for k, (a, b) in enumerate(ev_pairs):
            per_launch_ms[k] += a.elapsed_time(b)
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = shard.max_over_ranks(t0.elapsed_time(t1), device="cuda")
    ms_per_step = total_ms / args.steps
    per_step_events = len(items) * nev + int_events
    value = per_step_events * world / (ms_per_step / 1e3)

    # e2e through the host-output entry point: every generated event copied to pinned host
    # memory inside the timed region; the integral's result is read back by the call itself.
    e2e = None
    if not args.no_e2e:
        host_elems = max_elems
        hbuf64 = torch.empty(host_elems, dtype=torch.float64, pin_memory=True)
        hbuf32 = hbuf64.view(torch.float32)
        d2h = 0
        h2d = 0

        def e2e_step():
            nonlocal d2h, h2d
            d2h = h2d = 0
            for dtype, massive, n in items:
                b = hbuf32 if dtype == "f32" else hbuf64
                out = b[: 4 * n * nev].view(n, 4, nev)
                w = b[4 * n * nev: (4 * n + 1) * nev]
                hp.generate_host_into(workloads.SWEEP_M, workloads.sweep_masses(n, massive), nev,
                                      1000 + n, out, w, dtype=dtype, event_offset=base_offset)
                d2h += bytes_per_event(n, dtype) * nev
                h2d += 8 * n  # the host array of daughter masses
            hp.integrate(INT_CFG["M"], INT_CFG["masses"], int_events, INT_CFG["seed"], kin_dtype="f32",
                         me=hp.ME_DALITZ_2BW, params=INT_CFG["params"], event_offset=base_offset)
            d2h += 56  # hydra_integral
            h2d += 8 * 3 + 8 * 6

        e2e_steps = max(1, min(args.steps, args.e2e_steps))
        e2e_step()  # warm-up (allocates staging)
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(e2e_steps):
            e2e_step()
        b.record(stream)
        barrier()
        e2e_ms = shard.max_over_ranks(a.elapsed_time(b) / e2e_steps, device="cuda")
        # the host link's own D2H rate (one device-to-pinned copy of up to 4 GB, outside the timed region)
        nb = min(1 << 32, hbuf64.numel() * 8)
        probe = torch.empty(nb, dtype=torch.uint8, device="cuda")
        hprobe = hbuf64.view(torch.uint8)[:nb]
        hprobe.copy_(probe, non_blocking=True)
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        hprobe.copy_(probe, non_blocking=True)
        c1.record(stream)
        c1.synchronize()
        link_gbs = nb / (c0.elapsed_time(c1) / 1e3) / 1e9
        del probe, hprobe
        achieved_link = d2h / (e2e_ms / 1e3) / 1e9
        e2e = {"value": per_step_events * world / (e2e_ms / 1e3), "unit": "events/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps,
               "ms_per_step": e2e_ms, "d2h_gbs": round(achieved_link, 1),
               "d2h_link_gbs_measured": round(link_gbs, 1), "link_frac": round(achieved_link / link_gbs, 4),
               "bound": "host link (every generated event is copied to pinned host memory)"}
        del hbuf64, hbuf32

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peaks = load_peaks()
    hbm = peaks["hbm_gbs"] * 1e9
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2032.0
    issue_limit = sms * 4 * 32 * sm_mhz * 1e6  # thread instructions per second
    breakdown = []
    for k, (dtype, massive, n) in enumerate(items):
        ms = per_launch_ms[k] / args.steps
        ev_s = nev / (ms / 1e3)
        # the launch's roofline: the slower of its output bytes at the measured HBM
        # copy peak and its method operations at the measured rates of the arithmetic it runs
        ops = method_ops(n, massless=not massive)
        by_hbm = hbm / bytes_per_event(n, dtype)
        by_fp = 1.0 / fp_seconds_per_event(ops, op_rates["f32" if dtype == "f32" else "df"])
        roof = min(by_hbm, by_fp)
        breakdown.append({"kernel": f"phsp_generate_kernel<{n},{'float' if dtype == 'f32' else 'df'}>",
                          "n": n, "dtype": dtype, "massive": massive, "events": nev, "ms": round(ms, 4),
                          "events_per_s": ev_s, "hbm_gbs": round(bytes_per_event(n, dtype) * ev_s / 1e9, 1),
                          "fp_ops_per_event": sum(ops.values()), "roof_hbm_events_per_s": by_hbm,
                          "roof_fp_events_per_s": by_fp, "roofline_bound": "hbm" if by_hbm <= by_fp else "fp",
                          "roofline_frac": round(ev_s / roof, 4),
                          "issue_frac": round(instr_per_event(dtype, n, massive) * ev_s / issue_limit, 4)})
    int_ms = per_launch_ms[-1] / args.steps
    breakdown.append({"kernel": "phsp_integrate_tiles<3,float,DALITZ_2BW>+reduce", "events": int_events,
                      "ms": round(int_ms, 4), "events_per_s": int_events / (int_ms / 1e3),
                      "mean": res["mean"], "sigma": math.sqrt(res["var_mean"])})

    def family(dtype):
        rows = [x for x in breakdown[:-1] if x["dtype"] == dtype]
        f_ms = sum(x["ms"] for x in rows)
        roof_ms = sum(x["events"] / min(x["roof_hbm_events_per_s"], x["roof_fp_events_per_s"]) * 1e3 for x in rows)
        f_bytes = sum(bytes_per_event(x["n"], dtype) * x["events"] for x in rows)
        f_ops = sum(x["fp_ops_per_event"] * x["events"] for x in rows)
        fp_ms = sum(x["ms"] for x in rows if x["roofline_bound"] == "fp")
        return {"ms": f_ms, "roof_ms": roof_ms, "bytes": f_bytes, "ops": f_ops, "launches": len(rows),
                "events": sum(x["events"] for x in rows), "fp_bound_ms": fp_ms}

    fams = {"f64": family("f64"), "f32": family("f32")}
    fam_ms = {"f64": fams["f64"]["ms"], "f32": fams["f32"]["ms"], "integrate": int_ms}
    dominant = max(fam_ms, key=fam_ms.get)
    d = fams["f64" if dominant != "f32" else "f32"]
    dk = "f64" if dominant != "f32" else "f32"
    achieved = d["ops"] / (d["ms"] / 1e3) / 1e12
    peak = d["ops"] / (d["roof_ms"] / 1e3) / 1e12
    roof = {"bound": "alu" if d["fp_bound_ms"] > d["ms"] / 2 else "hbm",
            "kernel": ("phsp_generate_kernel<N,df> (FP64 outputs, double-float arithmetic)" if dk == "f64"
                       else "phsp_generate_kernel<N,float>") + f", N=2..10, {d['launches']} launches/step",
            "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "T method-FP-ops/s",
            "frac": round(d["roof_ms"] / d["ms"], 4),
            "ms": round(d["ms"], 3), "roofline_ms": round(d["roof_ms"], 3),
            "peak_src": f"per launch min(HBM {peaks['hbm_gbs']:.0f} GB/s {peaks['src']} / (32N+8) B, "
                        f"{'double-float' if dk == 'f64' else 'FP32'} op rates of hydra_probe_op_rate "
                        "this run / method ops per event)",
            "hbm_frac": round(d["bytes"] / (d["ms"] / 1e3) / hbm, 4),
            "traffic": TRAFFIC_GB_PER_LAUNCH.get(dk), "traffic_unit": "GB/launch (ncu dram read+write)"}
    f32 = fams["f32"]
    f32_roof = {"bound": "hbm", "achieved": round(f32["bytes"] / (f32["ms"] / 1e3) / 1e9, 1),
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac_of_hbm": round(f32["bytes"] / (f32["ms"] / 1e3) / hbm, 4),
                "frac": round(f32["roof_ms"] / f32["ms"], 4)}
    detail = {
        "measured_peaks": measured, "dominant": dominant, "family_ms_per_step": {k: round(v, 3) for k, v in fam_ms.items()},
        "roofline": roof, "fp32_generator_roofline": f32_roof, "breakdown": breakdown, "clocks": clk, "e2e": e2e,
        "launch_shapes": {"source": tuning.get("source"),
                          "generate": {k: f"{v['block']}x{v['ept']}" for k, v in tuning["generate"].items()},
                          "integrate": {k: f"{v['block']}x{v['ept']}" for k, v in tuning["integrate"].items()}},
    }
    line = {
        "metric": METRIC,
        "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 + f64 (FP64 outputs from double-float arithmetic, within 1e-12 of FP64)",
        "data": "synthetic",
        "config": {"workload": "N-body sweep N=2..10 massless+massive, M=10 GeV, FP32 and FP64 SoA "
                               "outputs, 1e8 events each; Dalitz 2-BW integral, 1e9 events",
                   "events_per_launch": nev, "integrate_events": int_events,
                   "l2": "outputs >> L2 (126 MB); no flush", "parallelism": f"replicas x{world}"},
        "gpu_launches": args.steps * (len(items) + 2 * math.ceil(int_events / 2 ** 26) + 1),
        "clocks": {k: clk.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "roofline": {k: roof[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "ms", "roofline_ms")},
        "fp32_generator_roofline": {k: f32_roof[k] for k in ("frac", "frac_of_hbm")},
        "family_ms": {k: round(v, 2) for k, v in fam_ms.items()},
    }
    if e2e is not None:
        line["e2e"] = {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step", "link_frac")}
    detail["c1_fp64_three_body"] = run_c1()
    if not args.no_batch:
        detail["batch"] = run_batch_workload()
        detail["extensions"] = run_extras(hbm_peak_gbs=peaks["hbm_gbs"])
        line["batch_speedup_vs_plain"] = round(detail["batch"]["speedup_vs_plain"], 3)
    if not args.no_serve:
        detail["serve"] = run_serve_workload(duration_s=args.serve_seconds)
        sv = detail["serve"]
        line["serve"] = {"p50_ms": round(sv["batched_native_loop"]["p50_ms"], 3),
                         "p99_ms": round(sv["batched_native_loop"]["p99_ms"], 3),
                         "plain_p99_ms": round(sv["plain"]["p99_ms"], 3),
                         "events_per_s": sv["batched_native_loop"]["events_per_s"]}
    if not args.no_cpu_baseline:
        cb = cpu_baseline(args.cpu_seconds, nev, int_events)
        detail["cpu_baseline"] = cb
        detail["cpu_all_cores"] = cpu_all_cores(cb["sample_events"], nev, int_events)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    emit_detail(detail, args.detail_out)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_c1(reps: int = 20) -> dict:
    """The FP64 three-body workload (B -> J/psi K pi like, M = 5.2795 GeV, 1e5 events, seed 42):
    one generator launch timed with CUDA events (best of `reps` after a warm-up; 10.4 MB of
    outputs, latency-bound) and checked on the host: 4-momentum conservation and on-shell
    daughters of every event, relative to the event scale."""
    import numpy as np
    import torch
    import paper_1711_05683_b300 as hp
    c = workloads.B_TO_JPSI_K_PI
    nev = c["nevents"]
    stream = torch.cuda.current_stream()
    p, w = hp.generate(c["M"], c["masses"], nev, c["seed"], dtype="f64")
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hp.generate_into(c["M"], c["masses"], nev, c["seed"], p, w, dtype="f64")
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    ev = p[:, :, :nev].cpu().numpy()
    tot = ev.sum(axis=0)
    cons = float(max(np.abs(tot[0] - c["M"]).max(), np.abs(tot[1:]).max()) / c["M"])
    m2 = ev[:, 0] ** 2 - (ev[:, 1:] ** 2).sum(axis=1)
    shell = float((np.abs(m2 - np.array(c["masses"])[:, None] ** 2) / c["M"] ** 2).max())
    return {"events": nev, "us": round(best * 1e3, 2), "events_per_s": nev / (best / 1e3),
            "max_conservation_error": cons, "max_on_shell_error": shell}


# ----------------------------------------------------------------------------- batched requests
ARENA_BYTES = 40 * 10 ** 9  # HBM budget for the outputs of one wave


def batch_waves(reqs, arena_bytes=ARENA_BYTES):
    """Greedy waves of consecutive requests whose FP32 outputs fit the arena; returns
    (wave list of (request, byte offset, ld)) ."""
    waves, cur, off = [], [], 0
    for r in reqs:
        ld = (r.nevents + 3) // 4 * 4
        nbytes = (4 * len(r.masses) + 1) * ld * 4
        if cur and off + nbytes > arena_bytes:
            waves.append(cur)
            cur, off = [], 0
        cur.append((r, off, ld))
        off += (nbytes + 255) // 256 * 256
    if cur:
        waves.append(cur)
    return waves


def run_batch_workload(count: int = 4096, reps: int = 2, arena_bytes: int = ARENA_BYTES) -> dict:
    """Uneven generate requests (N 2..8, M 1..10 GeV, masses U[0, M/2N], events log-uniform
    1e3..1e7, per-request seeds), FP32 outputs overwritten wave to wave: one hydra_phsp_batch_run
    call with a device budget of arena_bytes (the library packs the waves, one persistent graph
    launch each, shape from the autotuner) against one plain hydra_phsp_generate launch per
    request into an arena of the same size (greedy waves in request order).  Wall time of the
    blocking call (best of `reps` after a warm-up that allocates the library's kept arena)
    against CUDA-event time of the plain launches plus their final synchronisation."""
    import numpy as np
    import torch
    import paper_1711_05683_b300 as hp
    reqs = workloads.batch_requests(count)
    total = sum(r.nevents for r in reqs)
    out_bytes = sum((4 * len(r.masses) + 1) * r.nevents * 4 for r in reqs)
    table = np.zeros(count, dtype=hp.batch_request_dtype())
    for i, r in enumerate(reqs):
        n = len(r.masses)
        rec = table[i]
        rec["kind"], rec["n"], rec["dtype"], rec["M"] = hp.REQ_GENERATE, n, hp.F32, r.M
        rec["masses"][:n] = r.masses
        rec["seed"], rec["nevents"], rec["dest"] = r.seed, r.nevents, hp.DEST_NONE
    stream = torch.cuda.current_stream()
    hp.batch_run(table, arena_bytes, stream=stream)  # warm-up: the library allocates and keeps its buffers
    waves, slices = hp.batch_stats()
    best_b = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hp.batch_run(table, arena_bytes, stream=stream)
        best_b = min(best_b, time.perf_counter() - t0)
    shape = hp.get_batch_shape("f32")
    hp.shutdown()  # release the kept arena before the plain arm allocates its own
    # plain arm: one launch per request into a same-size arena, greedy waves
    pwaves = batch_waves(reqs, arena_bytes)
    arena = torch.empty(arena_bytes // 4, dtype=torch.float32, device="cuda")
    base = arena.data_ptr()
    L = hp.lib()
    import ctypes
    sh = ctypes.c_void_p(stream.cuda_stream)
    plain_args = []
    for wave in pwaves:
        for r, off, ld in wave:
            n = len(r.masses)
            plain_args.append((r.M, n, (ctypes.c_double * n)(*r.masses), r.nevents, r.seed,
                               ctypes.c_void_p(base + off), ld, ctypes.c_void_p(base + off + 4 * n * ld * 4)))

    def plain():
        for M, n, m, nev, seed, out, ld, w in plain_args:
            rc = L.hydra_phsp_generate(M, n, m, nev, seed, 0, 0, out, ld, w, sh)
            if rc:
                raise hp.HydraError(rc, L.hydra_last_error().decode())

    plain()
    torch.cuda.synchronize()
    best_p = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plain()
        torch.cuda.synchronize()
        best_p = min(best_p, time.perf_counter() - t0)
    del arena
    torch.cuda.empty_cache()
    return {"requests": count, "events": total, "output_bytes": out_bytes, "budget_bytes": arena_bytes,
            "batched": {"call": "hydra_phsp_batch_run", "events_per_s": total / best_b, "s": best_b,
                        "hbm_gbs": out_bytes / best_b / 1e9, "waves": waves, "slices": slices,
                        "shape": {"block": shape[0], "ept_by_n": shape[1][2:]}},
            "plain_launches": {"events_per_s": total / best_p, "s": best_p, "waves": len(pwaves),
                               "hbm_gbs": out_bytes / best_p / 1e9},
            "speedup_vs_plain": best_p / best_b}


# ----------------------------------------------------------------------------- extensions
def run_extras(nev: int = 100_000_000, reps: int = 3, hbm_peak_gbs: float | None = None) -> dict:
    """Events/s of the moving-parent generator (per-event parent momenta read from HBM),
    accept-reject unweighting and matrix-element evaluation on stored events (FP32, N=3,
    Dalitz decay, 1e8 events; best of `reps` after one warm-up, CUDA events), with each
    kernel's algorithmic bytes per event and their rate as a fraction of the measured copy
    bandwidth: moving parent 12 B read + 52 B written; unweighting the weights read twice (the
    maximum and the accept pass, 8 B), one accept bit written and read back, and 8 B per kept
    index; evaluation 12 components + the weight read (52 B)."""
    import torch
    import paper_1711_05683_b300 as hp
    d = INT_CFG
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b) / 1e3)
        return best

    moms = torch.randn((3, nev), dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    res = {}
    t = timed(lambda: hp.generate_boosted(d["M"], d["masses"], nev, 3, mothers=moms, dtype="f32"))
    res["boosted_generate_f32_n3"] = {"events_per_s": nev / t, "hbm_gbs": nev * (52 + 12) / t / 1e9}
    p, w = hp.generate(d["M"], d["masses"], nev, 3, dtype="f32")
    t = timed(lambda: hp.unweight(3, w, 3, dtype="f32"))
    kept = len(hp.unweight(3, w, 3, dtype="f32")[0])
    res["unweight_f32_n3"] = {"events_per_s": nev / t, "kept": kept,
                              "hbm_gbs": (nev * (8 + 0.25) + 8 * kept) / t / 1e9}
    t = timed(lambda: hp.evaluate(p, w, me=hp.ME_DALITZ_2BW, params=d["params"], dtype="f32"))
    res["evaluate_dalitz_f32"] = {"events_per_s": nev / t, "hbm_gbs": nev * 52 / t / 1e9}
    if hbm_peak_gbs:
        for key in ("boosted_generate_f32_n3", "unweight_f32_n3", "evaluate_dalitz_f32"):
            res[key]["hbm_frac_of_measured_copy"] = round(res[key]["hbm_gbs"] / hbm_peak_gbs, 4)
    del p, w, moms
    torch.cuda.empty_cache()
    res.update(run_vegas(nev, 10, reps=reps))
    return res


# ----------------------------------------------------------------------------- lambda A/B
def run_lambda_ab(nev: int = 100_000_000, reps: int = 3, ns=(3, 10)) -> dict:
    """FP32 generation (the sweep's massive decays, nev events) with Kallen's lambda as the
    FP32 product of its four gap factors (the default) against the same factors multiplied in
    FP64 (hydra_set_fp32_lambda): ms per launch, best of `reps` after one warm-up, CUDA
    events on the launching stream, both arms at the launch shape the library holds for the
    kernel."""
    import torch
    import paper_1711_05683_b300 as hp
    buf = torch.empty(max(4 * n + 1 for n in ns) * nev, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    out = {"events": nev}
    saved = hp.get_fp32_lambda()
    try:
        for n in ns:
            o = buf[: 4 * n * nev].view(n, 4, nev)
            w = buf[4 * n * nev: (4 * n + 1) * nev]
            masses = workloads.sweep_masses(n, True)
            row = {}
            for name, mode in (("lambda_f32", hp.LAMBDA_FACTORED_F32), ("lambda_f64", hp.LAMBDA_F64)):
                hp.set_fp32_lambda(mode)
                hp.generate_into(workloads.SWEEP_M, masses, nev, 1000 + n, o, w, dtype="f32")
                best = float("inf")
                for _ in range(reps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    hp.generate_into(workloads.SWEEP_M, masses, nev, 1000 + n, o, w, dtype="f32")
                    b.record(stream)
                    b.synchronize()
                    best = min(best, a.elapsed_time(b))
                row[name + "_ms"] = round(best, 4)
            row["slowdown_f64"] = round(row["lambda_f64_ms"] / row["lambda_f32_ms"], 3)
            out[f"N{n}"] = row
    finally:
        hp.set_fp32_lambda(saved)
    return out


# ----------------------------------------------------------------------------- VEGAS
# Thread instructions per point of the double-float VEGAS kernels (ncu smsp__inst_executed.sum
# x 32 / points on 4e6-point iterations, 100 bins).
VEGAS_INSTR_PER_POINT = {("dalitz", "eval"): 1283, ("dalitz", "hist"): 108,
                         ("flat10", "eval"): 2479, ("flat10", "hist"): 457}


def run_vegas(calls: int = 100_000_000, iterations: int = 10, reps: int = 3,
              cases=("dalitz", "flat10")) -> dict:
    """Points/s of hp.vegas (FP64, double-float arithmetic, 100 bins per dimension): the
    Dalitz matrix element (N=3, `calls` points per iteration) and the flat N=10 integrand
    (calls/10 points); the whole call timed (all iterations and grid refinements), best
    of `reps` after one warm-up, with the issue-limit fraction of its kernels."""
    import torch
    import paper_1711_05683_b300 as hp
    d = INT_CFG
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = {}
    for case in cases:
        if case == "dalitz":
            M, m, me, par, c = d["M"], d["masses"], hp.ME_DALITZ_2BW, d["params"], calls
        else:
            M, m, me, par, c = workloads.SWEEP_M, workloads.sweep_masses(10, True), hp.ME_FLAT, (), max(2, calls // 10)
        hp.vegas(M, m, 5, c, iterations, bins=100, me=me, params=par)
        torch.cuda.synchronize()
        best = float("inf")
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        for _ in range(reps):
            t0 = time.perf_counter()
            r = hp.vegas(M, m, 5, c, iterations, bins=100, me=me, params=par)
            best = min(best, time.perf_counter() - t0)
        ck = clocks.stop()
        pps = c * iterations / best
        instr = VEGAS_INSTR_PER_POINT[(case, "eval")] + VEGAS_INSTR_PER_POINT[(case, "hist")] * (iterations - 1) / iterations
        sm_mhz = ck.get("sm_mhz") or ck.get("sm_max_mhz") or 2032.0
        issue_peak = sms * 4 * 32 * sm_mhz * 1e6
        out[f"vegas_{case}_f64"] = {
            "points_per_s": pps, "calls": c, "iterations": iterations, "bins": 100, "seconds": best,
            "mean": r["mean"], "sigma": r["sigma"], "chi2_dof": r["chi2_dof"], "clocks": ck,
            "roofline": {"bound": "alu", "achieved": round(instr * pps / 1e12, 2), "peak": round(issue_peak / 1e12, 2),
                         "unit": "T thread-instructions/s issued", "frac": round(instr * pps / issue_peak, 4),
                         "peak_src": f"SM issue limit: {sms} SMs x 4 schedulers x 32 lanes x {sm_mhz:.0f} MHz"}}
    return out


# ----------------------------------------------------------------------------- serving loop
def run_serve_workload(duration_s: float = 30.0, rate_hz: float = 2000.0) -> dict:
    """Poisson stream (mean rate_hz) of generate (N 2..8, 1e3..1e6 events, float32 out to
    pinned host memory) and Dalitz integrate (1e5..1e8 events) requests, 50/50, served by
    the continuous-batching server (its loop in Python, and the same policy with the loop in
    C++) and by one-at-a-time plain calls; p50/p99 latency from arrival to result in host
    memory, and events/s."""
    import torch
    from paper_1711_05683_b300 import serve
    reqs = workloads.serve_stream(rate_hz=rate_hz, duration_s=duration_s)
    warm = workloads.serve_stream(rate_hz=rate_hz, duration_s=0.5, rng_seed=1)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()  # return what earlier phases cached, before the servers reserve theirs
    srv = serve.Server()
    srv.run(warm)
    res_b = srv.run(reqs)
    srv.close()
    torch.cuda.synchronize()
    nat = serve.NativeServer()  # the same policy with the loop in C++
    nat.run(warm)
    res_n = nat.run(reqs)
    torch.cuda.synchronize()
    plain = serve.PlainServer()
    plain.run(warm)
    res_p = plain.run(reqs, max_wall=duration_s * 3)
    # the same stream replayed 4x faster (8000 requests/s offered): behaviour under load
    fast = [r for r in reqs if r.arrival < duration_s / 2]
    srv = serve.Server()
    res_b4 = srv.run(fast, time_scale=0.25)
    srv.close()
    res_n4 = nat.run(fast, time_scale=0.25)
    nat.close()
    res_p4 = serve.PlainServer().run(fast, time_scale=0.25, max_wall=duration_s * 2)
    for r in (res_b, res_n, res_p, res_b4, res_n4, res_p4):
        r.pop("done", None)
    return {"requests": len(reqs), "duration_s": duration_s, "rate_hz": rate_hz,
            "offered_events": sum(r.nevents for r in reqs), "batched": res_b, "batched_native_loop": res_n,
            "plain": res_p,
            "p99_ratio_plain_over_batched": res_p["p99_ms"] / res_b["p99_ms"] if res_b["p99_ms"] else None,
            "at_4x_rate": {"requests": len(fast), "rate_hz": 4 * rate_hz, "batched": res_b4,
                           "batched_native_loop": res_n4, "plain": res_p4}}


# ----------------------------------------------------------------------------- CPU oracle arm
def cpu_baseline(seconds: float, nev_full: int, int_full: int) -> dict:
    """The oracle (single-threaded FP64 C) on a uniformly scaled-down copy of the step: every
    item on the same fraction of its full event count, sized to take about `seconds`."""
    import oracle
    oracle.build()
    items = oracle_step_items(nev_full, int_full)
    sizes = oracle_sample_sizes(items, seconds)
    t0 = time.perf_counter()
    run_oracle_step(items, sizes)
    wall = time.perf_counter() - t0
    ev = sum(sizes)
    frac = sizes[0] / nev_full
    return {"value": ev / wall, "unit": "events/s", "cores": 1, "kind": "oracle",
            "sample": f"the step scaled down uniformly: {sizes[0]} events per generator item (36) and {sizes[-1]} "
                      f"integrated ({frac:.2e} of the full counts), {wall:.1f} s; FP64 oracle for both precisions",
            "sample_events": {label: k for (label, _, _), k in zip(items, sizes)},
            "host_cores_available": os.cpu_count()}


def _oracle_range(job):
    """One worker's share of an all-cores oracle run (spawned process; the oracle's C library
    is loaded in the worker)."""
    import oracle
    kind, M, masses, count, seed, offset = job
    if kind == "generate":
        oracle.generate(M, masses, count, seed, event_offset=offset)
    else:
        oracle.integrate_sums(M, masses, count, seed, me=1, params=INT_CFG["params"], event_offset=offset)
    return count


def cpu_all_cores(sample: dict, nev_full: int, int_full: int) -> dict:
    """Context only: the same oracle on every host core, each item's sample (4x the
    single-thread sample) split into equal event ranges over a spawned process pool; wall time
    scaled to the item's full count."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    procs = os.cpu_count() or 1
    total_t = 0.0
    total_ev = 0
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_range, [("generate", 10.0, (0.0, 0.0), 64, 1, 0)] * procs)  # warm the workers
        for dtype, massive, n in sweep_items():
            m = 4 * sample[f"{dtype}/{'massive' if massive else 'massless'}/N{n}"]
            part = (m + procs - 1) // procs
            jobs = [("generate", workloads.SWEEP_M, workloads.sweep_masses(n, massive), part, 1000 + n, i * part)
                    for i in range(procs)]
            t0 = time.perf_counter()
            pool.map(_oracle_range, jobs)
            total_t += (time.perf_counter() - t0) * nev_full / (part * procs)
            total_ev += nev_full
        m = 4 * sample["integrate"]
        part = (m + procs - 1) // procs
        jobs = [("integrate", INT_CFG["M"], INT_CFG["masses"], part, INT_CFG["seed"], i * part) for i in range(procs)]
        t0 = time.perf_counter()
        pool.map(_oracle_range, jobs)
        total_t += (time.perf_counter() - t0) * int_full / (part * procs)
        total_ev += int_full
    return {"value": total_ev / total_t, "unit": "events/s", "cores": procs, "kind": "oracle",
            "sample": "every item of the step on all host cores: 4x the single-thread sample split "
                      "into equal event ranges over a spawned process pool, wall time scaled to the "
                      "full count; context, not a baseline"}


def oracle_step_items(nev_full: int, int_full: int):
    """The step's 37 items for the oracle: (label, callable(k), full event count)."""
    import oracle
    items = []
    for dtype, massive, n in sweep_items():
        masses = workloads.sweep_masses(n, massive)
        items.append((f"{dtype}/{'massive' if massive else 'massless'}/N{n}",
                      (lambda k, masses=masses, n=n: oracle.generate(workloads.SWEEP_M, masses, k, 1000 + n)),
                      nev_full))
    items.append(("integrate", lambda k: oracle.integrate(INT_CFG["M"], INT_CFG["masses"], k, INT_CFG["seed"], me=1,
                                                          params=INT_CFG["params"]), int_full))
    return items


def oracle_sample_sizes(items, seconds: float) -> list[int]:
    """Event counts of a uniformly scaled-down step: each item's full count times one fraction,
    chosen from each item's rate on 4096 events (best of two, untimed) so that the sampled step
    takes about `seconds`; the smallest item's count a multiple of 64 (at least 64) and the
    others in exact proportion to their full counts."""
    full_s = 0.0
    for label, fn, full in items:
        best = float("inf")
        for _ in range(2):
            t0 = time.perf_counter()
            fn(4096)
            best = min(best, time.perf_counter() - t0)
        full_s += full * best / 4096
    f = seconds / full_s
    smallest = min(full for _, _, full in items)
    base = int(max(64, round(smallest * f / 64) * 64))  # the smallest item's sample
    return [int(round(base * full / smallest)) for _, _, full in items]


def run_oracle_step(items, sizes) -> None:
    for (label, fn, full), k in zip(items, sizes):
        fn(k)


def run_reference(args) -> None:
    """The reference arm: the oracle (single-threaded FP64 C) on the host cores.  Every step
    is a uniformly scaled-down copy of the CUDA arm's step (each item on the same fraction of
    its full event count, sized once before the warm-up so that a step takes about
    --ref-step-seconds); value = sampled events / timed wall time, ms_per_step = the wall time
    of one such step as run."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    items = oracle_step_items(args.events, args.int_events)
    sizes = oracle_sample_sizes(items, args.ref_step_seconds)
    for _ in range(args.warmup):
        run_oracle_step(items, sizes)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run_oracle_step(items, sizes)
    wall = time.perf_counter() - t0
    ms_per_step = wall / args.steps * 1e3
    ev_step = sum(sizes)
    value = ev_step / (ms_per_step / 1e3)
    full_events = sum(full for _, _, full in items)
    sample = (f"each step: the CUDA arm's step scaled down uniformly, {sizes[0]} events per generator item (36) "
              f"and {sizes[-1]} integrated ({sizes[0] / args.events:.2e} of the full counts); FP64 oracle for "
              "both precisions")
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "events/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "the CUDA arm's step (N-body sweep N=2..10 massless+massive, M=10 GeV, FP32 "
                                   "and FP64; Dalitz integral) scaled down uniformly",
                       "events_per_launch": sizes[0], "integrate_events": sizes[-1], "events_per_step": ev_step,
                       "full_step_events": full_events,
                       "extrapolated_ms_per_full_step": round(full_events / value * 1e3, 1)},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": value},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--events", type=int, default=GEN_EVENTS)
    ap.add_argument("--int-events", type=int, default=INT_CFG["nevents"])
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--arena-gb", type=float, default=40.0)
    ap.add_argument("--workload", default="sweep", choices=["sweep", "batch", "serve", "vegas", "lambda-ab"])
    ap.add_argument("--vegas-calls", type=int, default=100_000_000)
    ap.add_argument("--vegas-iterations", type=int, default=10)
    ap.add_argument("--vegas-case", default="both", choices=["both", "dalitz", "flat10"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--ref-step-seconds", type=float, default=3.0,
                    help="reference arm: wall time of one sampled step of the oracle")
    ap.add_argument("--detail-out", default=None, help="also write the detail record (JSON) to this file")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        import torch
        import paper_1711_05683_b300 as hp
        from paper_1711_05683_b300 import build as hp_build
        hp_build.build()
        torch.cuda.set_device(0)
        hp.lib()
        from paper_1711_05683_b300 import autotune
        tuning = autotune.load_or_tune()
        print(json.dumps({"workload": "batch", "tuning_source": tuning.get("source"),
                          **run_batch_workload(args.batch_count, reps=args.steps,
                                                                   arena_bytes=int(args.arena_gb * 1e9))}),
              flush=True)
    elif args.workload == "serve":
        import torch
        import paper_1711_05683_b300 as hp
        from paper_1711_05683_b300 import build as hp_build
        hp_build.build()
        torch.cuda.set_device(0)
        hp.lib()
        print(json.dumps({"workload": "serve", **run_serve_workload(duration_s=args.serve_seconds)}), flush=True)
    elif args.workload == "lambda-ab":
        import torch
        import paper_1711_05683_b300 as hp
        from paper_1711_05683_b300 import build as hp_build
        hp_build.build()
        torch.cuda.set_device(0)
        hp.lib()
        print(json.dumps({"workload": "lambda-ab", **run_lambda_ab(args.events, reps=args.steps)}), flush=True)
    elif args.workload == "vegas":
        import torch
        import paper_1711_05683_b300 as hp
        from paper_1711_05683_b300 import build as hp_build
        hp_build.build()
        torch.cuda.set_device(0)
        hp.lib()
        cases = ("dalitz", "flat10") if args.vegas_case == "both" else (args.vegas_case,)
        print(json.dumps({"workload": "vegas", **run_vegas(args.vegas_calls, args.vegas_iterations,
                                                           reps=args.steps, cases=cases)}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
