"""Host-side checks of bench.py's output contract and roofline arithmetic (no GPU).

The driver reads exactly one JSON line from stdout; it must stay short (the tail of stdout
is what is kept) and carry the required keys.  The reference arm (the oracle on host cores)
is run here on a tiny sampled step; the CUDA arm's roofline helpers are checked directly.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

REQUIRED = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
            "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def test_reference_arm_prints_one_short_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--ref-step-seconds", "0.4"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    assert len(lines[0]) < 2048
    line = json.loads(lines[0])
    for k in REQUIRED:
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    # the timed region it reports is the one it ran: steps x ms_per_step well under a minute here
    assert line["steps"] * line["ms_per_step"] < 60_000
    cfg = line["config"]
    assert cfg["events_per_step"] == 36 * cfg["events_per_launch"] + cfg["integrate_events"]
    # the sample is the full step scaled down uniformly: integral / generator item = 10 (1e9 / 1e8)
    assert abs(cfg["integrate_events"] / cfg["events_per_launch"] - 10.0) < 0.01
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


@pytest.mark.parametrize("n", range(2, 11))
def test_method_ops_totals(n):
    # 48 per boosted two-body step, 31 for the parent's decay, 1 for C_n; massless: 43 and 26
    assert bench.fp_ops_per_event(n) == 48 * (n - 2) + 32
    assert bench.fp_ops_per_event(n, massless=True) == 43 * (n - 2) + 27
    ops = bench.method_ops(n)
    assert all(v >= 0 for v in ops.values())
    assert ops["sincos"] == n - 1 and ops["div"] == n - 2


def test_fp_ceiling_uses_each_rate():
    rates = {"add": 1.0, "mul": 2.0, "fma": 4.0, "sqrt": 8.0, "rcp": 16.0}
    ops = {"add": 1, "mul": 2, "fma": 4, "sqrt": 8, "rcp": 16, "div": 1, "sincos": 8}
    # 1 + 1 + 1 + 1 + 1 + (1/16 + 1/2) + 1
    assert bench.fp_seconds_per_event(ops, rates) == pytest.approx(6.5625)
