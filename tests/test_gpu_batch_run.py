"""hydra_phsp_batch_run: whole requests under a device-memory budget, split into waves inside
the library, against the single-request entry points (same events bit for bit, same integral
bits) and, on sampled events, against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1711_05683_b300 as hp  # noqa: E402
import workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_05683_b300 import build as hp_build
    hp_build.build()
    torch.cuda.set_device(0)


def fill(rec, kind, M, masses, nevents, seed, dtype="f32", event_offset=0, me=0, params=(), dest=hp.DEST_NONE,
         out=None, weights=None, ld=0):
    rec["kind"], rec["n"], rec["dtype"], rec["me"], rec["M"] = kind, len(masses), hp._dtype_code(dtype), me, M
    rec["masses"][: len(masses)] = masses
    rec["params"][: len(params)] = params
    rec["seed"], rec["event_offset"], rec["nevents"], rec["dest"] = seed, event_offset, nevents, dest
    rec["out"] = 0 if out is None else out
    rec["weights"] = 0 if weights is None else weights
    rec["ld"] = ld


def host_arrays(n, nevents, ld, dtype):
    tdt = torch.float32 if dtype == "f32" else torch.float64
    out = torch.full((n, 4, ld), float("nan"), dtype=tdt, pin_memory=True)
    w = torch.full((nevents,), float("nan"), dtype=tdt, pin_memory=True)
    return out, w


def single(M, masses, nevents, seed, dtype, event_offset=0):
    p, w = hp.generate(M, masses, nevents, seed, dtype=dtype, event_offset=event_offset)
    torch.cuda.synchronize()
    return p[:, :, :nevents].cpu(), w[:nevents].cpu()


def test_c4_mix_over_several_waves_matches_single_calls_and_oracle():
    """A sample of the uneven C4 mix (N 2..8, M 1..10 GeV, per-request seeds, events
    log-uniform) to pinned host memory with a 96 MB budget: several waves, requests larger than
    half the arena split across waves, every event equal to a single call bit for bit, and a
    few events of each of the first requests equal to the oracle within the FP32 tolerance."""
    reqs = workloads.batch_requests(48, log_events=(3.0, 5.6))
    table = np.zeros(len(reqs), dtype=hp.batch_request_dtype())
    hosts = []
    for i, r in enumerate(reqs):
        ld = r.nevents + 5  # a host row stride that is not a multiple of 4
        out, w = host_arrays(len(r.masses), r.nevents, ld, "f32")
        fill(table[i], hp.REQ_GENERATE, r.M, r.masses, r.nevents, r.seed, dest=hp.DEST_HOST,
             out=out.data_ptr(), weights=w.data_ptr(), ld=ld)
        hosts.append((out, w))
    hp.batch_run(table, 96 << 20)
    waves, slices = hp.batch_stats()
    assert waves >= 2 and slices >= len(reqs), (waves, slices)
    assert (table["status"] == 0).all()
    for i, r in enumerate(reqs):
        p1, w1 = single(r.M, r.masses, r.nevents, r.seed, "f32")
        out, w = hosts[i]
        assert torch.equal(out[:, :, : r.nevents], p1), i
        assert torch.equal(w, w1), i
    for i, r in enumerate(reqs[:6]):
        k = min(r.nevents, 200)
        ref_p, ref_w = oracle.generate(r.M, r.masses, k, r.seed)
        gp = hosts[i][0][:, :, :k].double().numpy()
        scale = np.maximum(r.M, ref_p[:, 0, :].max(axis=0))
        assert float((np.abs(gp - ref_p) / scale).max()) <= 2e-5
        assert float((np.abs(hosts[i][1][:k].double().numpy() - ref_w) / ref_w).max()) <= 2e-5


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_mixed_destinations_and_integrals_match_single_calls(dtype):
    """Generate requests to device buffers, to the host and dropped, with Dalitz and flat
    integrals (one longer than a 2^26-event slice) in one call: device and host outputs equal
    single calls bit for bit, integral results equal hydra_phsp_integrate bit for bit."""
    rng = np.random.default_rng(11)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    d = workloads.D0_DALITZ
    specs = []
    for i in range(9):
        n = int(rng.integers(2, 11))
        M, masses = workloads.random_decay(rng, n)
        specs.append(("gen", M, masses, int(rng.integers(1, 200_000)), [hp.DEST_DEVICE, hp.DEST_HOST, hp.DEST_NONE][i % 3]))
    specs.insert(2, ("int", d["M"], d["masses"], 3_000_001, hp.ME_DALITZ_2BW))
    specs.insert(6, ("int", 7.0, (0.3, 0.2, 0.1, 0.4), (1 << 26) + 12_345, hp.ME_FLAT))
    table = np.zeros(len(specs), dtype=hp.batch_request_dtype())
    keep = []
    for i, (kind, M, masses, nev, x) in enumerate(specs):
        seed, off = int(rng.integers(1, 2 ** 62)), int(rng.integers(0, 2 ** 40))
        if kind == "int":
            fill(table[i], hp.REQ_INTEGRATE, M, masses, nev, seed, dtype, off, me=x,
                 params=d["params"] if x == hp.ME_DALITZ_2BW else ())
            keep.append(None)
            continue
        n = len(masses)
        if x == hp.DEST_DEVICE:
            ld = hp.padded_ld(nev)
            out = torch.empty((n, 4, ld), dtype=tdt, device="cuda")
            w = torch.empty(ld, dtype=tdt, device="cuda")
        elif x == hp.DEST_HOST:
            ld = nev
            out, w = host_arrays(n, nev, ld, dtype)
        else:
            ld, out, w = 0, None, None
        fill(table[i], hp.REQ_GENERATE, M, masses, nev, seed, dtype, off, dest=x,
             out=None if out is None else out.data_ptr(), weights=None if w is None else w.data_ptr(), ld=ld)
        keep.append((out, w))
    hp.batch_run(table, 1 << 30)
    torch.cuda.synchronize()
    for i, (kind, M, masses, nev, x) in enumerate(specs):
        rec = table[i]
        assert rec["status"] == 0
        if kind == "int":
            ref = hp.integrate(M, masses, nev, int(rec["seed"]), kin_dtype=dtype, me=x,
                               params=d["params"] if x == hp.ME_DALITZ_2BW else (), event_offset=int(rec["event_offset"]))
            for k in ("mean", "var_mean", "sum_f", "sum_f2", "sum_w", "sum_w2"):
                assert float(rec["result"][k]) == ref[k], (i, k)
            assert int(rec["result"]["n"]) == nev
        elif x != hp.DEST_NONE:
            out, w = keep[i]
            p1, w1 = single(M, masses, nev, int(rec["seed"]), dtype, int(rec["event_offset"]))
            assert torch.equal(out[:, :, :nev].cpu(), p1) and torch.equal(w[:nev].cpu(), w1), i


def test_repeated_calls_reuse_and_shape_does_not_change_results():
    """Two calls in a row (the second reuses the kept buffers) and a call after another batch
    launch shape give the same bits."""
    reqs = workloads.batch_requests(12, log_events=(3.0, 5.0), base_seed=77)
    res = []
    saved = hp.get_batch_shape("f32")
    try:
        for shape in (None, None, (512, [1] * 11), (128, [2, 2, 2, 4, 4, 4, 4, 1, 2, 1, 2])):
            if shape:
                hp.set_batch_shape("f32", *shape)
            table = np.zeros(len(reqs), dtype=hp.batch_request_dtype())
            outs = []
            for i, r in enumerate(reqs):
                out, w = host_arrays(len(r.masses), r.nevents, r.nevents, "f32")
                fill(table[i], hp.REQ_GENERATE, r.M, r.masses, r.nevents, r.seed, dest=hp.DEST_HOST,
                     out=out.data_ptr(), weights=w.data_ptr(), ld=r.nevents)
                outs.append((out, w))
            hp.batch_run(table, 64 << 20)
            res.append(outs)
    finally:
        hp.set_batch_shape("f32", saved[0], saved[1])
    for outs in res[1:]:
        for (a, b), (c, e) in zip(res[0], outs):
            assert torch.equal(a, c) and torch.equal(b, e)


def test_invalid_request_launches_nothing():
    """A request below threshold among valid ones: its status and the call's error say so,
    and no output is written."""
    table = np.zeros(3, dtype=hp.batch_request_dtype())
    outs = []
    for i in range(3):
        out, w = host_arrays(3, 1000, 1000, "f32")
        masses = (1.0, 2.0, 3.0) if i == 1 else (0.1, 0.2, 0.3)
        fill(table[i], hp.REQ_GENERATE, 5.0, masses, 1000, 3 + i, dest=hp.DEST_HOST, out=out.data_ptr(),
             weights=w.data_ptr(), ld=1000)
        outs.append((out, w))
    with pytest.raises(hp.HydraError):
        hp.batch_run(table, 64 << 20)
    assert table["status"][1] == 2 and table["status"][0] == 0
    assert all(torch.isnan(o).all() for o, _ in outs)


def test_integrals_only_fp64():
    """Only integral requests (FP64, flat and Dalitz, one longer than 2^26 events): no arena is
    needed; every result equals hydra_phsp_integrate bit for bit."""
    d = workloads.D0_DALITZ
    specs = [(d["M"], d["masses"], 5_000_003, hp.ME_DALITZ_2BW, d["params"]),
             (10.0, workloads.sweep_masses(6, True), (1 << 26) + 1, hp.ME_FLAT, ()),
             (3.0, (0.1, 0.2), 77, hp.ME_FLAT, ())]
    table = np.zeros(len(specs), dtype=hp.batch_request_dtype())
    for i, (M, masses, nev, me, par) in enumerate(specs):
        fill(table[i], hp.REQ_INTEGRATE, M, masses, nev, 100 + i, "f64", event_offset=i << 40, me=me, params=par)
    hp.batch_run(table, 256 << 20)
    for i, (M, masses, nev, me, par) in enumerate(specs):
        ref = hp.integrate(M, masses, nev, 100 + i, kin_dtype="f64", me=me, params=par, event_offset=i << 40)
        for k in ("mean", "var_mean", "sum_f", "sum_f2", "sum_w", "sum_w2"):
            assert float(table[i]["result"][k]) == ref[k], (i, k)


def test_one_wave_per_request_then_a_larger_budget():
    """A budget that holds one request's outputs per wave (every request its own wave), then the
    same requests with a budget 16 times larger (the kept arena is replaced): same bits."""
    rng = np.random.default_rng(3)
    reqs = []
    for i in range(6):
        n = 8 - i % 2  # 17-20 MB of outputs each: more than half of the small budget's arena
        M, masses = workloads.random_decay(rng, n)
        reqs.append((M, masses, 150_000 + 1000 * i, 900 + i))
    outs = []
    for budget in (24 << 20, 384 << 20):
        table = np.zeros(len(reqs), dtype=hp.batch_request_dtype())
        keep = []
        for i, (M, masses, nev, seed) in enumerate(reqs):
            out, w = host_arrays(len(masses), nev, nev, "f32")
            fill(table[i], hp.REQ_GENERATE, M, masses, nev, seed, dest=hp.DEST_HOST, out=out.data_ptr(),
                 weights=w.data_ptr(), ld=nev)
            keep.append((out, w))
        hp.batch_run(table, budget)
        outs.append((hp.batch_stats(), keep))
    (w_small, _), small = outs[0]
    (w_large, _), large = outs[1]
    assert w_small >= len(reqs) > w_large
    for (a, b), (c, e), (M, masses, nev, seed) in zip(small, large, reqs):
        assert torch.equal(a, c) and torch.equal(b, e)
        p1, w1 = single(M, masses, nev, seed, "f32")
        assert torch.equal(a, p1) and torch.equal(b, w1)


def test_c4_full_mix_sampled():
    """Config C4 at full size, as bench.py runs it: the 4096 uneven requests (4.6e9 events,
    ~390 GB of FP32 outputs) through one hydra_phsp_batch_run call with a 40 GB budget; the
    outputs of every request are dropped with their wave except those of 8 sampled requests
    (first, last, the largest, and five others), which go to device buffers.  Each sampled
    request equals a single call bit for bit and, on 64 of its events, the oracle."""
    reqs = workloads.batch_requests(4096)
    sample = sorted({0, 4095, max(range(4096), key=lambda i: reqs[i].nevents), 17, 1000, 2048, 3001, 3999})
    table = np.zeros(len(reqs), dtype=hp.batch_request_dtype())
    bufs = {}
    for i, r in enumerate(reqs):
        if i in sample:
            ld = hp.padded_ld(r.nevents)
            out = torch.empty((len(r.masses), 4, ld), dtype=torch.float32, device="cuda")
            w = torch.empty(ld, dtype=torch.float32, device="cuda")
            bufs[i] = (out, w)
            fill(table[i], hp.REQ_GENERATE, r.M, r.masses, r.nevents, r.seed, dest=hp.DEST_DEVICE,
                 out=out.data_ptr(), weights=w.data_ptr(), ld=ld)
        else:
            fill(table[i], hp.REQ_GENERATE, r.M, r.masses, r.nevents, r.seed)
    try:
        hp.batch_run(table, 40 * 10 ** 9)
        waves, slices = hp.batch_stats()
        assert waves >= 9 and slices >= len(reqs)
        torch.cuda.synchronize()
        for i in sample:
            r = reqs[i]
            out, w = bufs[i]
            p1, w1 = single(r.M, r.masses, r.nevents, r.seed, "f32")
            assert torch.equal(out[:, :, : r.nevents].cpu(), p1) and torch.equal(w[: r.nevents].cpu(), w1), i
            k = min(64, r.nevents)
            ref_p, ref_w = oracle.generate(r.M, r.masses, k, r.seed)
            scale = np.maximum(r.M, ref_p[:, 0, :].max(axis=0))
            assert float((np.abs(out[:, :, :k].double().cpu().numpy() - ref_p) / scale).max()) <= 2e-5
            assert float((np.abs(w[:k].double().cpu().numpy() - ref_w) / ref_w).max()) <= 2e-5
    finally:
        del bufs
        hp.shutdown()  # release the call's kept 40 GB arena
        torch.cuda.empty_cache()
