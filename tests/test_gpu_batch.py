"""The batched persistent kernel against the single-request entry points.

A batch slice must give exactly the events of hydra_phsp_generate and exactly the bits of
hydra_phsp_integrate for the same request, whatever else is in the batch, with or without
the CUDA graph, and with integral requests split into slices across runs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def gen_record(rec, M, masses, count, seed, dtype, out, w, first=0, event_offset=0):
    rec["kind"] = hp.REQ_GENERATE
    rec["n"] = len(masses)
    rec["dtype"] = hp.F32 if dtype == "f32" else hp.F64
    rec["M"] = M
    rec["masses"][: len(masses)] = masses
    rec["seed"] = seed
    rec["event_offset"] = event_offset
    rec["first"] = first
    rec["count"] = count
    rec["out"] = out.data_ptr()
    rec["ld"] = out.shape[-1]
    rec["weights"] = w.data_ptr()


def int_record(rec, M, masses, total, seed, dtype, me, params, seg, first, count, event_offset=0):
    rec["kind"] = hp.REQ_INTEGRATE
    rec["n"] = len(masses)
    rec["dtype"] = hp.F32 if dtype == "f32" else hp.F64
    rec["me"] = me
    rec["M"] = M
    rec["masses"][: len(masses)] = masses
    rec["params"][: len(params)] = params
    rec["seed"] = seed
    rec["event_offset"] = event_offset
    rec["first"] = first
    rec["count"] = count
    rec["total"] = total
    rec["seg_partials"] = seg.data_ptr()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("use_graph,reverse", [(True, False), (False, False), (True, True)])
def test_batch_generate_matches_single_calls(dtype, use_graph, reverse):
    """Mixed N (the run hands out tiles grouped by N, in a different order from the table's),
    ragged counts and tails of every events-per-thread group; the table also in reverse."""
    rng = np.random.default_rng(7)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    counts = [1, 3, 5, 2047, 2048, 2049, 10_001, 77_777, 300_000, 4, 123_457, 6, 7, 130, 2050]
    table = np.zeros(len(counts), dtype=hp.request_dtype())
    outs = []
    slots = list(range(len(counts)))[::-1] if reverse else list(range(len(counts)))
    for i, c in zip(slots, counts):
        n = int(rng.integers(2, 11))
        M, masses = workloads.random_decay(rng, n)
        ld = hp.padded_ld(c)
        out = torch.empty((n, 4, ld), dtype=tdt, device="cuda")
        w = torch.empty(ld, dtype=tdt, device="cuda")
        seed, off = int(rng.integers(1, 2 ** 62)), int(rng.integers(0, 2 ** 40))
        gen_record(table[i], M, masses, c, seed, dtype, out, w, event_offset=off)
        outs.append((M, masses, c, seed, off, out, w))
    b = hp.Batch(64)
    b.run(table, use_graph=use_graph)
    torch.cuda.synchronize()
    for M, masses, c, seed, off, out, w in outs:
        p_ref, w_ref = hp.generate(M, masses, c, seed, dtype=dtype, event_offset=off)
        torch.cuda.synchronize()
        assert torch.equal(out[:, :, :c], p_ref[:, :, :c])
        assert torch.equal(w[:c], w_ref)
    b.close()


def test_batch_generate_slices_of_one_request():
    """A request split into slices (first > 0) writes the events of one big call."""
    M, masses = 10.0, workloads.sweep_masses(6, True)
    total = 50_000
    p_ref, w_ref = hp.generate(M, masses, total, 31, dtype="f32", event_offset=9)
    cuts = [0, 1, 4096, 4099, 33_333, total]
    table = np.zeros(len(cuts) - 1, dtype=hp.request_dtype())
    bufs = []
    for i in range(len(cuts) - 1):
        a, z = cuts[i], cuts[i + 1]
        ld = hp.padded_ld(z - a)
        out = torch.empty((6, 4, ld), dtype=torch.float32, device="cuda")
        w = torch.empty(ld, dtype=torch.float32, device="cuda")
        gen_record(table[i], M, masses, z - a, 31, "f32", out, w, first=a, event_offset=9)
        bufs.append((a, z, out, w))
    b = hp.Batch(16)
    b.run(table)
    torch.cuda.synchronize()
    for a, z, out, w in bufs:
        assert torch.equal(out[:, :, : z - a], p_ref[:, :, a:z])
        assert torch.equal(w[: z - a], w_ref[a:z])
    b.close()


@pytest.mark.parametrize("kin", ["f32", "f64"])
def test_batch_integrals_match_single_calls_across_runs(kin):
    """Integral requests sliced over three runs, mixed with generation, give the bits of
    hydra_phsp_integrate."""
    d = workloads.D0_DALITZ
    S = hp.SEGMENT_EVENTS
    reqs = [  # (M, masses, total, seed, me, params, slice sizes)
        (d["M"], d["masses"], 3 * S + 12_345, 5, hp.ME_DALITZ_2BW, d["params"], [S, 2 * S, 12_345]),
        (10.0, workloads.sweep_masses(7, True), 1_000_003, 6, hp.ME_FLAT, (), [1_000_003]),
        (d["M"], d["masses"], 2 * S, 8, hp.ME_DALITZ_2BW, d["params"], [S, S]),
        (5.0, (0.1, 0.2), 5, 9, hp.ME_FLAT, (), [5]),
    ]
    segs = [torch.zeros(8 * hp.segments(r[2]), dtype=torch.float64, device="cuda") for r in reqs]
    b = hp.Batch(32)
    firsts = [0] * len(reqs)
    results = {}
    out = torch.empty((3, 4, 4096), dtype=torch.float32 if kin == "f32" else torch.float64, device="cuda")
    w = torch.empty(4096, dtype=out.dtype, device="cuda")
    for run in range(3):
        recs = []
        for k, (M, masses, total, seed, me, params, slices) in enumerate(reqs):
            if run < len(slices):
                recs.append((k, M, masses, total, seed, me, params, firsts[k], slices[run]))
                firsts[k] += slices[run]
        table = np.zeros(len(recs) + 1, dtype=hp.request_dtype())
        for i, (k, M, masses, total, seed, me, params, first, count) in enumerate(recs):
            int_record(table[i], M, masses, total, seed, kin, me, params, segs[k], first, count,
                       event_offset=1000 * k)
        gen_record(table[len(recs)], d["M"], d["masses"], 4000, 3, kin, out, w)
        b.run(table)
        for i, (k, M, masses, total, seed, me, params, first, count) in enumerate(recs):
            if first + count == total:
                results[k] = b.result(i)
    for k, (M, masses, total, seed, me, params, slices) in enumerate(reqs):
        ref = hp.integrate(M, masses, total, seed, kin_dtype=kin, me=me, params=params,
                           event_offset=1000 * k)
        assert results[k] == ref, (k, results[k], ref)
    b.close()


def test_batch_rejects_bad_slices():
    d = workloads.D0_DALITZ
    b = hp.Batch(4)
    seg = torch.zeros(8 * 4, dtype=torch.float64, device="cuda")
    table = np.zeros(1, dtype=hp.request_dtype())
    int_record(table[0], d["M"], d["masses"], 3 * hp.SEGMENT_EVENTS, 1, "f32", hp.ME_DALITZ_2BW,
               d["params"], seg, first=100, count=1000)
    with pytest.raises(hp.HydraError) as e:
        b.run(table)
    assert e.value.name == "HYDRA_ERR_INVALID_ARG"
    int_record(table[0], d["M"], d["masses"], 3 * hp.SEGMENT_EVENTS, 1, "f32", hp.ME_DALITZ_2BW,
               d["params"], seg, first=0, count=1000)
    with pytest.raises(hp.HydraError):
        b.run(table)  # a slice that does not end its request must hold whole segments
    table[0]["kind"] = hp.REQ_GENERATE
    table[0]["out"] = 0
    with pytest.raises(hp.HydraError):
        b.run(table)
    b.close()


def test_integral_checkpoint_and_resume():
    """An integral's whole running state is (seed, next event index, segment partials): copy
    the partials to the host, drop every device object, restore into a new batch runner and
    continue; the result equals one uninterrupted call bit for bit."""
    d = workloads.D0_DALITZ
    S = hp.SEGMENT_EVENTS
    total = 5 * S + 777
    ref = hp.integrate(d["M"], d["masses"], total, 17, kin_dtype="f32", me=hp.ME_DALITZ_2BW,
                       params=d["params"])
    seg = torch.zeros(8 * hp.segments(total), dtype=torch.float64, device="cuda")
    b = hp.Batch(4)
    t = np.zeros(1, dtype=hp.request_dtype())
    int_record(t[0], d["M"], d["masses"], total, 17, "f32", hp.ME_DALITZ_2BW, d["params"], seg, 0, 3 * S)
    b.run(t)
    torch.cuda.synchronize()
    checkpoint = {"next": 3 * S, "seg": seg.cpu().clone()}
    b.close()
    del seg
    seg2 = checkpoint["seg"].cuda()
    b2 = hp.Batch(4)
    int_record(t[0], d["M"], d["masses"], total, 17, "f32", hp.ME_DALITZ_2BW, d["params"], seg2,
               checkpoint["next"], total - checkpoint["next"])
    b2.run(t)
    assert b2.result(0) == ref
    b2.close()
