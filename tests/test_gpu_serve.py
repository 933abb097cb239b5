"""The continuous-batching server: every request's result is the same alone (single-request
entry points) and in the mix, bit for bit, and latencies are recorded for all requests."""
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


def _server(kind, **kw):
    from paper_1711_05683_b300 import serve
    return (serve.NativeServer if kind == "native" else serve.Server)(**kw)


@pytest.mark.parametrize("kind", ["python", "native"])
@pytest.mark.parametrize("tick_cap", [1 << 27, 1 << 18])
def test_served_results_equal_single_requests(tick_cap, kind):
    """Every request's result alone equals its result in the mix; with a small per-tick event
    cap the same stream runs as many short oldest-first ticks and still gives the same bits;
    for the Python loop and the C++ loop (hydra_server_run)."""
    reqs = workloads.serve_stream(rate_hz=2000, duration_s=0.15, gen_log_events=(2.0, 5.0),
                                  int_log_events=(4.0, 7.4), rng_seed=99)
    assert any(r.kind == "integrate" and r.nevents > 2 ** 21 for r in reqs)  # sliced over ticks
    srv = _server(kind, max_slices=512, int_slice_segments=1, pinned_bytes=1 << 30, keep_outputs=True,
                  budget_bytes=8 * 10 ** 9, max_tick_events=tick_cap)
    res = srv.run(reqs)
    srv.close()
    assert res["completed"] == len(reqs)
    assert res["ticks"] > 1
    for a in res["done"]:
        r = a.req
        if r.kind == "generate":
            p, w = hp.generate(r.M, r.masses, r.nevents, r.seed, dtype="f32")
            torch.cuda.synchronize()
            assert torch.equal(a.host_out[:, :, : r.nevents], p[:, :, : r.nevents].cpu())
            assert torch.equal(a.host_w[: r.nevents], w.cpu())
        else:
            ref = hp.integrate(r.M, r.masses, r.nevents, r.seed, kin_dtype="f32", me=r.me, params=r.params)
            assert a.result == ref


def test_plain_server_matches_too():
    from paper_1711_05683_b300 import serve
    reqs = workloads.serve_stream(rate_hz=500, duration_s=0.05, gen_log_events=(2.0, 4.0),
                                  int_log_events=(4.0, 5.0), rng_seed=3)
    res = serve.PlainServer(keep_outputs=True).run(reqs)
    assert res["completed"] == len(reqs) and res["p99_ms"] >= res["p50_ms"]


@pytest.mark.parametrize("kind", ["python", "native"])
def test_cancelled_request_leaves_the_others_intact(kind):
    """Host-side fault injection: a client withdraws a long integral mid-flight; the server
    drops it between ticks and every other request still gets its single-request result.  The
    integral is 1000 ticks of 2^21 events (tens of ms of GPU work), so it is still running when
    the client withdraws it 5 ms into the run on any GPU."""
    from paper_1711_05683_b300 import serve
    d = workloads.D0_DALITZ
    reqs = workloads.serve_stream(rate_hz=1000, duration_s=0.05, gen_log_events=(2.0, 4.0),
                                  int_log_events=(4.0, 5.0), rng_seed=11)
    big = workloads.Request("integrate", d["M"], d["masses"], 1000 * 2 ** 21, 123, me=1,
                            params=d["params"], arrival=0.0)
    reqs = [big] + list(reqs)
    srv = _server(kind, max_slices=256, int_slice_segments=1, pinned_bytes=1 << 28, keep_outputs=True)
    res = srv.run(reqs, cancel_after={0: 0.005})
    srv.close()
    assert res["cancelled"] == [0]
    assert res["completed"] == len(reqs) - 1
    assert res["ticks"] < 1000  # withdrawn before its last slice
    for a in res["done"]:
        r = a.req
        assert a.rid != 0
        if r.kind == "integrate":
            assert a.result == hp.integrate(r.M, r.masses, r.nevents, r.seed, kin_dtype="f32", me=r.me,
                                            params=r.params)
        else:
            p, w = hp.generate(r.M, r.masses, r.nevents, r.seed, dtype="f32")
            assert torch.equal(a.host_w[: r.nevents], w.cpu())


@pytest.mark.parametrize("kind", ["python", "native"])
def test_tight_budget_waits_for_space_and_refuses_what_never_fits(kind):
    """Admission by budget: with a 96 MB budget the requests are admitted as earlier ones free
    their blocks, every result still equals the single-request one, and a request larger than
    the whole budget is refused instead of blocking the queue.  The device ring wraps several
    times while outputs are still being copied to the host on the copy stream, so a block
    handed out again before its copy had landed would show in the outputs."""
    from paper_1711_05683_b300 import serve
    reqs = workloads.serve_stream(rate_hz=4000, duration_s=0.05, gen_log_events=(5.0, 5.6),
                                  int_log_events=(4.0, 5.0), rng_seed=21)
    huge = workloads.Request("generate", 5.0, (0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8), 2_000_000, 77,
                             arrival=0.01)
    reqs = sorted(list(reqs) + [huge], key=lambda r: r.arrival)
    big_rid = reqs.index(huge)
    gen_bytes = sum((4 * len(r.masses) + 1) * hp.padded_ld(r.nevents) * 4 for r in reqs
                    if r.kind == "generate" and r is not huge)
    srv = _server(kind, max_slices=64, int_slice_segments=1, pinned_bytes=4 << 30, keep_outputs=True,
                  budget_bytes=96 * 10 ** 6)
    srv_dev_ring_size = 96 * 10 ** 6 - min(256 << 20, 96 * 10 ** 6 // 16)
    assert srv_dev_ring_size < gen_bytes < 4 << 30  # the device budget is the tight one
    res = srv.run(reqs, max_wall=60.0)
    srv.close()
    assert res["refused"] == [big_rid]
    assert res["completed"] == len(reqs) - 1
    for a in res["done"]:
        r = a.req
        if r.kind == "generate":
            p, w = hp.generate(r.M, r.masses, r.nevents, r.seed, dtype="f32")
            torch.cuda.synchronize()
            assert torch.equal(a.host_out[:, :, : r.nevents], p[:, :, : r.nevents].cpu())
            assert torch.equal(a.host_w[: r.nevents], w.cpu())
        else:
            assert a.result == hp.integrate(r.M, r.masses, r.nevents, r.seed, kin_dtype="f32", me=r.me,
                                            params=r.params)
    assert gen_bytes > 3 * srv_dev_ring_size


@pytest.mark.parametrize("kind", ["python", "native"])
def test_kept_outputs_filling_the_pinned_ring_are_refused_not_waited_for(kind):
    """With keep_outputs the pinned ring is never released; once it is full, later generate
    requests are refused (nothing could ever free space) and the run ends."""
    from paper_1711_05683_b300 import serve
    reqs = workloads.serve_stream(rate_hz=2000, duration_s=0.05, gen_log_events=(5.0, 5.3),
                                  int_log_events=(4.0, 4.5), rng_seed=5)
    srv = _server(kind, max_slices=64, int_slice_segments=1, pinned_bytes=64 << 20, keep_outputs=True,
                  budget_bytes=2 * 10 ** 9)
    res = srv.run(reqs, max_wall=60.0)
    srv.close()
    gens = [i for i, r in enumerate(reqs) if r.kind == "generate"]
    assert res["refused"] and set(res["refused"]) <= set(gens)
    assert res["completed"] + len(res["refused"]) == len(reqs)
