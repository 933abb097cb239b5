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


@pytest.mark.parametrize("kind", ["python", "native"])
def test_invalid_request_does_not_end_service(kind):
    """A request below threshold, one with an unknown matrix element and one with n = 11 among
    valid ones: each is answered invalid when it arrives and every other request still gets its
    single-request bits."""
    d = workloads.D0_DALITZ
    reqs = list(workloads.serve_stream(rate_hz=2000, duration_s=0.03, gen_log_events=(2.0, 4.0),
                                       int_log_events=(4.0, 5.0), rng_seed=21))
    bad = [workloads.Request("generate", 1.0, (0.5, 0.4, 0.3), 1000, 5, arrival=reqs[1].arrival),
           workloads.Request("integrate", d["M"], d["masses"], 10_000, 6, me=7, params=d["params"],
                             arrival=reqs[3].arrival),
           workloads.Request("generate", 30.0, (0.1,) * 11, 1000, 7, arrival=reqs[5].arrival)]
    reqs = sorted(reqs + bad, key=lambda r: r.arrival)
    bad_ids = sorted(i for i, r in enumerate(reqs) if any(r is b for b in bad))
    srv = _server(kind, max_slices=256, int_slice_segments=1, pinned_bytes=1 << 28, keep_outputs=True)
    res = srv.run(reqs)
    srv.close()
    assert sorted(res["invalid"]) == bad_ids
    assert res["completed"] == len(reqs) - len(bad)
    for a in res["done"]:
        r = a.req
        if r.kind == "integrate":
            assert a.result == hp.integrate(r.M, r.masses, r.nevents, r.seed, kin_dtype="f32", me=r.me,
                                            params=r.params)
        else:
            p, w = hp.generate(r.M, r.masses, r.nevents, r.seed, dtype="f32")
            torch.cuda.synchronize()
            assert torch.equal(a.host_out[:, :, : r.nevents], p[:, :, : r.nevents].cpu())


def test_native_live_requests_pushed_while_running():
    """Live service: a client thread pushes a stream of generate and integrate requests (real
    arrival spacing) while the C++ loop runs on its worker thread; each outcome, polled by
    ticket from the main thread, equals the single-request result bit for bit."""
    import threading
    import time
    from paper_1711_05683_b300 import serve
    reqs = workloads.serve_stream(rate_hz=2000, duration_s=0.1, gen_log_events=(2.0, 4.5),
                                  int_log_events=(4.0, 6.5), rng_seed=5)
    srv = serve.NativeServer(max_slices=256, int_slice_segments=1, pinned_bytes=1 << 29, keep_outputs=True,
                             budget_bytes=4 * 10 ** 9)
    srv.start()
    tickets = [None] * len(reqs)

    def client():
        t0 = time.perf_counter()
        for i, r in enumerate(reqs):
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            tickets[i] = srv.submit(r)

    th = threading.Thread(target=client)
    th.start()
    th.join()
    outs = [srv.poll(t, timeout=30.0, request=r) for t, r in zip(tickets, reqs)]
    srv.stop(timeout=30.0)
    assert len(set(tickets)) == len(reqs)
    for r, o in zip(reqs, outs):
        assert o["status"] == hp.SERVE_DONE and o["latency"] >= 0.0
        if r.kind == "integrate":
            assert o["result"] == hp.integrate(r.M, r.masses, r.nevents, r.seed, kin_dtype="f32", me=r.me,
                                               params=r.params)
        else:
            p, w = hp.generate(r.M, r.masses, r.nevents, r.seed, dtype="f32")
            torch.cuda.synchronize()
            assert torch.equal(o["host_out"][:, :, : r.nevents], p[:, :, : r.nevents].cpu())
            assert torch.equal(o["host_w"][: r.nevents], w.cpu())
    # a polled ticket is consumed; submitting after stop is refused
    with pytest.raises(hp.HydraError):
        srv.poll(tickets[0], timeout=0.0)
    with pytest.raises(hp.HydraError):
        srv.submit(reqs[0])
    srv.close()


def test_native_live_submit_validates_at_once():
    from paper_1711_05683_b300 import serve
    srv = serve.NativeServer(max_slices=16, pinned_bytes=1 << 24, budget_bytes=1 << 28)
    srv.start()
    with pytest.raises(hp.HydraError) as e:
        srv.submit(workloads.Request("generate", 1.0, (0.5, 0.6), 100, 1))
    assert e.value.name == "HYDRA_ERR_BELOW_THRESHOLD"
    srv.stop(timeout=5.0)
    srv.close()


def test_native_deadline_times_out_and_destroys_cleanly():
    """A 20 ms deadline on a run whose integral needs thousands of 2^21-event ticks: the run ends
    with HYDRA_ERR_TIMEOUT after its ticks in flight, the integral is answered timed out, small
    requests that finished before keep their results, and the server is reusable and then
    destroyed cleanly; the same for a live server stopped with a short timeout."""
    from paper_1711_05683_b300 import serve
    d = workloads.D0_DALITZ
    big = workloads.Request("integrate", d["M"], d["masses"], 4000 * 2 ** 21, 9, me=1, params=d["params"],
                            arrival=0.0)
    small = workloads.Request("generate", 5.0, (0.1, 0.2, 0.3), 1000, 3, arrival=0.0)
    srv = serve.NativeServer(max_slices=64, int_slice_segments=1, pinned_bytes=1 << 26, keep_outputs=True,
                             budget_bytes=1 << 30)
    srv.set_deadline(0.02)
    res = srv.run([small, big])
    assert res["deadline_passed"] and res["timed_out"] == [1]
    srv.set_deadline(0.0)
    again = srv.run([workloads.Request("generate", 5.0, (0.1, 0.2, 0.3), 1000, 4, arrival=0.0)])
    assert again["completed"] == 1 and not again["deadline_passed"]
    srv.start()
    t_big = srv.submit(big)
    with pytest.raises(hp.HydraError) as e:
        srv.stop(timeout=0.005)
    assert e.value.name == "HYDRA_ERR_TIMEOUT"
    assert srv.poll(t_big, timeout=0.0)["status"] == hp.SERVE_TIMED_OUT
    srv.close()


def test_native_live_concurrent_clients_and_withdrawal():
    """Four client threads submit at once (the server's inbox is shared); one client withdraws
    its long integral 2 ms after submitting it.  Every other outcome equals the single-request
    result; the withdrawn one is reported withdrawn."""
    import threading
    from paper_1711_05683_b300 import serve
    d = workloads.D0_DALITZ
    reqs = list(workloads.serve_stream(rate_hz=4000, duration_s=0.05, gen_log_events=(2.0, 4.0),
                                       int_log_events=(4.0, 6.0), rng_seed=8))
    big = workloads.Request("integrate", d["M"], d["masses"], 2000 * 2 ** 21, 77, me=1, params=d["params"])
    srv = serve.NativeServer(max_slices=256, int_slice_segments=1, pinned_bytes=1 << 28, keep_outputs=True,
                             budget_bytes=2 * 10 ** 9)
    srv.start()
    tickets = {}
    lock = threading.Lock()

    def client(c):
        for i in range(c, len(reqs), 4):
            t = srv.submit(reqs[i])
            with lock:
                tickets[i] = t

    threads = [threading.Thread(target=client, args=(c,)) for c in range(4)]
    for th in threads:
        th.start()
    t_big = srv.submit(big, withdraw=0.002)
    for th in threads:
        th.join()
    outs = {i: srv.poll(t, timeout=30.0, request=reqs[i]) for i, t in tickets.items()}
    o_big = srv.poll(t_big, timeout=30.0, request=big)
    srv.stop(timeout=30.0)
    srv.close()
    assert o_big["status"] == hp.SERVE_WITHDRAWN
    assert len(set(tickets.values()) | {t_big}) == len(reqs) + 1
    for i, o in outs.items():
        r = reqs[i]
        assert o["status"] == hp.SERVE_DONE
        if r.kind == "integrate":
            assert o["result"] == hp.integrate(r.M, r.masses, r.nevents, r.seed, kin_dtype="f32", me=r.me,
                                               params=r.params)
        else:
            p, w = hp.generate(r.M, r.masses, r.nevents, r.seed, dtype="f32")
            torch.cuda.synchronize()
            assert torch.equal(o["host_out"][:, :, : r.nevents], p[:, :, : r.nevents].cpu())
