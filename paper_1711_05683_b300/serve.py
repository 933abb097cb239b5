"""Continuous-batching server for phase-space requests (generate and integrate).

Requests arrive over time.  Each tick the server admits arrived requests while their
device memory fits the HBM budget, then packs one slice of each active request, oldest first
and up to `max_tick_events` events per tick (so that under overload requests still finish
close to arrival order), into one batch run (hydra_batch_run: one persistent launch,
replayed CUDA graph):
  * a generate request is one slice (its whole event count); its events land in a device
    staging buffer and are copied to pinned host memory right after the run;
  * an integrate request advances by up to `int_slice_segments` segments of 2^21 events per
    tick (16 by default: a 1e8-event integral takes 3 ticks); its running state is device resident: the next counter-event index (the Philox
    counter, kept on the host as an integer) and its compensated segment partial sums
    (a caller-owned device array the batch kernels update in place).  A long integral
    therefore shares the GPU with requests that arrive while it runs.
Two batch runners alternate so that tick i+1 is packed and enqueued while tick i runs.  The
copies of finished generate outputs to pinned host memory go on a stream of their own, which
waits for the tick's kernels: the next ticks compute while earlier outputs cross the host link,
and requests that copy nothing (integrals) do not queue behind other requests' copies.  An
integrate request completes when the host observes the event recorded after its last slice; a
generate request when it observes the event recorded after its copy; latency = completion
time - arrival time.

The HBM budget is reserved when the server starts, as two device rings (staging outputs, and
integral partials in a small ring of their own); requests take blocks of them and return them
when harvested, so the serving loop never allocates device memory (an allocation can
synchronise the device and stall every request in flight).  Pinned host memory is a ring in
the same way.

Every slice computes exactly the events of the single-request entry points, so a request's
result is the same alone and in the mix (tests check this bit for bit).  A request that would
not fit the budget even with nothing else admitted, or that cannot be admitted while nothing
is active or in flight (so nothing would ever release memory, e.g. when kept outputs have
filled the pinned ring), is refused (listed in the result's "refused") instead of blocking
the queue.

`PlainServer` is the comparison: one request at a time in arrival order with the
single-request entry points (generate + copy to host, or integrate).
"""
from __future__ import annotations

import contextlib
import dataclasses
import gc
import time
from collections import deque

import numpy as np

import paper_1711_05683_b300 as hp


@contextlib.contextmanager
def _no_gc_pauses():
    """The serving loops run with Python's cyclic garbage collector off: a full collection
    over the tens of thousands of request records alive in a run pauses the loop for tens of
    milliseconds, which lands directly in the latency tail.  Reference counting still frees
    everything the loops drop; the collector is restored afterwards."""
    was = gc.isenabled()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


@dataclasses.dataclass
class _Active:
    rid: int
    req: object                     # workloads.Request
    arrival: float                  # absolute wall time
    next_first: int = 0             # next event index (the request's RNG counter)
    nbytes: int = 0
    ld: int = 0                     # generate: row stride of the [n, 4, ld] outputs
    host_out: object = None         # generate, kept outputs: pinned host copy [n, 4, ld]
    host_w: object = None           #   and its weights
    result: dict | None = None
    done_tick: int = -1
    ring_start: int = -1            # block of the pinned host ring (generate)
    dev_start: int = -1             # block of the device arena (staging or partials)
    latency: float = -1.0           # seconds from arrival to completion
    rec: object = None              # the request's hydra_request record (static fields)


class Ring:
    """A byte buffer (pinned host or device memory) handed out in arrival order as a ring of
    256-byte-aligned blocks; blocks may be released in any order (when their request is
    harvested) and a block is only handed out where it overlaps no live one."""

    def __init__(self, buf):
        self.buf = buf
        self.size = buf.numel()
        self.head = 0
        self.live = deque()  # (start, end) in allocation order

    def alloc(self, nbytes: int):
        nbytes = (nbytes + 255) // 256 * 256
        if nbytes > self.size:
            return None
        start = self.head if self.head + nbytes <= self.size else 0
        end = start + nbytes
        for s, e in self.live:
            if s < end and start < e:
                return None
        self.head = end
        self.live.append((start, end))
        return start

    def free(self, start: int):
        for i, (s, _e) in enumerate(self.live):
            if s == start:
                del self.live[i]
                return

    def view(self, start: int, nbytes: int, dtype):
        return self.buf[start: start + nbytes].view(dtype)


def PinnedRing(nbytes: int) -> Ring:
    import torch
    return Ring(torch.empty(nbytes, dtype=torch.uint8, pin_memory=True))


def DeviceRing(nbytes: int) -> Ring:
    import torch
    return Ring(torch.empty(nbytes, dtype=torch.uint8, device="cuda"))


class Server:
    def __init__(self, budget_bytes: int = 40 * 10 ** 9, max_slices: int = 4096,
                 int_slice_segments: int = 16, pinned_bytes: int = 4 << 30,
                 keep_outputs: bool = False, use_graph: bool = True, max_tick_events: int = 1 << 27):
        import torch
        self.torch = torch
        self.budget = budget_bytes
        self.used = 0
        self.int_slice = int_slice_segments * hp.SEGMENT_EVENTS
        self.runners = [hp.Batch(max_slices, max_integrate_tiles=max_slices * int_slice_segments * 1024),
                        hp.Batch(max_slices, max_integrate_tiles=max_slices * int_slice_segments * 1024)]
        self.table = np.zeros(max_slices, dtype=hp.request_dtype())
        self.max_slices = max_slices
        self.ring = PinnedRing(pinned_bytes)
        # staging outputs and (in a small ring of their own, so that long integrals do not
        # split the large one) integral partials; together they are the HBM budget
        self.seg_ring = DeviceRing(min(256 << 20, budget_bytes // 16))
        self.dev_ring = DeviceRing(budget_bytes - self.seg_ring.size)
        self.dev_base, self.seg_base = self.dev_ring.buf.data_ptr(), self.seg_ring.buf.data_ptr()
        self.keep_outputs = keep_outputs
        self.use_graph = use_graph
        self.max_tick_events = max_tick_events
        self.stream = torch.cuda.current_stream()
        self.copy_stream = torch.cuda.Stream()  # device-to-host copies of finished generate outputs

    # ------------------------------------------------------------------ state per request
    def _fits_ever(self, a: _Active) -> bool:
        """Whether the request could be admitted into empty rings (else it is refused)."""
        r = a.req
        if r.kind == "generate":
            nbytes = (4 * len(r.masses) + 1) * hp.padded_ld(r.nevents) * 4
            return nbytes <= self.dev_ring.size and nbytes <= self.ring.size
        return 64 * hp.segments(r.nevents) <= self.seg_ring.size

    def _admit(self, a: _Active) -> bool:
        """Reserve the request's ring blocks (integer offsets only: admission runs for every
        request inside the loop, so it creates no tensors) and build its record."""
        r = a.req
        if r.kind == "generate":
            ld = hp.padded_ld(r.nevents)
            nbytes = (4 * len(r.masses) + 1) * ld * 4
            dev = self.dev_ring.alloc(nbytes)
            if dev is None:
                return False
            host = self.ring.alloc(nbytes)
            if host is None:
                self.dev_ring.free(dev)
                return False
            a.ring_start, a.dev_start, a.ld = host, dev, ld
        else:
            nbytes = 64 * hp.segments(r.nevents)
            dev = self.seg_ring.alloc(nbytes)
            if dev is None:
                return False
            a.dev_start = dev
        a.nbytes = nbytes
        self.used += nbytes
        a.rec = np.zeros(1, dtype=self.table.dtype)[0]
        self._fill(a.rec, a)
        return True

    def _copy_to_host(self, a: _Active):
        """One copy of the request's whole block ([n, 4, ld] outputs then weights, the same
        layout on both sides) from the device ring to the pinned ring, on the current stream."""
        self.ring.buf[a.ring_start: a.ring_start + a.nbytes].copy_(
            self.dev_ring.buf[a.dev_start: a.dev_start + a.nbytes], non_blocking=True)

    def _release(self, a: _Active):
        self.used -= a.nbytes
        if a.req.kind == "generate":
            self.dev_ring.free(a.dev_start)
            if self.keep_outputs:
                n, ld = len(a.req.masses), a.ld
                hb = self.ring.view(a.ring_start, a.nbytes, self.torch.float32)
                a.host_out, a.host_w = hb[: 4 * n * ld].view(n, 4, ld), hb[4 * n * ld:]
            else:
                self.ring.free(a.ring_start)
        else:
            self.seg_ring.free(a.dev_start)

    def _fill(self, rec, a: _Active):
        """The request's static fields (the slice start and count are set per tick)."""
        r = a.req
        n = len(r.masses)
        rec["n"], rec["dtype"], rec["M"] = n, hp.F32, r.M
        rec["masses"][:n] = r.masses
        rec["seed"], rec["event_offset"] = r.seed, 0
        if r.kind == "generate":
            out = self.dev_base + a.dev_start
            rec["kind"] = hp.REQ_GENERATE
            rec["out"], rec["ld"], rec["weights"] = out, a.ld, out + 4 * n * a.ld * 4
        else:
            rec["kind"], rec["me"] = hp.REQ_INTEGRATE, r.me
            rec["params"][: len(r.params)] = r.params
            rec["total"], rec["seg_partials"] = r.nevents, self.seg_base + a.dev_start

    # ------------------------------------------------------------------ the loop
    def run(self, requests, time_scale: float = 1.0, max_wall: float | None = None,
            cancel_after: dict | None = None) -> dict:
        """Serve `requests` (sorted by arrival, seconds from start); returns latencies and
        throughput.  time_scale stretches the arrival times.  cancel_after maps a request
        index to a time (seconds from start) after which the client withdraws it: the server
        drops it at the next tick boundary and releases its memory (host-side fault
        injection; work already on the GPU finishes and is discarded)."""
        with _no_gc_pauses():
            return self._run(requests, time_scale, max_wall, cancel_after)

    def _run(self, requests, time_scale, max_wall, cancel_after) -> dict:
        torch = self.torch
        cancel_after = dict(cancel_after or {})
        cancelled, refused, invalid = [], [], []
        t0 = time.perf_counter()
        pending = deque(enumerate(requests))
        queue: deque[_Active] = deque()
        active: list[_Active] = []
        inflight: deque = deque()  # (tick, event, runner index, [(slot, active)], [finished integrals])
        copying: deque = deque()   # (copy-stream event, [finished generate requests])
        latencies, kinds, done = {}, {}, []
        tick = 0
        events_done = 0

        def complete(a: _Active, tnow: float):
            nonlocal events_done
            a.latency = latencies[a.rid] = tnow - a.arrival
            kinds[a.rid] = a.req.kind
            events_done += a.req.nevents
            done.append(a)
            self._release(a)

        while pending or queue or active or inflight or copying:
            now = time.perf_counter()
            if max_wall is not None and now - t0 > max_wall:
                break
            while pending and t0 + pending[0][1].arrival * time_scale <= now:
                rid, r = pending.popleft()
                if not _valid(r):  # answered at once; the others are served as usual
                    invalid.append(rid)
                    continue
                queue.append(_Active(rid, r, t0 + r.arrival * time_scale))
            while queue and len(active) < self.max_slices:
                if not self._fits_ever(queue[0]):  # larger than the budget: refused, not queued forever
                    refused.append(queue.popleft().rid)
                    continue
                if not self._admit(queue[0]):
                    if not active and not inflight and not copying:
                        # nothing will release memory (kept outputs fill the pinned ring): refuse
                        refused.append(queue.popleft().rid)
                        continue
                    break
                active.append(queue.popleft())
            # harvest finished ticks (oldest first): integrals complete with their last slice
            while inflight and (len(inflight) >= 2 or inflight[0][1].query()):
                t_i, ev, ri, slots, finishing = inflight.popleft()
                ev.synchronize()
                tnow = time.perf_counter()
                ending = {id(a) for a in finishing}
                for slot, a in slots:
                    if id(a) in ending:
                        a.result = self.runners[ri].result(slot)
                for a in finishing:
                    complete(a, tnow)
            # generate requests complete when their copy to host memory has landed
            while copying and copying[0][0].query():
                _evc, copied = copying.popleft()
                tnow = time.perf_counter()
                for a in copied:
                    complete(a, tnow)
            if cancel_after:
                keep = []
                for a in active:
                    t_c = cancel_after.get(a.rid)
                    if t_c is not None and now - t0 >= t_c and a.next_first < a.req.nevents:
                        cancelled.append(a.rid)
                        self._release(a)
                    else:
                        keep.append(a)
                active = keep
            launchable = [a for a in active if a.next_first < a.req.nevents]
            if launchable and len(inflight) < 2:
                ri = tick % 2
                slots, finishing = [], []
                room = self.max_tick_events  # oldest first, up to this many events per tick
                for a in launchable:
                    if a.req.kind == "generate":
                        count = a.req.nevents
                    else:
                        count = min(self.int_slice, a.req.nevents - a.next_first)
                    if slots and count > room:
                        break
                    room -= count
                    k = len(slots)
                    self.table[k] = a.rec
                    self.table[k]["first"] = a.next_first
                    self.table[k]["count"] = count
                    slots.append((k, a))
                    a.next_first += count
                    if a.next_first >= a.req.nevents:
                        finishing.append(a)
                self.runners[ri].run(self.table, len(slots), use_graph=self.use_graph, stream=self.stream)
                ev = torch.cuda.Event()
                ev.record(self.stream)
                copied = [a for a in finishing if a.req.kind == "generate"]
                if copied:
                    self.copy_stream.wait_event(ev)
                    with torch.cuda.stream(self.copy_stream):
                        for a in copied:
                            self._copy_to_host(a)
                    evc = torch.cuda.Event()
                    evc.record(self.copy_stream)
                    copying.append((evc, copied))
                inflight.append((tick, ev, ri, slots, [a for a in finishing if a.req.kind == "integrate"]))
                active = [a for a in active if a.next_first < a.req.nevents]
                tick += 1
            elif not inflight and not active and not queue and pending:
                wait = t0 + pending[0][1].arrival * time_scale - time.perf_counter()
                if wait > 0:
                    time.sleep(min(wait, 2e-4))
            elif (inflight and not inflight[0][1].query()) or (copying and not copying[0][0].query()):
                time.sleep(2e-5)
        wall = time.perf_counter() - t0
        out = _summary(latencies, events_done, wall, ticks=tick, done=done, kinds=kinds)
        out["cancelled"] = cancelled
        out["refused"] = refused
        out["invalid"] = invalid
        return out

    def close(self):
        for r in self.runners:
            r.close()
        self.dev_ring = self.seg_ring = None


def _valid(r) -> bool:
    """The checks of the single-request entry points, on the host: n, masses and threshold (the
    library's hydra_phsp_volume_factor), the kind, a positive count and, for integrals, a known
    matrix element with its parameters."""
    import math
    if r.kind not in ("generate", "integrate") or r.nevents <= 0:
        return False
    try:
        hp.volume_factor(r.M, r.masses)
    except hp.HydraError:
        return False
    if r.kind == "integrate":
        if r.me == hp.ME_DALITZ_2BW:
            return len(r.masses) == 3 and len(r.params) >= 6 and all(math.isfinite(v) for v in r.params[:6])
        return r.me == hp.ME_FLAT
    return True


class NativeServer:
    """The same serving policy with the loop in C++ (hydra_server_run: rings, two batch runners,
    the copy stream and the harvest without the interpreter in the loop).  The pinned ring is a
    page-locked host tensor owned here; results match `Server`'s, request by request, bit for
    bit, client withdrawal (cancel_after) included."""

    def __init__(self, budget_bytes: int = 40 * 10 ** 9, max_slices: int = 4096, int_slice_segments: int = 16,
                 pinned_bytes: int = 4 << 30, keep_outputs: bool = False, max_tick_events: int = 1 << 27):
        import ctypes
        import torch
        self.torch = torch
        self.keep_outputs = keep_outputs
        self.pinned = torch.empty(pinned_bytes, dtype=torch.uint8, pin_memory=True)
        h = ctypes.c_void_p()
        hp._check(hp.lib().hydra_server_create(int(budget_bytes), ctypes.c_void_p(self.pinned.data_ptr()),
                                               int(pinned_bytes), int(max_slices), int(int_slice_segments),
                                               int(max_tick_events), int(bool(keep_outputs)), ctypes.byref(h)))
        self._h = h

    def run(self, requests, time_scale: float = 1.0, max_wall: float | None = None,
            cancel_after: dict | None = None) -> dict:
        """Serve `requests` (sorted by arrival); cancel_after maps a request index to the time
        (seconds from the start) at which its client withdraws it.  max_wall is not used: the
        C++ loop runs until every request has completed, been refused or been withdrawn."""
        import ctypes
        torch = self.torch
        reqs = list(requests)
        cancel_after = dict(cancel_after or {})
        table = np.zeros(len(reqs), dtype=hp.serve_request_dtype())
        table["withdraw"] = -1.0
        for i, r in enumerate(reqs):
            rec = table[i]
            if i in cancel_after:
                rec["withdraw"] = float(cancel_after[i])
            n = len(r.masses)
            rec["arrival"], rec["n"], rec["M"] = r.arrival, n, r.M
            rec["kind"] = hp.REQ_GENERATE if r.kind == "generate" else hp.REQ_INTEGRATE
            rec["masses"][: min(n, 10)] = r.masses[:10]  # n > 10 is answered invalid by the loop
            rec["nevents"], rec["seed"], rec["me"] = r.nevents, r.seed, r.me
            rec["params"][: len(r.params)] = r.params
        outc = np.zeros(max(1, len(reqs)), dtype=hp.serve_outcome_dtype())
        wall, ticks = ctypes.c_double(), ctypes.c_uint64()
        with _no_gc_pauses():
            status = hp.lib().hydra_server_run(self._h, ctypes.c_void_p(table.ctypes.data), len(reqs),
                                               float(time_scale), ctypes.c_void_p(outc.ctypes.data),
                                               ctypes.byref(wall), ctypes.byref(ticks))
        deadline_passed = status == 7  # HYDRA_ERR_TIMEOUT: every request has an outcome all the same
        if not deadline_passed:
            hp._check(status)
        latencies, kinds, done, refused, cancelled, invalid, timed_out = {}, {}, [], [], [], [], []
        events = 0
        for i, r in enumerate(reqs):
            o = outc[i]
            if o["status"] != hp.SERVE_DONE:
                {hp.SERVE_WITHDRAWN: cancelled, hp.SERVE_INVALID: invalid,
                 hp.SERVE_TIMED_OUT: timed_out}.get(int(o["status"]), refused).append(i)
                continue
            a = _Active(i, r, r.arrival * time_scale)
            a.latency = latencies[i] = float(o["latency"])
            kinds[i] = r.kind
            events += r.nevents
            if r.kind == "integrate":
                a.result = {k: (int(o["result"][k]) if k == "n" else float(o["result"][k]))
                            for k in o["result"].dtype.names}
            elif self.keep_outputs:
                n, ld, off = len(r.masses), int(o["ld"]), int(o["host_offset"])
                hb = self.pinned[off: off + (4 * n + 1) * ld * 4].view(torch.float32)
                a.host_out, a.host_w = hb[: 4 * n * ld].view(n, 4, ld), hb[4 * n * ld:]
            done.append(a)
        out = _summary(latencies, events, wall.value, ticks=int(ticks.value), done=done, kinds=kinds)
        out["cancelled"] = cancelled
        out["refused"] = refused
        out["invalid"] = invalid
        out["timed_out"] = timed_out
        out["deadline_passed"] = deadline_passed
        return out

    def set_deadline(self, seconds: float) -> None:
        """Wall-clock limit of a run (0: none); a run that passes it raises HydraError with
        HYDRA_ERR_TIMEOUT after its ticks in flight have finished."""
        hp._check(hp.lib().hydra_server_set_deadline(self._h, float(seconds)))

    # -- live service: requests submitted while the C++ loop runs on its worker thread
    def start(self) -> None:
        hp._check(hp.lib().hydra_server_start(self._h))

    def submit(self, r, withdraw: float | None = None) -> int:
        """Queue request `r` (a workloads.Request); returns its ticket.  Invalid requests raise
        HydraError at once."""
        import ctypes
        rec = np.zeros(1, dtype=hp.serve_request_dtype())[0]
        n = len(r.masses)
        rec["kind"] = hp.REQ_GENERATE if r.kind == "generate" else hp.REQ_INTEGRATE
        rec["n"], rec["M"], rec["nevents"], rec["seed"], rec["me"] = n, r.M, r.nevents, r.seed, r.me
        rec["masses"][: min(n, 10)] = r.masses[:10]  # n > 10 is refused by the submission's checks
        rec["params"][: len(r.params)] = r.params
        rec["withdraw"] = -1.0 if withdraw is None else float(withdraw)
        arr = np.array([rec])
        ticket = ctypes.c_uint64()
        hp._check(hp.lib().hydra_server_submit(self._h, ctypes.c_void_p(arr.ctypes.data), ctypes.byref(ticket)))
        return ticket.value

    def poll(self, ticket: int, timeout: float = 10.0, request=None) -> dict:
        """Wait for a ticket's outcome: {"status", "latency", "result" or host views}."""
        import ctypes
        outc = np.zeros(1, dtype=hp.serve_outcome_dtype())
        hp._check(hp.lib().hydra_server_poll(self._h, int(ticket), float(timeout), ctypes.c_void_p(outc.ctypes.data)))
        o = outc[0]
        res = {"status": int(o["status"]), "latency": float(o["latency"])}
        if res["status"] == hp.SERVE_DONE and request is not None:
            if request.kind == "integrate":
                res["result"] = {k: (int(o["result"][k]) if k == "n" else float(o["result"][k]))
                                 for k in o["result"].dtype.names}
            elif self.keep_outputs:
                n, ld, off = len(request.masses), int(o["ld"]), int(o["host_offset"])
                hb = self.pinned[off: off + (4 * n + 1) * ld * 4].view(self.torch.float32)
                res["host_out"], res["host_w"] = hb[: 4 * n * ld].view(n, 4, ld), hb[4 * n * ld:]
        return res

    def stop(self, timeout: float = 60.0) -> None:
        hp._check(hp.lib().hydra_server_stop(self._h, float(timeout)))

    def close(self):
        if self._h:
            hp.lib().hydra_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PlainServer:
    """One request at a time, in arrival order, with the single-request entry points; generated
    events are copied to the same kind of pinned ring as the batched server uses."""

    def __init__(self, keep_outputs: bool = False, pinned_bytes: int = 4 << 30):
        import torch
        self.torch = torch
        self.keep_outputs = keep_outputs
        self.stream = torch.cuda.current_stream()
        self.ring = PinnedRing(pinned_bytes)
        self.dev = torch.empty(0, dtype=torch.uint8, device="cuda")  # staging, grown on demand

    def _staging(self, nbytes: int):
        if self.dev.numel() < nbytes:
            self.dev = self.torch.empty(max(nbytes, 2 * self.dev.numel()), dtype=self.torch.uint8, device="cuda")
        return self.dev[:nbytes]

    def run(self, requests, time_scale: float = 1.0, max_wall: float | None = None) -> dict:
        with _no_gc_pauses():
            return self._run(requests, time_scale, max_wall)

    def _run(self, requests, time_scale, max_wall) -> dict:
        torch = self.torch
        t0 = time.perf_counter()
        latencies, kinds, done = {}, {}, []
        events_done = 0
        for rid, r in enumerate(requests):
            arr = t0 + r.arrival * time_scale
            while time.perf_counter() < arr:
                time.sleep(min(2e-4, max(0.0, arr - time.perf_counter())))
            if max_wall is not None and time.perf_counter() - t0 > max_wall:
                break
            a = _Active(rid, r, arr)
            if r.kind == "generate":
                n = len(r.masses)
                ld = hp.padded_ld(r.nevents)
                nbytes = (4 * n + 1) * ld * 4
                db = self._staging(nbytes).view(torch.float32)
                p, w = db[: 4 * n * ld].view(n, 4, ld), db[4 * n * ld:]
                hp.generate_into(r.M, r.masses, r.nevents, r.seed, p, w, dtype="f32")
                start = self.ring.alloc(nbytes)
                if start is None:  # ring full: everything before is finished (synchronous server)
                    self.ring.live.clear()
                    start = self.ring.alloc(nbytes)
                hb = self.ring.buf[start: start + nbytes].view(torch.float32)
                ho, hw = hb[: 4 * n * ld].view(n, 4, ld), hb[4 * n * ld:]
                ho.copy_(p, non_blocking=True)
                hw.copy_(w, non_blocking=True)
                self.stream.synchronize()
                if self.keep_outputs:
                    a.host_out, a.host_w = ho.clone(), hw.clone()
                self.ring.free(start)
            else:
                a.result = hp.integrate(r.M, r.masses, r.nevents, r.seed, kin_dtype="f32", me=r.me,
                                        params=r.params)
            a.latency = latencies[rid] = time.perf_counter() - arr
            kinds[rid] = r.kind
            events_done += r.nevents
            done.append(a)
        wall = time.perf_counter() - t0
        return _summary(latencies, events_done, wall, done=done, kinds=kinds)


def _summary(latencies: dict, events: int, wall: float, ticks: int = 0, done=None, kinds=None) -> dict:
    lat = np.array(sorted(latencies.values())) if latencies else np.zeros(1)
    out = {"completed": len(latencies), "events": events, "wall_s": wall,
           "events_per_s": events / wall if wall > 0 else 0.0,
           "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "max_ms": float(lat.max() * 1e3), "ticks": ticks, "done": done}
    for kind in ("generate", "integrate"):
        v = np.array([latencies[k] for k in latencies if kinds and kinds.get(k) == kind])
        if len(v):
            out[kind] = {"n": int(len(v)), "p50_ms": float(np.percentile(v, 50) * 1e3),
                         "p99_ms": float(np.percentile(v, 99) * 1e3)}
    return out
