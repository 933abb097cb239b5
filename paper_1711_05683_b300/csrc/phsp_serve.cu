// phsp_serve.cu -- the continuous-batching serving loop in C++ (host code over hydra_batch_*).
//
// The same policy as the Python server (serve.py), without the interpreter in the loop:
// requests arrive over time; each turn of the loop admits arrived requests while their memory
// fits two device rings (staging outputs; integral segment partials) and the caller's pinned
// ring, harvests finished ticks and landed copies, and, with fewer than two ticks in flight,
// packs one slice of every active request, oldest first and up to max_tick_events events,
// into one batch run.  A generate request is one slice whose outputs are copied to the pinned
// ring on a copy stream that waits for the tick; an integral advances by int_slice_segments
// segments of 2^21 events per tick with its segment partials resident in the device ring.  A
// request that can never fit, or that cannot be admitted while nothing is active or in flight,
// is refused; a request that fails validation (the checks of hydra_phsp_generate /
// hydra_phsp_integrate) is marked invalid and the others are served as usual.  Every slice
// computes exactly the events of the single-request entry points.
//
// Requests come from one of two sources: an array replayed by arrival time (hydra_server_run)
// or requests submitted from any thread while a worker thread runs the loop
// (hydra_server_start / _submit / _poll / _stop).  A wall-clock deadline ends a run: no new
// tick is launched, the ticks in flight (bounded GPU work) are waited for, and requests not
// finished by then are marked as timed out.
//
// Every ring block is checked against its ring before a record is built from it, so a
// bookkeeping error ends the run with an error status instead of a kernel touching memory
// outside the rings.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <limits>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "hydra_phsp.h"
#include "phsp_host.h"
#include "phsp_integral.cuh"
#include "phsp_ring.h"

namespace {

using hydra::Ring;
constexpr uint64_t kSegmentEvents = uint64_t{1} << 21;
constexpr double kNever = std::numeric_limits<double>::infinity();

// One request inside the loop.
struct Entry {
    hydra_serve_request q{};
    int id = 0;               // index in the caller's array (replay) or in arrival order (live)
    uint64_t ticket = 0;      // live service
    double arrival = 0.0;     // seconds on the loop's clock
    double withdraw_at = kNever;
    uint64_t next_first = 0, nbytes = 0, ld = 0, dev = 0, host = 0;
    hydra_request rec{};
    bool finished = false;
};

struct Tick {
    cudaEvent_t ev;
    int runner;
    std::vector<std::pair<int, Entry*>> slots;
    std::vector<Entry*> integrals;  // integral requests whose last slice this tick runs
};

struct Copy {
    cudaEvent_t ev;
    std::vector<Entry*> gens;
};

using Clock = std::chrono::steady_clock;

// Where requests come from and where outcomes go.
struct Source {
    virtual ~Source() = default;
    // Append the requests that have arrived by `now` (loop clock) to `store` and `arrived`;
    // false once no further request will ever come.
    virtual bool take(double now, std::deque<Entry>& store, std::deque<Entry*>& arrived) = 0;
    // With nothing to do: wait until the next arrival may be due (at most `max_wait` seconds).
    virtual void idle(double now, double max_wait) = 0;
    virtual void finished(Entry* e, const hydra_serve_outcome& o) = 0;
};

// Checks of the single-request entry points: n, kind and count, the decay (masses, M,
// threshold) and, for integrals, the matrix element and its parameters.
hydra_status validate(const hydra_serve_request& q) {
    if (q.n < 2 || q.n > 10) return hydra::fail(HYDRA_ERR_UNSUPPORTED_N, "n = %d outside [2, 10]", q.n);
    if (q.kind != HYDRA_REQ_GENERATE && q.kind != HYDRA_REQ_INTEGRATE)
        return hydra::fail(HYDRA_ERR_INVALID_ARG, "unknown kind %d", q.kind);
    if (q.nevents == 0) return hydra::fail(HYDRA_ERR_INVALID_ARG, "nevents must be > 0");
    hydra::DecayConsts C;
    hydra_status st = hydra::make_consts(q.M, q.n, q.masses, q.seed, &C);
    if (st == HYDRA_OK && q.kind == HYDRA_REQ_INTEGRATE) {
        hydra::MEConsts P;
        st = hydra::make_me(static_cast<hydra_me_id>(q.me), q.n, q.params, 6, &P);
    }
    return st;
}

}  // namespace

struct hydra_server {
    int device = 0;
    uint64_t budget = 0;
    int max_slices = 0;
    uint64_t int_slice = 0, max_tick_events = 0;
    int keep_outputs = 0;
    double deadline = 0.0;              // seconds a run may take (0: no limit)
    unsigned char* dev_base = nullptr;  // staging ring then segment ring
    Ring dev_ring, seg_ring, host_ring;
    unsigned char* host_base = nullptr;  // the caller's pinned ring
    hydra_batch* runners[2] = {nullptr, nullptr};
    cudaStream_t compute = nullptr, copy = nullptr;
    std::vector<cudaEvent_t> events;  // free events
    // live service
    std::mutex mu;
    std::condition_variable cv;  // a submission, an outcome or the end of the loop
    std::thread worker;
    bool live = false, stopping = false, loop_done = false;
    std::atomic<double> stop_deadline{kNever};  // loop clock at which a stopping loop gives up
    Clock::time_point live_t0;
    struct Submitted {
        uint64_t ticket;
        hydra_serve_request q;
        double at;
    };
    std::deque<Submitted> inbox;
    std::unordered_map<uint64_t, hydra_serve_outcome> results;
    uint64_t next_ticket = 1;
    hydra_status live_status = HYDRA_OK;
    std::string live_error;
};

using namespace hydra;

namespace {

cudaEvent_t take_event(hydra_server* s) {
    if (!s->events.empty()) {
        cudaEvent_t e = s->events.back();
        s->events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

hydra_serve_outcome blank_outcome(int32_t status) {
    hydra_serve_outcome o{};
    o.latency = -1.0;
    o.host_offset = ~uint64_t{0};
    o.status = status;
    return o;
}

// The serving loop over one source.  `t0` is the loop clock's origin.
hydra_status serve_loop(hydra_server* s, Source& src, Clock::time_point t0, double run_deadline, double* wall_s,
                        uint64_t* ticks_out) {
    int prev_device = 0;
    cudaGetDevice(&prev_device);
    cudaError_t derr = cudaSetDevice(s->device);
    if (derr != cudaSuccess) return cuda_fail(derr, "server device");
    unsigned char* seg_base = s->dev_base + s->dev_ring.size;
    std::deque<Entry> store;
    std::deque<Entry*> queue;
    std::vector<Entry*> active;
    std::deque<Tick> inflight;
    std::deque<Copy> copying;
    std::vector<hydra_request> table;
    table.reserve(static_cast<size_t>(s->max_slices));
    uint64_t tick = 0;
    bool more = true;
    auto clock = [&]() { return std::chrono::duration<double>(Clock::now() - t0).count(); };
    hydra_status st = HYDRA_OK;

    auto finish = [&](Entry* a, hydra_serve_outcome o) {
        a->finished = true;
        src.finished(a, o);
    };
    auto release = [&](Entry* a) {
        if (a->rec.kind == HYDRA_REQ_GENERATE) {
            s->dev_ring.release(a->dev);
            s->host_ring.release(a->host);
        } else {
            s->seg_ring.release(a->dev);
        }
    };
    auto complete = [&](Entry* a, double tnow, const hydra_integral* res) {
        hydra_serve_outcome o = blank_outcome(HYDRA_SERVE_DONE);
        o.latency = tnow - a->arrival;
        if (a->rec.kind == HYDRA_REQ_GENERATE) {
            s->dev_ring.release(a->dev);
            if (s->keep_outputs) {
                o.host_offset = a->host;
                o.ld = a->ld;
            } else {
                s->host_ring.release(a->host);
            }
        } else {
            s->seg_ring.release(a->dev);
            if (res) o.result = *res;
        }
        finish(a, o);
    };
    auto fits_ever = [&](const hydra_serve_request& q) {
        if (q.kind == HYDRA_REQ_GENERATE) {
            const uint64_t ld = std::max<uint64_t>(4, (q.nevents + 3) / 4 * 4);
            const uint64_t nb = (4 * static_cast<uint64_t>(q.n) + 1) * ld * 4;
            return nb <= s->dev_ring.size && nb <= s->host_ring.size;
        }
        return 64 * ((q.nevents + kSegmentEvents - 1) / kSegmentEvents) <= s->seg_ring.size;
    };
    // 1: admitted; 0: no room now; -1: a ring handed out a block outside itself (internal error)
    auto admit = [&](Entry* a) -> int {
        const hydra_serve_request& q = a->q;
        hydra_request& r = a->rec;
        std::memset(&r, 0, sizeof r);
        r.n = q.n;
        r.dtype = HYDRA_F32;
        r.M = q.M;
        for (int i = 0; i < q.n; ++i) r.masses[i] = q.masses[i];
        r.seed = q.seed;
        if (q.kind == HYDRA_REQ_GENERATE) {
            a->ld = std::max<uint64_t>(4, (q.nevents + 3) / 4 * 4);
            a->nbytes = (4 * static_cast<uint64_t>(q.n) + 1) * a->ld * 4;
            if (!s->dev_ring.alloc(a->nbytes, &a->dev)) return 0;
            if (!s->host_ring.alloc(a->nbytes, &a->host)) {
                s->dev_ring.release(a->dev);
                return 0;
            }
            if (a->dev + a->nbytes > s->dev_ring.size || a->host + a->nbytes > s->host_ring.size) return -1;
            r.kind = HYDRA_REQ_GENERATE;
            r.out = s->dev_base + a->dev;
            r.ld = a->ld;
            r.weights = s->dev_base + a->dev + 4 * static_cast<uint64_t>(q.n) * a->ld * 4;
        } else {
            a->nbytes = 64 * ((q.nevents + kSegmentEvents - 1) / kSegmentEvents);
            if (!s->seg_ring.alloc(a->nbytes, &a->dev)) return 0;
            if (a->dev + a->nbytes > s->seg_ring.size) return -1;
            r.kind = HYDRA_REQ_INTEGRATE;
            r.me = q.me;
            for (int i = 0; i < 6; ++i) r.params[i] = q.params[i];
            r.total = q.nevents;
            r.seg_partials = reinterpret_cast<double*>(seg_base + a->dev);
        }
        return 1;
    };
    // finished ticks, oldest first (all of them when `all`): integrals complete with their last slice
    auto harvest_ticks = [&](bool all) {
        while (!inflight.empty() && (all || inflight.size() >= 2 || cudaEventQuery(inflight.front().ev) == cudaSuccess)) {
            Tick t = std::move(inflight.front());
            inflight.pop_front();
            const cudaError_t err = cudaEventSynchronize(t.ev);
            s->events.push_back(t.ev);
            if (err != cudaSuccess) return cuda_fail(err, "server tick");
            const double tnow = clock();
            for (const auto& sl : t.slots) {
                if (std::find(t.integrals.begin(), t.integrals.end(), sl.second) == t.integrals.end()) continue;
                hydra_integral res{};
                const hydra_status rs = hydra_batch_result(s->runners[t.runner], sl.first, &res);
                if (rs != HYDRA_OK) return rs;
                complete(sl.second, tnow, &res);
            }
        }
        return HYDRA_OK;
    };
    // generate requests complete when their copy to host memory has landed
    auto harvest_copies = [&](bool all) {
        while (!copying.empty() && (all || cudaEventQuery(copying.front().ev) == cudaSuccess)) {
            Copy c = std::move(copying.front());
            copying.pop_front();
            const cudaError_t err = cudaEventSynchronize(c.ev);
            s->events.push_back(c.ev);
            if (err != cudaSuccess) return cuda_fail(err, "server copy");
            const double tnow = clock();
            for (Entry* a : c.gens) complete(a, tnow, nullptr);
        }
        return HYDRA_OK;
    };

    while (st == HYDRA_OK) {
        const double now = clock();
        if (more) {
            const size_t before = store.size();
            more = src.take(now, store, queue);
            // invalid requests are answered at once; the others wait in arrival order
            for (size_t i = before; i < store.size(); ++i) {
                Entry* a = &store[i];
                if (validate(a->q) != HYDRA_OK) {
                    queue.erase(std::find(queue.begin(), queue.end(), a));
                    finish(a, blank_outcome(HYDRA_SERVE_INVALID));
                }
            }
        }
        if (!more && queue.empty() && active.empty() && inflight.empty() && copying.empty()) break;
        const double deadline = std::min(run_deadline, s->stop_deadline.load());
        if (now > deadline) {
            st = fail(HYDRA_ERR_TIMEOUT, "server run exceeded its deadline of %.3f s", deadline);
            break;
        }
        while (!queue.empty() && static_cast<int>(active.size()) < s->max_slices) {
            Entry* a = queue.front();
            if (!fits_ever(a->q)) {  // larger than the rings: refused, not queued forever
                queue.pop_front();
                finish(a, blank_outcome(HYDRA_SERVE_REFUSED));
                continue;
            }
            const int adm = admit(a);
            if (adm < 0) {
                st = fail(HYDRA_ERR_INVALID_ARG, "server ring handed out a block outside itself");
                break;
            }
            if (adm == 0) {
                if (active.empty() && inflight.empty() && copying.empty()) {  // nothing would release memory
                    queue.pop_front();
                    finish(a, blank_outcome(HYDRA_SERVE_REFUSED));
                    continue;
                }
                break;
            }
            active.push_back(a);
            queue.pop_front();
        }
        if (st != HYDRA_OK) break;
        st = harvest_ticks(false);
        if (st != HYDRA_OK) break;
        // client withdrawal between ticks: an admitted request not yet fully launched is dropped
        // and its memory released (slices already in flight finish on the compute stream before
        // any later use of the released blocks)
        active.erase(std::remove_if(active.begin(), active.end(), [&](Entry* a) {
                         if (now < a->withdraw_at || a->next_first >= a->q.nevents) return false;
                         release(a);
                         finish(a, blank_outcome(HYDRA_SERVE_WITHDRAWN));
                         return true;
                     }),
                     active.end());
        st = harvest_copies(false);
        if (st != HYDRA_OK) break;
        bool launched = false;
        if (inflight.size() < 2) {
            table.clear();
            Tick t;
            t.runner = static_cast<int>(tick % 2);
            std::vector<Entry*> gens;
            uint64_t room = s->max_tick_events;
            for (Entry* a : active) {
                const hydra_serve_request& q = a->q;
                if (a->next_first >= q.nevents) continue;
                const uint64_t count = q.kind == HYDRA_REQ_GENERATE ? q.nevents
                                                                    : std::min(s->int_slice, q.nevents - a->next_first);
                if (!table.empty() && count > room) break;
                room = count > room ? 0 : room - count;
                hydra_request r = a->rec;
                r.first = a->next_first;
                r.count = count;
                t.slots.emplace_back(static_cast<int>(table.size()), a);
                table.push_back(r);
                a->next_first += count;
                if (a->next_first >= q.nevents) (q.kind == HYDRA_REQ_GENERATE ? gens : t.integrals).push_back(a);
                if (static_cast<int>(table.size()) >= s->max_slices) break;
            }
            if (!table.empty()) {
                const NvtxRange nvtx_tick("hydra_server_tick");
                st = hydra_batch_run(s->runners[t.runner], table.data(), static_cast<int>(table.size()), 1,
                                     reinterpret_cast<hydra_stream_t>(s->compute));
                if (st != HYDRA_OK) break;
                t.ev = take_event(s);
                cudaError_t err = cudaEventRecord(t.ev, s->compute);
                if (err == cudaSuccess && !gens.empty()) {
                    err = cudaStreamWaitEvent(s->copy, t.ev, 0);
                    for (Entry* a : gens)
                        if (err == cudaSuccess)
                            err = cudaMemcpyAsync(s->host_base + a->host, s->dev_base + a->dev, a->nbytes,
                                                  cudaMemcpyDeviceToHost, s->copy);
                    Copy c;
                    c.ev = take_event(s);
                    c.gens = std::move(gens);
                    if (err == cudaSuccess) err = cudaEventRecord(c.ev, s->copy);
                    copying.push_back(std::move(c));
                }
                inflight.push_back(std::move(t));
                if (err != cudaSuccess) {
                    st = cuda_fail(err, "server tick launch");
                    break;
                }
                active.erase(std::remove_if(active.begin(), active.end(),
                                            [&](Entry* a) { return a->next_first >= a->q.nevents; }),
                             active.end());
                ++tick;
                launched = true;
            }
        }
        if (!launched && inflight.empty() && copying.empty() && active.empty() && queue.empty() && more)
            src.idle(now, std::min(2e-4, std::min(run_deadline, s->stop_deadline.load()) - now));
    }
    // the ticks and copies in flight are bounded GPU work: wait for them, then answer every
    // request still open (completed work as done, the rest as timed out on a deadline or
    // refused after an internal error)
    cudaStreamSynchronize(s->compute);
    cudaStreamSynchronize(s->copy);
    const hydra_status drain = harvest_ticks(true);
    const hydra_status drain2 = harvest_copies(true);
    if (st == HYDRA_OK) st = drain != HYDRA_OK ? drain : drain2;
    const int32_t open_status = st == HYDRA_ERR_TIMEOUT ? HYDRA_SERVE_TIMED_OUT : HYDRA_SERVE_REFUSED;
    for (Entry* a : active) release(a);
    for (Entry& e : store)
        if (!e.finished) finish(&e, blank_outcome(open_status));
    if (more) {  // requests that never arrived before the loop ended (replay) or were still queued (live)
        std::deque<Entry> rest;
        std::deque<Entry*> rest_q;
        src.take(kNever, rest, rest_q);
        for (Entry& e : rest) finish(&e, blank_outcome(open_status));
    }
    if (wall_s) *wall_s = clock();
    if (ticks_out) *ticks_out = tick;
    cudaSetDevice(prev_device);
    return st;
}

// Replay of an array sorted by arrival (hydra_server_run).
struct ReplaySource : Source {
    const hydra_serve_request* reqs;
    int nreq, next = 0;
    double scale;
    hydra_serve_outcome* outcomes;
    Clock::time_point t0;
    bool take(double now, std::deque<Entry>& store, std::deque<Entry*>& arrived) override {
        while (next < nreq && reqs[next].arrival * scale <= now) {
            store.emplace_back();
            Entry& e = store.back();
            e.q = reqs[next];
            e.id = next;
            e.arrival = reqs[next].arrival * scale;
            e.withdraw_at = reqs[next].withdraw >= 0.0 ? reqs[next].withdraw : kNever;
            arrived.push_back(&e);
            ++next;
        }
        return next < nreq;
    }
    void idle(double now, double max_wait) override {
        // sleep only when the next arrival is more than 0.2 ms away (closer ones are waited for
        // by the loop itself, for arrival-time precision)
        if (next < nreq && reqs[next].arrival * scale - now > 2e-4 && max_wait > 1e-4)
            std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    void finished(Entry* e, const hydra_serve_outcome& o) override { outcomes[e->id] = o; }
};

// Requests submitted while the worker thread runs the loop.
struct LiveSource : Source {
    hydra_server* s;
    int count = 0;
    bool take(double now, std::deque<Entry>& store, std::deque<Entry*>& arrived) override {
        std::lock_guard<std::mutex> lk(s->mu);
        while (!s->inbox.empty()) {
            const hydra_server::Submitted& sub = s->inbox.front();
            store.emplace_back();
            Entry& e = store.back();
            e.q = sub.q;
            e.id = count++;
            e.ticket = sub.ticket;
            e.arrival = sub.at;
            e.withdraw_at = sub.q.withdraw >= 0.0 ? sub.at + sub.q.withdraw : kNever;
            arrived.push_back(&e);
            s->inbox.pop_front();
        }
        return !s->stopping;
    }
    void idle(double, double max_wait) override {
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->inbox.empty() && !s->stopping && max_wait > 0.0)
            s->cv.wait_for(lk, std::chrono::duration<double>(max_wait));
    }
    void finished(Entry* e, const hydra_serve_outcome& o) override {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->results[e->ticket] = o;
        }
        s->cv.notify_all();
    }
};

}  // namespace

extern "C" {

hydra_status hydra_server_create(uint64_t budget_bytes, void* pinned, uint64_t pinned_bytes, int max_slices,
                                 int int_slice_segments, uint64_t max_tick_events, int keep_outputs,
                                 hydra_server** out) {
    if (!out) return fail(HYDRA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!pinned || pinned_bytes < 256 || budget_bytes < (uint64_t{1} << 24) || max_slices < 1 ||
        int_slice_segments < 1 || max_tick_events < 1)
        return fail(HYDRA_ERR_INVALID_ARG, "bad server arguments");
    hydra_server* s = new hydra_server();
    cudaGetDevice(&s->device);
    s->budget = budget_bytes;
    s->max_slices = max_slices;
    s->int_slice = static_cast<uint64_t>(int_slice_segments) * kSegmentEvents;
    s->max_tick_events = max_tick_events;
    s->keep_outputs = keep_outputs;
    s->seg_ring.size = std::min<uint64_t>(uint64_t{256} << 20, budget_bytes / 16) / 256 * 256;
    s->dev_ring.size = (budget_bytes - s->seg_ring.size) / 256 * 256;
    s->host_ring.size = pinned_bytes / 256 * 256;
    s->host_base = static_cast<unsigned char*>(pinned);
    cudaError_t err = cudaMalloc(&s->dev_base, s->dev_ring.size + s->seg_ring.size);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (err != cudaSuccess) {
        const hydra_status st = err == cudaErrorMemoryAllocation ? fail(HYDRA_ERR_OOM, "server rings: %s", cudaGetErrorString(err))
                                                                : cuda_fail(err, "server create");
        cudaGetLastError();
        hydra_server_destroy(s);
        return st;
    }
    for (int r = 0; r < 2; ++r) {
        const hydra_status st = hydra_batch_create(max_slices, static_cast<uint64_t>(max_slices) * int_slice_segments * 1024,
                                                   &s->runners[r]);
        if (st != HYDRA_OK) {
            hydra_server_destroy(s);
            return st;
        }
    }
    *out = s;
    return HYDRA_OK;
}

hydra_status hydra_server_set_deadline(hydra_server* s, double seconds) {
    if (!s || !(seconds >= 0.0)) return fail(HYDRA_ERR_INVALID_ARG, "need a server and a deadline >= 0");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->live) return fail(HYDRA_ERR_BUSY, "the server is serving live requests");
    s->deadline = seconds;
    return HYDRA_OK;
}

hydra_status hydra_server_run(hydra_server* s, const hydra_serve_request* reqs, int nreq, double time_scale,
                              hydra_serve_outcome* outcomes, double* wall_s, uint64_t* ticks_out) {
    const NvtxRange nvtx_range("hydra_server_run");
    if (!s || !outcomes || (nreq > 0 && !reqs) || nreq < 0 || !(time_scale >= 0.0))
        return fail(HYDRA_ERR_INVALID_ARG, "bad run arguments");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->live) return fail(HYDRA_ERR_BUSY, "the server is serving live requests");
    }
    for (int i = 1; i < nreq; ++i)
        if (reqs[i].arrival < reqs[i - 1].arrival) return fail(HYDRA_ERR_INVALID_ARG, "requests must be sorted by arrival");
    for (int i = 0; i < nreq; ++i) outcomes[i] = blank_outcome(HYDRA_SERVE_REFUSED);
    ReplaySource src;
    src.reqs = reqs;
    src.nreq = nreq;
    src.scale = time_scale;
    src.outcomes = outcomes;
    const Clock::time_point t0 = Clock::now();
    return serve_loop(s, src, t0, s->deadline > 0.0 ? s->deadline : kNever, wall_s, ticks_out);
}

hydra_status hydra_server_start(hydra_server* s) {
    if (!s) return fail(HYDRA_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->live) return fail(HYDRA_ERR_BUSY, "the server is already serving live requests");
    s->live = true;
    s->stopping = false;
    s->loop_done = false;
    s->stop_deadline = kNever;
    s->live_status = HYDRA_OK;
    s->live_error.clear();
    s->results.clear();
    s->inbox.clear();
    s->live_t0 = Clock::now();
    s->worker = std::thread([s]() {
        LiveSource src;
        src.s = s;
        // the loop's deadline: the server's run deadline, or the stop deadline once set
        const hydra_status st = serve_loop(s, src, s->live_t0, s->deadline > 0.0 ? s->deadline : kNever, nullptr, nullptr);
        {
            std::lock_guard<std::mutex> lk2(s->mu);
            s->live_status = st;
            if (st != HYDRA_OK) s->live_error = g_last_error;
            s->loop_done = true;
        }
        s->cv.notify_all();
    });
    return HYDRA_OK;
}

hydra_status hydra_server_submit(hydra_server* s, const hydra_serve_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket) return fail(HYDRA_ERR_INVALID_ARG, "NULL argument");
    const hydra_status st = validate(*req);
    if (st != HYDRA_OK) return st;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->live || s->stopping) return fail(HYDRA_ERR_BUSY, "the server is not accepting live requests");
        *ticket = s->next_ticket++;
        const double at = std::chrono::duration<double>(Clock::now() - s->live_t0).count();
        s->inbox.push_back(hydra_server::Submitted{*ticket, *req, at});
    }
    s->cv.notify_all();
    return HYDRA_OK;
}

hydra_status hydra_server_poll(hydra_server* s, uint64_t ticket, double timeout_s, hydra_serve_outcome* outcome) {
    if (!s || !outcome || !(timeout_s >= 0.0)) return fail(HYDRA_ERR_INVALID_ARG, "bad poll arguments");
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket == 0 || ticket >= s->next_ticket) return fail(HYDRA_ERR_INVALID_ARG, "unknown ticket %llu",
                                                             static_cast<unsigned long long>(ticket));
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    for (;;) {
        auto it = s->results.find(ticket);
        if (it != s->results.end()) {
            *outcome = it->second;
            s->results.erase(it);
            return HYDRA_OK;
        }
        if (s->loop_done) {
            if (s->live_status != HYDRA_OK) return fail(s->live_status, "%s", s->live_error.c_str());
            return fail(HYDRA_ERR_INVALID_ARG, "ticket %llu has no outcome (already polled)",
                        static_cast<unsigned long long>(ticket));
        }
        if (s->cv.wait_until(lk, until) == std::cv_status::timeout && s->results.find(ticket) == s->results.end())
            return fail(HYDRA_ERR_TIMEOUT, "ticket %llu not finished within %.3f s", static_cast<unsigned long long>(ticket),
                        timeout_s);
    }
}

hydra_status hydra_server_stop(hydra_server* s, double timeout_s) {
    if (!s || !(timeout_s >= 0.0)) return fail(HYDRA_ERR_INVALID_ARG, "bad stop arguments");
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (!s->live) return fail(HYDRA_ERR_INVALID_ARG, "the server is not serving live requests");
        s->stopping = true;
        s->cv.notify_all();
        // the loop drains what was submitted; past the timeout it stops launching, waits for its
        // ticks in flight and answers the rest as timed out
        const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
        if (!s->cv.wait_until(lk, until, [&] { return s->loop_done; }))
            s->stop_deadline = std::chrono::duration<double>(until - s->live_t0).count();
    }
    if (s->worker.joinable()) s->worker.join();
    std::lock_guard<std::mutex> lk(s->mu);
    s->live = false;
    s->stop_deadline = kNever;
    const hydra_status st = s->live_status;
    if (st != HYDRA_OK) return fail(st, "%s", s->live_error.c_str());
    return HYDRA_OK;
}

hydra_status hydra_server_destroy(hydra_server* s) {
    if (!s) return HYDRA_OK;
    bool live = false;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        live = s->live;
    }
    if (live) hydra_server_stop(s, 0.0);
    if (s->compute) cudaStreamSynchronize(s->compute);
    if (s->copy) cudaStreamSynchronize(s->copy);
    for (hydra_batch*& b : s->runners)
        if (b) hydra_batch_destroy(b);
    for (cudaEvent_t e : s->events) cudaEventDestroy(e);
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->copy) cudaStreamDestroy(s->copy);
    if (s->dev_base) cudaFree(s->dev_base);
    delete s;
    return HYDRA_OK;
}

}  // extern "C"
