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
// is refused.  Every slice computes exactly the events of the single-request entry points.
//
// Every ring block is checked against its ring before a record is built from it, so a
// bookkeeping error ends the run with an error status instead of a kernel touching memory
// outside the rings.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <deque>
#include <thread>
#include <utility>
#include <vector>

#include "hydra_phsp.h"
#include "phsp_host.h"

namespace {

constexpr uint64_t kSegmentEvents = uint64_t{1} << 21;

// Byte ring handed out in arrival order as 256-byte-aligned blocks; blocks may be released in
// any order and a block is only handed out where it overlaps no live one.
struct Ring {
    uint64_t size = 0, head = 0;
    std::deque<std::pair<uint64_t, uint64_t>> live;
    bool alloc(uint64_t nbytes, uint64_t* start) {
        nbytes = (nbytes + 255) / 256 * 256;
        if (nbytes > size) return false;
        const uint64_t s = head + nbytes <= size ? head : 0;
        const uint64_t e = s + nbytes;
        for (const auto& b : live)
            if (b.first < e && s < b.second) return false;
        head = e;
        live.emplace_back(s, e);
        *start = s;
        return true;
    }
    void release(uint64_t start) {
        for (auto it = live.begin(); it != live.end(); ++it)
            if (it->first == start) {
                live.erase(it);
                return;
            }
    }
};

struct Active {
    int rid = 0;
    double arrival = 0.0;  // seconds on the loop's clock
    uint64_t next_first = 0, nbytes = 0, ld = 0, dev = 0, host = 0;
    hydra_request rec{};
};

struct Tick {
    cudaEvent_t ev;
    int runner;
    std::vector<std::pair<int, Active*>> slots;
    std::vector<Active*> integrals;  // integral requests whose last slice this tick runs
};

struct Copy {
    cudaEvent_t ev;
    std::vector<Active*> gens;
};

}  // namespace

struct hydra_server {
    int device = 0;
    uint64_t budget = 0;
    int max_slices = 0;
    uint64_t int_slice = 0, max_tick_events = 0;
    int keep_outputs = 0;
    unsigned char* dev_base = nullptr;  // staging ring then segment ring
    Ring dev_ring, seg_ring, host_ring;
    unsigned char* host_base = nullptr;  // the caller's pinned ring
    hydra_batch* runners[2] = {nullptr, nullptr};
    cudaStream_t compute = nullptr, copy = nullptr;
    std::vector<cudaEvent_t> events;  // free events
};

using namespace hydra;

static cudaEvent_t take_event(hydra_server* s) {
    if (!s->events.empty()) {
        cudaEvent_t e = s->events.back();
        s->events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

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

hydra_status hydra_server_destroy(hydra_server* s) {
    if (!s) return HYDRA_OK;
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

hydra_status hydra_server_run(hydra_server* s, const hydra_serve_request* reqs, int nreq, double time_scale,
                              hydra_serve_outcome* outcomes, double* wall_s, uint64_t* ticks_out) {
    if (!s || !outcomes || (nreq > 0 && !reqs) || nreq < 0 || !(time_scale >= 0.0))
        return fail(HYDRA_ERR_INVALID_ARG, "bad run arguments");
    for (int i = 1; i < nreq; ++i)
        if (reqs[i].arrival < reqs[i - 1].arrival) return fail(HYDRA_ERR_INVALID_ARG, "requests must be sorted by arrival");
    for (int i = 0; i < nreq; ++i) {
        const hydra_serve_request& q = reqs[i];
        if (q.n < 2 || q.n > 10) return fail(HYDRA_ERR_UNSUPPORTED_N, "request %d: n = %d", i, q.n);
        if ((q.kind != HYDRA_REQ_GENERATE && q.kind != HYDRA_REQ_INTEGRATE) || q.nevents == 0)
            return fail(HYDRA_ERR_INVALID_ARG, "request %d: kind %d, %llu events", i, q.kind,
                        static_cast<unsigned long long>(q.nevents));
        outcomes[i] = hydra_serve_outcome{};
        outcomes[i].latency = -1.0;
        outcomes[i].host_offset = ~uint64_t{0};
        outcomes[i].status = HYDRA_SERVE_REFUSED;  // until it completes or is withdrawn
    }
    bool any_withdraw = false;
    for (int i = 0; i < nreq; ++i) any_withdraw = any_withdraw || reqs[i].withdraw >= 0.0;
    unsigned char* seg_base = s->dev_base + s->dev_ring.size;
    std::vector<Active> pool(static_cast<size_t>(nreq));
    std::deque<Active*> queue;
    std::vector<Active*> active;
    std::deque<Tick> inflight;
    std::deque<Copy> copying;
    std::vector<hydra_request> table;
    table.reserve(static_cast<size_t>(s->max_slices));
    uint64_t tick = 0;
    int next = 0;
    const auto t0 = std::chrono::steady_clock::now();
    auto clock = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
    hydra_status st = HYDRA_OK;

    auto release = [&](Active* a) {
        if (a->rec.kind == HYDRA_REQ_GENERATE) {
            s->dev_ring.release(a->dev);
            s->host_ring.release(a->host);
        } else {
            s->seg_ring.release(a->dev);
        }
    };
    auto complete = [&](Active* a, double tnow) {
        outcomes[a->rid].latency = tnow - a->arrival;
        outcomes[a->rid].status = HYDRA_SERVE_DONE;
        if (a->rec.kind == HYDRA_REQ_GENERATE) {
            s->dev_ring.release(a->dev);
            if (s->keep_outputs) {
                outcomes[a->rid].host_offset = a->host;
                outcomes[a->rid].ld = a->ld;
            } else {
                s->host_ring.release(a->host);
            }
        } else {
            s->seg_ring.release(a->dev);
        }
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
    auto admit = [&](Active* a) -> int {
        const hydra_serve_request& q = reqs[a->rid];
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

    while (st == HYDRA_OK && (next < nreq || !queue.empty() || !active.empty() || !inflight.empty() || !copying.empty())) {
        const double now = clock();
        while (next < nreq && reqs[next].arrival * time_scale <= now) {
            Active& a = pool[static_cast<size_t>(next)];
            a.rid = next;
            a.arrival = reqs[next].arrival * time_scale;
            queue.push_back(&a);
            ++next;
        }
        while (!queue.empty() && static_cast<int>(active.size()) < s->max_slices) {
            Active* a = queue.front();
            if (!fits_ever(reqs[a->rid])) {  // larger than the rings: refused, not queued forever
                queue.pop_front();
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
                    continue;
                }
                break;
            }
            active.push_back(a);
            queue.pop_front();
        }
        if (st != HYDRA_OK) break;
        // finished ticks, oldest first: integrals complete with their last slice
        while (!inflight.empty() && (inflight.size() >= 2 || cudaEventQuery(inflight.front().ev) == cudaSuccess)) {
            Tick t = std::move(inflight.front());
            inflight.pop_front();
            cudaError_t err = cudaEventSynchronize(t.ev);
            if (err != cudaSuccess) {
                st = cuda_fail(err, "server tick");
                break;
            }
            const double tnow = clock();
            for (const auto& sl : t.slots)
                if (std::find(t.integrals.begin(), t.integrals.end(), sl.second) != t.integrals.end()) {
                    st = hydra_batch_result(s->runners[t.runner], sl.first, &outcomes[sl.second->rid].result);
                    if (st != HYDRA_OK) break;
                }
            for (Active* a : t.integrals) complete(a, tnow);
            s->events.push_back(t.ev);
        }
        if (st != HYDRA_OK) break;
        // client withdrawal between ticks: an admitted request not yet fully launched is dropped
        // and its memory released (slices already in flight finish on the compute stream before
        // any later use of the released blocks)
        if (any_withdraw) {
            active.erase(std::remove_if(active.begin(), active.end(), [&](Active* a) {
                             const hydra_serve_request& q = reqs[a->rid];
                             if (q.withdraw < 0.0 || now < q.withdraw || a->next_first >= q.nevents) return false;
                             outcomes[a->rid].status = HYDRA_SERVE_WITHDRAWN;
                             release(a);
                             return true;
                         }),
                         active.end());
        }
        // generate requests complete when their copy to host memory has landed
        while (!copying.empty() && cudaEventQuery(copying.front().ev) == cudaSuccess) {
            Copy c = std::move(copying.front());
            copying.pop_front();
            const double tnow = clock();
            for (Active* a : c.gens) complete(a, tnow);
            s->events.push_back(c.ev);
        }
        bool launched = false;
        if (inflight.size() < 2) {
            table.clear();
            Tick t;
            t.runner = static_cast<int>(tick % 2);
            std::vector<Active*> gens;
            uint64_t room = s->max_tick_events;
            for (Active* a : active) {
                const hydra_serve_request& q = reqs[a->rid];
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
                st = hydra_batch_run(s->runners[t.runner], table.data(), static_cast<int>(table.size()), 1,
                                     reinterpret_cast<hydra_stream_t>(s->compute));
                if (st != HYDRA_OK) break;
                t.ev = take_event(s);
                cudaError_t err = cudaEventRecord(t.ev, s->compute);
                if (err == cudaSuccess && !gens.empty()) {
                    err = cudaStreamWaitEvent(s->copy, t.ev, 0);
                    for (Active* a : gens)
                        if (err == cudaSuccess)
                            err = cudaMemcpyAsync(s->host_base + a->host, s->dev_base + a->dev, a->nbytes,
                                                  cudaMemcpyDeviceToHost, s->copy);
                    Copy c;
                    c.ev = take_event(s);
                    c.gens = std::move(gens);
                    if (err == cudaSuccess) err = cudaEventRecord(c.ev, s->copy);
                    copying.push_back(std::move(c));
                }
                if (err != cudaSuccess) {
                    st = cuda_fail(err, "server tick launch");
                    break;
                }
                inflight.push_back(std::move(t));
                active.erase(std::remove_if(active.begin(), active.end(),
                                            [&](Active* a) { return a->next_first >= reqs[a->rid].nevents; }),
                             active.end());
                ++tick;
                launched = true;
            }
        }
        if (!launched && inflight.empty() && copying.empty() && active.empty() && queue.empty() && next < nreq) {
            const double wait = reqs[next].arrival * time_scale - clock();
            if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::microseconds(100));
        }
    }
    cudaStreamSynchronize(s->compute);
    cudaStreamSynchronize(s->copy);
    for (Tick& t : inflight) s->events.push_back(t.ev);
    for (Copy& c : copying) s->events.push_back(c.ev);
    if (wall_s) *wall_s = clock();
    if (ticks_out) *ticks_out = tick;
    return st;
}

}  // extern "C"
