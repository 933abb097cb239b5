// phsp_batch.cu -- many uneven phase-space requests in one persistent launch.
//
// A run is a table of request slices (generation or integration, any n, masses and event
// count).  phsp_batch_kernel is persistent: each warp takes the next 2048-event tile of the
// whole table with one atomic (in an order that groups the slices by kind, matrix element and
// N, so that the warps resident on an SM at one time mostly run the same unrolled event code
// instead of several N's bodies competing for the instruction cache: +12% on a mix of N = 2..8
// requests), finds its slice by binary search over the tile prefix sums,
// stages that slice's decay constants in shared memory and runs the same event code as the
// single-request kernels (generation: structure-of-arrays stores; integration: the same
// tile_sums, so a request gives the same bits alone or in any batch).  Integral slices are
// then reduced per 2^21-event segment into caller-owned segment storage (the state that
// persists between the slices of a long request), and slices that end their request are
// folded into a result.  The three kernels of a run are captured once in a CUDA graph.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "hydra_phsp.h"
#include "phsp_device.cuh"
#include "phsp_host.h"
#include "phsp_integral.cuh"

namespace hydra {

constexpr int kBatchBlock = 256;
constexpr int kBatchWarps = kBatchBlock / 32;
constexpr int kBatchEPT = 2;                 // events per thread in the batch kernel (integral tiles, FP64 generation)
constexpr uint64_t kSegEvents = uint64_t(kTileEvents) * kSegTiles;  // 2^21

struct BatchEntry {
    DecayConsts C;
    MEConsts P;
    uint64_t event_offset, first, count, total;
    void* out;
    uint64_t ld;
    void* weights;
    double* seg;
    uint64_t partial_begin;  // integrate: first slot of this slice in the run's tile partials
    int32_t n, kind, me, dtype;
};

struct BatchHeader {
    unsigned long long tile_counter;  // reset to 0 by every run's table copy
    int32_t nreq, nfinal;
    uint64_t ntiles, nsegjobs;
    const BatchEntry* entries;
    const uint64_t* tile_prefix;  // [nreq + 1], over the slices in tile_order
    const uint64_t* seg_prefix;   // [nreq + 1], over the slices in table order
    const int32_t* tile_order;    // [nreq]: table index of the j-th slice in tile order
    const int32_t* final_idx;     // [nfinal]
};

// Largest r in [0, n) with prefix[r] <= x (prefix[0] = 0 <= x).
__device__ __forceinline__ int find_slot(const uint64_t* __restrict__ prefix, int n, uint64_t x) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Events per thread of a generation tile: four for FP32 up to N = 6 (where the single-request
// kernels are bound by HBM writes and 16-byte stores pay), two above and for FP64.
template <int N, typename R>
__host__ __device__ constexpr int gen_tile_ept() {
    return (std::is_same<R, float>::value && N >= 3 && N <= 6) ? 4 : 2;
}

template <int N, typename R>
__device__ __forceinline__ void generate_tile(const DecayConsts& C, const BatchEntry& e, uint64_t lt, int lane) {
    constexpr int kEPT = gen_tile_ept<N, R>();
    using Out = typename Prec<R>::Out;
    Out* out = static_cast<Out*>(e.out);
    Out* w = static_cast<Out*>(e.weights);
    const uint64_t base = lt * kTileEvents;
#pragma unroll 1
    for (int it = 0; it < kTileEvents / (32 * kEPT); ++it) {
        const uint64_t j0 = base + static_cast<uint64_t>(it * 32 + lane) * kEPT;
        if (j0 + kEPT <= e.count) {
            uint64_t ev[kEPT];
#pragma unroll
            for (int q = 0; q < kEPT; ++q) ev[q] = e.event_offset + e.first + j0 + q;
            StoreSink<R, kEPT> sink{out + j0, w + j0, e.ld};
            raubold_lynch_group<N, R, kEPT>(C, ev, sink);
        } else {
            for (uint64_t j = j0; j < e.count && j < j0 + kEPT; ++j) {
                uint64_t ev[1] = {e.event_offset + e.first + j};
                StoreSink<R, 1> sink{out + j, w + j, e.ld};
                raubold_lynch_group<N, R, 1>(C, ev, sink);
            }
        }
    }
}

template <typename R>
__device__ __forceinline__ void generate_tile_n(int n, const DecayConsts& C, const BatchEntry& e, uint64_t lt, int lane) {
    switch (n) {
        case 2: generate_tile<2, R>(C, e, lt, lane); break;
        case 3: generate_tile<3, R>(C, e, lt, lane); break;
        case 4: generate_tile<4, R>(C, e, lt, lane); break;
        case 5: generate_tile<5, R>(C, e, lt, lane); break;
        case 6: generate_tile<6, R>(C, e, lt, lane); break;
        case 7: generate_tile<7, R>(C, e, lt, lane); break;
        case 8: generate_tile<8, R>(C, e, lt, lane); break;
        case 9: generate_tile<9, R>(C, e, lt, lane); break;
        case 10: generate_tile<10, R>(C, e, lt, lane); break;
    }
}

template <typename R>
__device__ __forceinline__ TileSums integrate_tile_n(int n, int me, const DecayConsts& C, const MEConsts& P,
                                                     const BatchEntry& e, uint64_t tile, int lane) {
    if (me == HYDRA_ME_DALITZ_2BW)
        return tile_sums<3, R, HYDRA_ME_DALITZ_2BW, kBatchEPT>(C, P, e.total, e.event_offset, tile, lane);
    switch (n) {
        case 2: return tile_sums<2, R, HYDRA_ME_FLAT, kBatchEPT>(C, P, e.total, e.event_offset, tile, lane);
        case 3: return tile_sums<3, R, HYDRA_ME_FLAT, kBatchEPT>(C, P, e.total, e.event_offset, tile, lane);
        case 4: return tile_sums<4, R, HYDRA_ME_FLAT, kBatchEPT>(C, P, e.total, e.event_offset, tile, lane);
        case 5: return tile_sums<5, R, HYDRA_ME_FLAT, kBatchEPT>(C, P, e.total, e.event_offset, tile, lane);
        case 6: return tile_sums<6, R, HYDRA_ME_FLAT, kBatchEPT>(C, P, e.total, e.event_offset, tile, lane);
        case 7: return tile_sums<7, R, HYDRA_ME_FLAT, kBatchEPT>(C, P, e.total, e.event_offset, tile, lane);
        case 8: return tile_sums<8, R, HYDRA_ME_FLAT, kBatchEPT>(C, P, e.total, e.event_offset, tile, lane);
        case 9: return tile_sums<9, R, HYDRA_ME_FLAT, kBatchEPT>(C, P, e.total, e.event_offset, tile, lane);
        default: return tile_sums<10, R, HYDRA_ME_FLAT, kBatchEPT>(C, P, e.total, e.event_offset, tile, lane);
    }
}

// RG: arithmetic of generation tiles (float, double or df); RI: of integral tiles.
template <typename RG, typename RI>
__global__ void __launch_bounds__(kBatchBlock) phsp_batch_kernel(BatchHeader* __restrict__ hdr,
                                                                 TileSums* __restrict__ partials) {
    if constexpr (std::is_same<RG, df>::value) {
        df_sincos_table_init();
        __syncthreads();
    }
    __shared__ DecayConsts sC[kBatchWarps];
    __shared__ MEConsts sP[kBatchWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nreq = hdr->nreq;
    const uint64_t ntiles = hdr->ntiles;
    const BatchEntry* __restrict__ entries = hdr->entries;
    const uint64_t* __restrict__ prefix = hdr->tile_prefix;
    const int32_t* __restrict__ order = hdr->tile_order;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&hdr->tile_counter, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        const int j = find_slot(prefix, nreq, t);
        const BatchEntry& e = entries[order[j]];
        {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(&e.C);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&sC[warp]);
            for (int i = lane; i < static_cast<int>(sizeof(DecayConsts) / 4); i += 32) dst[i] = src[i];
            const uint32_t* srcp = reinterpret_cast<const uint32_t*>(&e.P);
            uint32_t* dstp = reinterpret_cast<uint32_t*>(&sP[warp]);
            for (int i = lane; i < static_cast<int>(sizeof(MEConsts) / 4); i += 32) dstp[i] = srcp[i];
        }
        __syncwarp();
        const uint64_t lt = t - prefix[j];
        if (e.kind == HYDRA_REQ_GENERATE) {
            generate_tile_n<RG>(e.n, sC[warp], e, lt, lane);
        } else {
            const TileSums ts = integrate_tile_n<RI>(e.n, e.me, sC[warp], sP[warp], e, e.first / kTileEvents + lt, lane);
            if (lane == 0) partials[e.partial_begin + lt] = ts;
        }
        __syncwarp();
    }
}

// One warp per (integral slice, segment): the slice's tile partials -> the request's
// segment storage, with the same segment_sums as the single-request path.
__global__ void __launch_bounds__(kSegBlock) batch_reduce_segments(const BatchHeader* __restrict__ hdr,
                                                                   const TileSums* __restrict__ partials) {
    const uint64_t njobs = hdr->nsegjobs;
    for (uint64_t job = blockIdx.x; job < njobs; job += gridDim.x) {  // one block per segment job
        const int r = find_slot(hdr->seg_prefix, hdr->nreq, job);
        const BatchEntry& e = hdr->entries[r];
        const uint64_t s = job - hdr->seg_prefix[r];
        const uint64_t slice_tiles = (e.count + kTileEvents - 1) / kTileEvents;
        const uint64_t t0 = s * kSegTiles;
        const uint64_t nt = slice_tiles - t0 < kSegTiles ? slice_tiles - t0 : kSegTiles;
        segment_sums_block(partials + e.partial_begin + t0, nt, e.seg + (e.first / kSegEvents + s) * 8);
    }
}

// One warp per slice that ends its request: fold all segments of the request.
__global__ void __launch_bounds__(kBatchBlock) batch_finalize(const BatchHeader* __restrict__ hdr,
                                                              hydra_integral* __restrict__ results) {
    const int lane = threadIdx.x & 31;
    const int gw = static_cast<int>((static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
    const int nw = static_cast<int>((static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5);
    for (int k = gw; k < hdr->nfinal; k += nw) {
        const int r = hdr->final_idx[k];
        const BatchEntry& e = hdr->entries[r];
        const uint64_t nseg = (e.total + kSegEvents - 1) / kSegEvents;
        fold_segments(e.seg, nseg, e.total, lane, results + r);
    }
}

}  // namespace hydra

using namespace hydra;

struct hydra_batch {
    int device = 0;
    int max_requests = 0;
    uint64_t max_tiles = 0;
    size_t table_bytes = 0;
    unsigned char* d_table = nullptr;  // header | entries | tile_prefix | seg_prefix | tile_order | final_idx
    unsigned char* h_table = nullptr;  // pinned staging of the same layout
    TileSums* d_partials = nullptr;
    hydra_integral* d_results = nullptr;
    hydra_integral* h_results = nullptr;
    cudaEvent_t table_done = nullptr;  // the table copy of the latest run has completed
    cudaEvent_t run_done = nullptr;    // the latest run has completed
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};  // per variant (see run_variant)
    int grid_main[3] = {0, 0, 0};
    int grid_aux = 0;
    std::vector<uint8_t> finalized;  // per slice of the latest run
    std::vector<int32_t> kinds;
    int last_nreq = 0;
    std::mutex mu;
};

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

size_t table_size(int nreq, int nfinal) {
    size_t off = align_up(sizeof(BatchHeader), 256);
    off += static_cast<size_t>(nreq) * sizeof(BatchEntry);
    off = align_up(off, 8) + (static_cast<size_t>(nreq) + 1) * 8;  // tile prefix
    off += (static_cast<size_t>(nreq) + 1) * 8;                     // seg prefix
    off += static_cast<size_t>(nreq) * 4;                           // tile order
    off += static_cast<size_t>(nfinal) * 4;
    return align_up(off, 256);
}

// Variant 0: FP32; 1: FP64 with native FP64 arithmetic; 2: FP64 with double-float generation and integrals.
int run_variant(int dtype) {
    if (dtype == HYDRA_F32) return 0;
    return g_fp64_arith.load(std::memory_order_relaxed) == HYDRA_FP64_NATIVE ? 1 : 2;
}

void launch_run_kernels(hydra_batch* b, int v, cudaStream_t s) {
    BatchHeader* hdr = reinterpret_cast<BatchHeader*>(b->d_table);
    if (v == 0)
        phsp_batch_kernel<float, float><<<b->grid_main[v], kBatchBlock, 0, s>>>(hdr, b->d_partials);
    else if (v == 1)
        phsp_batch_kernel<double, double><<<b->grid_main[v], kBatchBlock, 0, s>>>(hdr, b->d_partials);
    else
        phsp_batch_kernel<df, df><<<b->grid_main[v], kBatchBlock, 0, s>>>(hdr, b->d_partials);
    batch_reduce_segments<<<b->grid_aux, kSegBlock, 0, s>>>(hdr, b->d_partials);
    batch_finalize<<<b->grid_aux, kBatchBlock, 0, s>>>(hdr, b->d_results);
}

hydra_status capture_graph(hydra_batch* b, int v) {
    cudaStream_t cs;
    cudaError_t err = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (err != cudaSuccess) return cuda_fail(err, "capture stream");
    cudaGraph_t g = nullptr;
    err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
        launch_run_kernels(b, v, cs);
        err = cudaStreamEndCapture(cs, &g);
    }
    if (err == cudaSuccess) err = cudaGraphInstantiate(&b->graph[v], g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (err != cudaSuccess) return cuda_fail(err, "batch graph capture");
    return HYDRA_OK;
}

}  // namespace

extern "C" {

hydra_status hydra_batch_create(int max_requests, uint64_t max_integrate_tiles, hydra_batch** out) {
    if (!out) return fail(HYDRA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_requests < 1 || max_requests > (1 << 20))
        return fail(HYDRA_ERR_INVALID_ARG, "max_requests = %d outside [1, 2^20]", max_requests);
    hydra_batch* b = new hydra_batch();
    b->max_requests = max_requests;
    b->max_tiles = max_integrate_tiles ? max_integrate_tiles : 1;
    b->table_bytes = table_size(max_requests, max_requests);
    cudaError_t err = cudaGetDevice(&b->device);
    if (err == cudaSuccess) err = cudaMalloc(&b->d_table, b->table_bytes);
    if (err == cudaSuccess) err = cudaMallocHost(&b->h_table, b->table_bytes);
    if (err == cudaSuccess) err = cudaMalloc(&b->d_partials, b->max_tiles * sizeof(TileSums));
    if (err == cudaSuccess) err = cudaMalloc(&b->d_results, static_cast<size_t>(max_requests) * sizeof(hydra_integral));
    if (err == cudaSuccess) err = cudaMallocHost(&b->h_results, static_cast<size_t>(max_requests) * sizeof(hydra_integral));
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->table_done, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->run_done, cudaEventDisableTiming);
    if (err != cudaSuccess) {
        const hydra_status st = err == cudaErrorMemoryAllocation ? fail(HYDRA_ERR_OOM, "batch buffers: %s", cudaGetErrorString(err))
                                                                : cuda_fail(err, "batch create");
        cudaGetLastError();
        hydra_batch_destroy(b);
        return st;
    }
    int sms = 148, occ = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, phsp_batch_kernel<float, float>, kBatchBlock, 0);
    b->grid_main[0] = sms * (occ > 0 ? occ : 1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, phsp_batch_kernel<double, double>, kBatchBlock, 0);
    b->grid_main[1] = sms * (occ > 0 ? occ : 1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, phsp_batch_kernel<df, df>, kBatchBlock, 0);
    b->grid_main[2] = sms * (occ > 0 ? occ : 1);
    b->grid_aux = sms;
    for (int v = 0; v < 3; ++v) {
        const hydra_status st = capture_graph(b, v);
        if (st != HYDRA_OK) {
            hydra_batch_destroy(b);
            return st;
        }
    }
    *out = b;
    return HYDRA_OK;
}

hydra_status hydra_batch_run(hydra_batch* b, const hydra_request* reqs, int nreq, int use_graph,
                             hydra_stream_t stream) {
    if (!b) return fail(HYDRA_ERR_INVALID_ARG, "batch is NULL");
    if (nreq < 1 || nreq > b->max_requests)
        return fail(HYDRA_ERR_INVALID_ARG, "nreq = %d outside [1, %d]", nreq, b->max_requests);
    if (!reqs) return fail(HYDRA_ERR_INVALID_ARG, "reqs is NULL");
    std::lock_guard<std::mutex> lk(b->mu);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != b->device) return fail(HYDRA_ERR_INVALID_ARG, "batch belongs to device %d, current is %d", b->device, dev);
    const int dt = reqs[0].dtype;
    if (dt != HYDRA_F32 && dt != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "request 0: unknown dtype %d", dt);
    // the previous run's table copy must be done before the staging memory is rewritten
    cudaError_t err = cudaEventSynchronize(b->table_done);
    if (err != cudaSuccess) return cuda_fail(err, "batch staging wait");

    unsigned char* h = b->h_table;
    const size_t entries_off = align_up(sizeof(BatchHeader), 256);
    BatchEntry* E = reinterpret_cast<BatchEntry*>(h + entries_off);
    const size_t tp_off = align_up(entries_off + static_cast<size_t>(nreq) * sizeof(BatchEntry), 8);
    const size_t sp_off = tp_off + (static_cast<size_t>(nreq) + 1) * 8;
    const size_t to_off = sp_off + (static_cast<size_t>(nreq) + 1) * 8;
    const size_t fi_off = to_off + static_cast<size_t>(nreq) * 4;
    uint64_t* tp = reinterpret_cast<uint64_t*>(h + tp_off);
    uint64_t* sp = reinterpret_cast<uint64_t*>(h + sp_off);
    int32_t* to = reinterpret_cast<int32_t*>(h + to_off);
    int32_t* fi = reinterpret_cast<int32_t*>(h + fi_off);
    b->finalized.assign(nreq, 0);
    b->kinds.assign(nreq, 0);
    uint64_t tiles = 0, segs = 0, ptiles = 0;
    int nfinal = 0;
    for (int i = 0; i < nreq; ++i) {
        const hydra_request& r = reqs[i];
        BatchEntry& e = E[i];
        std::memset(&e, 0, sizeof e);
        hydra_status st = make_consts(r.M, r.n, r.masses, r.seed, &e.C);
        if (st != HYDRA_OK) return fail(st, "request %d: %s", i, g_last_error.c_str());
        if (r.dtype != dt) return fail(HYDRA_ERR_INVALID_ARG, "request %d: dtype %d differs from request 0 (%d)", i, r.dtype, dt);
        if (r.count == 0) return fail(HYDRA_ERR_INVALID_ARG, "request %d: empty slice", i);
        if (r.event_offset + r.first + r.count < r.event_offset)
            return fail(HYDRA_ERR_INVALID_ARG, "request %d: counter-event index overflows 64 bits", i);
        e.event_offset = r.event_offset;
        e.first = r.first;
        e.count = r.count;
        e.n = r.n;
        e.kind = r.kind;
        e.dtype = r.dtype;
        const uint64_t slice_tiles = (r.count + kTileEvents - 1) / kTileEvents;
        sp[i] = segs;
        b->kinds[i] = r.kind;
        if (r.kind == HYDRA_REQ_GENERATE) {
            if (!r.out || !r.weights) return fail(HYDRA_ERR_INVALID_ARG, "request %d: NULL output", i);
            if ((reinterpret_cast<uintptr_t>(r.out) & 15u) || (reinterpret_cast<uintptr_t>(r.weights) & 15u))
                return fail(HYDRA_ERR_MISALIGNED, "request %d: outputs must be 16-byte aligned", i);
            if (r.ld < r.count || r.ld % 4 != 0)
                return fail(HYDRA_ERR_MISALIGNED, "request %d: ld = %llu must be >= count and a multiple of 4", i,
                            static_cast<unsigned long long>(r.ld));
            e.out = r.out;
            e.ld = r.ld;
            e.weights = r.weights;
        } else if (r.kind == HYDRA_REQ_INTEGRATE) {
            st = make_me(static_cast<hydra_me_id>(r.me), r.n, r.params, 6, &e.P);
            if (st != HYDRA_OK) return fail(st, "request %d: %s", i, g_last_error.c_str());
            if (!r.seg_partials) return fail(HYDRA_ERR_INVALID_ARG, "request %d: NULL seg_partials", i);
            if (r.first % kSegEvents != 0)
                return fail(HYDRA_ERR_INVALID_ARG, "request %d: integral slice must start on a multiple of 2^21 events", i);
            if (r.first + r.count > r.total || r.total == 0)
                return fail(HYDRA_ERR_INVALID_ARG, "request %d: slice beyond the request's total", i);
            const bool ends = r.first + r.count == r.total;
            if (!ends && r.count % kSegEvents != 0)
                return fail(HYDRA_ERR_INVALID_ARG, "request %d: an integral slice that does not end its request must hold a multiple of 2^21 events", i);
            e.me = r.me;
            e.total = r.total;
            e.seg = r.seg_partials;
            e.partial_begin = ptiles;
            ptiles += slice_tiles;
            segs += (slice_tiles + kSegTiles - 1) / kSegTiles;
            if (ends) {
                fi[nfinal++] = i;
                b->finalized[i] = 1;
            }
        } else {
            return fail(HYDRA_ERR_INVALID_ARG, "request %d: unknown kind %d", i, r.kind);
        }
        tiles += slice_tiles;
    }
    sp[nreq] = segs;
    // tile order: a stable counting sort of the slices by (kind, matrix element, N)
    {
        constexpr int kKeys = 4 * 16;
        auto key = [&](int i) {
            const hydra_request& r = reqs[i];
            const int group = r.kind == HYDRA_REQ_GENERATE ? 0 : 1 + (r.me == HYDRA_ME_DALITZ_2BW ? 1 : 0);
            return group * 16 + r.n;
        };
        int start[kKeys + 1] = {0};
        for (int i = 0; i < nreq; ++i) ++start[key(i) + 1];
        for (int k = 0; k < kKeys; ++k) start[k + 1] += start[k];
        for (int i = 0; i < nreq; ++i) to[start[key(i)]++] = i;
        uint64_t acc = 0;
        for (int j = 0; j < nreq; ++j) {
            tp[j] = acc;
            acc += (reqs[to[j]].count + kTileEvents - 1) / kTileEvents;
        }
        tp[nreq] = acc;  // == tiles
    }
    if (ptiles > b->max_tiles)
        return fail(HYDRA_ERR_INVALID_ARG, "integral slices need %llu tiles; the batch holds %llu",
                    static_cast<unsigned long long>(ptiles), static_cast<unsigned long long>(b->max_tiles));
    BatchHeader* H = reinterpret_cast<BatchHeader*>(h);
    H->tile_counter = 0;
    H->nreq = nreq;
    H->nfinal = nfinal;
    H->ntiles = tiles;
    H->nsegjobs = segs;
    H->entries = reinterpret_cast<const BatchEntry*>(b->d_table + entries_off);
    H->tile_prefix = reinterpret_cast<const uint64_t*>(b->d_table + tp_off);
    H->seg_prefix = reinterpret_cast<const uint64_t*>(b->d_table + sp_off);
    H->tile_order = reinterpret_cast<const int32_t*>(b->d_table + to_off);
    H->final_idx = reinterpret_cast<const int32_t*>(b->d_table + fi_off);
    const size_t bytes = fi_off + static_cast<size_t>(nfinal) * 4;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    err = cudaMemcpyAsync(b->d_table, b->h_table, bytes, cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = cudaEventRecord(b->table_done, s);
    if (err != cudaSuccess) return cuda_fail(err, "batch table copy");
    const int v = run_variant(dt);
    if (use_graph) {
        err = cudaGraphLaunch(b->graph[v], s);
    } else {
        launch_run_kernels(b, v, s);
        err = cudaGetLastError();
    }
    if (err != cudaSuccess) return cuda_fail(err, "batch launch");
    if (nfinal > 0) {
        err = cudaMemcpyAsync(b->h_results, b->d_results, static_cast<size_t>(nreq) * sizeof(hydra_integral),
                              cudaMemcpyDeviceToHost, s);
        if (err != cudaSuccess) return cuda_fail(err, "batch result copy");
    }
    err = cudaEventRecord(b->run_done, s);
    if (err != cudaSuccess) return cuda_fail(err, "batch event");
    b->last_nreq = nreq;
    return HYDRA_OK;
}

hydra_status hydra_batch_result(hydra_batch* b, int i, hydra_integral* result) {
    if (!b || !result) return fail(HYDRA_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(b->mu);
    if (i < 0 || i >= b->last_nreq) return fail(HYDRA_ERR_INVALID_ARG, "slice %d outside the latest run", i);
    if (b->kinds[i] != HYDRA_REQ_INTEGRATE || !b->finalized[i])
        return fail(HYDRA_ERR_INVALID_ARG, "slice %d is not an integral slice that ends its request", i);
    const cudaError_t err = cudaEventSynchronize(b->run_done);
    if (err != cudaSuccess) return cuda_fail(err, "batch wait");
    *result = b->h_results[i];
    return HYDRA_OK;
}

hydra_status hydra_batch_destroy(hydra_batch* b) {
    if (!b) return HYDRA_OK;
    if (b->run_done) cudaEventSynchronize(b->run_done);
    for (int v = 0; v < 3; ++v)
        if (b->graph[v]) cudaGraphExecDestroy(b->graph[v]);
    if (b->d_table) cudaFree(b->d_table);
    if (b->h_table) cudaFreeHost(b->h_table);
    if (b->d_partials) cudaFree(b->d_partials);
    if (b->d_results) cudaFree(b->d_results);
    if (b->h_results) cudaFreeHost(b->h_results);
    if (b->table_done) cudaEventDestroy(b->table_done);
    if (b->run_done) cudaEventDestroy(b->run_done);
    delete b;
    return HYDRA_OK;
}

}  // extern "C"
