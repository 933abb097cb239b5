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

#include "phsp_batch.cuh"

namespace hydra {

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
    int block_f32 = kBatchBlock;  // threads per block of FP32 runs (the process-wide shape at creation)
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

// Launch shape of the persistent kernel, process-wide (hydra_set_batch_shape): threads per block
// of FP32 runs (read when a runner is created) and events per thread of generation tiles by n
// (read by every run).  Defaults: 256 threads; FP32 four events per thread for n = 3..6 (where
// generation is bound by HBM writes and 16-byte stores pay) and two otherwise; FP64 two.
std::mutex g_shape_mu;
int g_batch_block_f32 = kBatchBlock;
int32_t g_batch_ept[2][kNMax + 1] = {{2, 2, 2, 4, 4, 4, 4, 2, 2, 2, 2}, {2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2}};

// Variant 0: FP32; 1: FP64 with native FP64 arithmetic; 2: FP64 with double-float generation and integrals.
int run_variant(int dtype) {
    if (dtype == HYDRA_F32) return 0;
    return g_fp64_arith.load(std::memory_order_relaxed) == HYDRA_FP64_NATIVE ? 1 : 2;
}

void launch_run_kernels(hydra_batch* b, int v, cudaStream_t s) {
    BatchHeader* hdr = reinterpret_cast<BatchHeader*>(b->d_table);
    if (v == 0) {
        launch_batch_kernel_f32(b->block_f32, b->grid_main[v], hdr, b->d_partials, s);
    } else if (v == 1) {
        phsp_batch_kernel<double, double, kBatchBlock><<<b->grid_main[v], kBatchBlock, 0, s>>>(hdr, b->d_partials);
    } else {
        phsp_batch_kernel<df, df, kBatchBlock><<<b->grid_main[v], kBatchBlock, 0, s>>>(hdr, b->d_partials);
    }
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
    {
        std::lock_guard<std::mutex> lk(g_shape_mu);
        b->block_f32 = g_batch_block_f32;
    }
    int sms = 148, occ = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel_f32(b->block_f32), b->block_f32, 0);
    b->grid_main[0] = sms * (occ > 0 ? occ : 1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, phsp_batch_kernel<double, double, kBatchBlock>, kBatchBlock, 0);
    b->grid_main[1] = sms * (occ > 0 ? occ : 1);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, phsp_batch_kernel<df, df, kBatchBlock>, kBatchBlock, 0);
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
    const NvtxRange nvtx_range("hydra_batch_run");
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
    {
        std::lock_guard<std::mutex> lk(g_shape_mu);
        std::memcpy(H->gen_ept, g_batch_ept[dt == HYDRA_F32 ? 0 : 1], sizeof H->gen_ept);
    }
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

hydra_status hydra_set_batch_shape(hydra_dtype dtype, int block, const int32_t* ept_by_n) {
    if (dtype != HYDRA_F32 && dtype != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(dtype));
    if (!ept_by_n) return fail(HYDRA_ERR_INVALID_ARG, "ept_by_n is NULL");
    if (dtype == HYDRA_F32 ? (block != 128 && block != 256 && block != 512) : block != kBatchBlock)
        return fail(HYDRA_ERR_INVALID_ARG, "block = %d: FP32 runs take 128, 256 or 512 threads, FP64 runs 256", block);
    for (int n = 2; n <= kNMax; ++n) {
        const int e = ept_by_n[n];
        const bool ok = dtype == HYDRA_F32 ? (e == 1 || e == 2 || (e == 4 && n <= 6)) : e == 2;
        if (!ok)
            return fail(HYDRA_ERR_INVALID_ARG, "events per thread %d for n = %d: FP32 takes 1, 2 (or 4 for n <= 6), "
                        "FP64 2", e, n);
    }
    std::lock_guard<std::mutex> lk(g_shape_mu);
    if (dtype == HYDRA_F32) g_batch_block_f32 = block;
    for (int n = 2; n <= kNMax; ++n) g_batch_ept[dtype == HYDRA_F32 ? 0 : 1][n] = ept_by_n[n];
    return HYDRA_OK;
}

hydra_status hydra_get_batch_shape(hydra_dtype dtype, int* block, int32_t* ept_by_n) {
    if (dtype != HYDRA_F32 && dtype != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(dtype));
    if (!block || !ept_by_n) return fail(HYDRA_ERR_INVALID_ARG, "NULL output");
    std::lock_guard<std::mutex> lk(g_shape_mu);
    *block = dtype == HYDRA_F32 ? g_batch_block_f32 : kBatchBlock;
    std::memcpy(ept_by_n, g_batch_ept[dtype == HYDRA_F32 ? 0 : 1], sizeof(int32_t) * (kNMax + 1));
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

// ------------------------------------------------------------------------------------
// Whole requests under a device-memory budget (hydra_phsp_batch_run): the requests are cut
// into waves whose generated outputs fit an arena inside the budget, each wave is one run of
// a batch runner (one graph launch), and outputs bound for the host are copied out of the
// arena on a copy stream while the next wave computes into the other half of the arena.
// ------------------------------------------------------------------------------------
namespace {

constexpr uint64_t kRunIntSlice = uint64_t(1) << 26;   // events per integral slice (32768 tiles)
constexpr uint64_t kRunIntSlicesPerWave = 16;          // integral slices per wave (16 MiB of tile partials)
constexpr int kRunMaxSlices = 8192;                    // slices per wave

thread_local uint64_t t_last_waves = 0, t_last_slices = 0;

struct Slice {
    int req;
    uint64_t first, count;
    uint64_t arena_off, ld;  // generate slices in the arena (NONE / HOST destinations)
};

size_t elem_of(int dtype) { return dtype == HYDRA_F32 ? sizeof(float) : sizeof(double); }

hydra_status validate_request(hydra_batch_request& r, int i, int dt) {
    DecayConsts C;
    hydra_status st = make_consts(r.M, r.n, r.masses, r.seed, &C);
    if (st == HYDRA_OK && r.dtype != dt)
        st = fail(HYDRA_ERR_INVALID_ARG, "dtype %d differs from request 0 (%d)", r.dtype, dt);
    if (st == HYDRA_OK && r.nevents == 0) st = fail(HYDRA_ERR_INVALID_ARG, "nevents must be > 0");
    if (st == HYDRA_OK && r.event_offset + r.nevents < r.event_offset)
        st = fail(HYDRA_ERR_INVALID_ARG, "event_offset + nevents overflows 64 bits");
    if (st == HYDRA_OK && r.kind == HYDRA_REQ_GENERATE) {
        if (r.dest != HYDRA_DEST_NONE && r.dest != HYDRA_DEST_HOST && r.dest != HYDRA_DEST_DEVICE)
            st = fail(HYDRA_ERR_INVALID_ARG, "unknown destination %d", r.dest);
        else if (r.dest != HYDRA_DEST_NONE && (!r.out || !r.weights))
            st = fail(HYDRA_ERR_INVALID_ARG, "NULL output");
        else if (r.dest != HYDRA_DEST_NONE && r.ld < r.nevents)
            st = fail(HYDRA_ERR_INVALID_ARG, "ld = %llu < nevents", static_cast<unsigned long long>(r.ld));
        else if (r.dest == HYDRA_DEST_DEVICE &&
                 ((reinterpret_cast<uintptr_t>(r.out) & 15u) || (reinterpret_cast<uintptr_t>(r.weights) & 15u) || r.ld % 4))
            st = fail(HYDRA_ERR_MISALIGNED, "device outputs must be 16-byte aligned with ld a multiple of 4");
    } else if (st == HYDRA_OK && r.kind == HYDRA_REQ_INTEGRATE) {
        MEConsts P;
        st = make_me(static_cast<hydra_me_id>(r.me), r.n, r.params, 6, &P);
    } else if (st == HYDRA_OK) {
        st = fail(HYDRA_ERR_INVALID_ARG, "unknown kind %d", r.kind);
    }
    r.status = st;
    if (st != HYDRA_OK) return fail(st, "request %d: %s", i, g_last_error.c_str());
    return HYDRA_OK;
}

// What hydra_phsp_batch_run keeps on a device between calls (released by hydra_shutdown): the
// arena, the integral segment storage, the batch runner and the copy stream with its events.
// A call reuses them when they are large enough (and the runner's FP32 block is still the
// process-wide one), else replaces them; calls on one device are serialised by `mu`.
struct RunScratch {
    std::mutex mu;
    hydra_batch* batch = nullptr;
    int batch_slices = 0;
    uint64_t batch_tiles = 0;
    unsigned char* arena = nullptr;
    uint64_t arena_bytes = 0;
    double* segs = nullptr;
    uint64_t seg_cap = 0;
    cudaStream_t copy = nullptr;
    cudaEvent_t gen_done[2] = {nullptr, nullptr}, copy_done[2] = {nullptr, nullptr};

    void release() {
        if (copy) cudaStreamSynchronize(copy);
        if (batch) hydra_batch_destroy(batch);
        if (arena) cudaFree(arena);
        if (segs) cudaFree(segs);
        for (int k = 0; k < 2; ++k) {
            if (gen_done[k]) cudaEventDestroy(gen_done[k]);
            if (copy_done[k]) cudaEventDestroy(copy_done[k]);
            gen_done[k] = copy_done[k] = nullptr;
        }
        if (copy) cudaStreamDestroy(copy);
        batch = nullptr;
        arena = nullptr;
        segs = nullptr;
        copy = nullptr;
        batch_slices = 0;
        batch_tiles = arena_bytes = seg_cap = 0;
    }
};

std::mutex g_run_mu;
std::vector<RunScratch*> g_run_scratch;

RunScratch* run_scratch_for(int dev) {
    std::lock_guard<std::mutex> lk(g_run_mu);
    if (static_cast<int>(g_run_scratch.size()) <= dev) g_run_scratch.resize(dev + 1, nullptr);
    if (!g_run_scratch[dev]) g_run_scratch[dev] = new RunScratch();
    return g_run_scratch[dev];
}

// Make `rs` hold a runner for max_slices slices and ptiles integral tiles, an arena of at least
// arena_need bytes and at most arena_bytes (this call's share of its budget), segment storage
// for nsegs segments and, for host outputs, the copy stream.  Each buffer is allocated only when
// the one held is missing or too small (an arena larger than this call's share, or a runner far
// larger than needed, is released first).
hydra_status ensure_run_scratch(RunScratch* rs, int max_slices, uint64_t ptiles, uint64_t arena_need,
                                uint64_t arena_bytes, uint64_t nsegs, bool need_copy) {
    int block = kBatchBlock;
    {
        std::lock_guard<std::mutex> lk(g_shape_mu);
        block = g_batch_block_f32;
    }
    if (rs->batch && (rs->batch_slices < max_slices || rs->batch_tiles < ptiles || rs->batch->block_f32 != block ||
                      rs->batch_slices > 2 * max_slices + 64)) {
        hydra_batch_destroy(rs->batch);
        rs->batch = nullptr;
    }
    if (rs->arena && (rs->arena_bytes < arena_need || rs->arena_bytes > arena_bytes)) {
        cudaFree(rs->arena);
        rs->arena = nullptr;
        rs->arena_bytes = 0;
    }
    if (rs->segs && rs->seg_cap < nsegs) {
        cudaFree(rs->segs);
        rs->segs = nullptr;
        rs->seg_cap = 0;
    }
    if (!rs->batch) {
        const hydra_status st = hydra_batch_create(max_slices, ptiles ? ptiles : 1, &rs->batch);
        if (st != HYDRA_OK) return st;
        rs->batch_slices = max_slices;
        rs->batch_tiles = ptiles ? ptiles : 1;
    }
    cudaError_t err = cudaSuccess;
    if (arena_need && !rs->arena) {
        err = cudaMalloc(&rs->arena, arena_need);
        if (err == cudaSuccess) rs->arena_bytes = arena_need;
        else rs->arena = nullptr;
    }
    if (err == cudaSuccess && nsegs && !rs->segs) {
        err = cudaMalloc(&rs->segs, nsegs * 8 * sizeof(double));
        if (err == cudaSuccess) rs->seg_cap = nsegs;
        else rs->segs = nullptr;
    }
    if (err == cudaSuccess && need_copy && !rs->copy) {
        err = cudaStreamCreateWithFlags(&rs->copy, cudaStreamNonBlocking);
        for (int k = 0; k < 2 && err == cudaSuccess; ++k) {
            err = cudaEventCreateWithFlags(&rs->gen_done[k], cudaEventDisableTiming);
            if (err == cudaSuccess) err = cudaEventCreateWithFlags(&rs->copy_done[k], cudaEventDisableTiming);
        }
    }
    if (err != cudaSuccess) {
        cudaGetLastError();
        return err == cudaErrorMemoryAllocation ? fail(HYDRA_ERR_OOM, "batch run buffers: %s", cudaGetErrorString(err))
                                                : cuda_fail(err, "batch run set-up");
    }
    return HYDRA_OK;
}

}  // namespace

extern "C" {

hydra_status hydra_phsp_batch_run(hydra_batch_request* reqs, int nreq, size_t budget_bytes, hydra_stream_t stream) {
    const NvtxRange nvtx_range("hydra_phsp_batch_run");
    t_last_waves = t_last_slices = 0;
    if (!reqs || nreq < 1) return fail(HYDRA_ERR_INVALID_ARG, "need at least one request");
    const int dt = reqs[0].dtype;
    if (dt != HYDRA_F32 && dt != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "request 0: unknown dtype %d", dt);
    for (int i = 0; i < nreq; ++i) reqs[i].status = HYDRA_OK;
    for (int i = 0; i < nreq; ++i) {
        const hydra_status st = validate_request(reqs[i], i, dt);
        if (st != HYDRA_OK) return st;
    }
    const size_t elem = elem_of(dt);
    // integral segment storage (8 doubles per 2^21 events of each integral request) and the
    // runner's fixed buffers come out of the budget first; the rest is the output arena
    std::vector<uint64_t> seg_off(nreq, 0);
    uint64_t nsegs = 0, int_slices = 0;
    bool any_host = false;
    for (int i = 0; i < nreq; ++i) {
        if (reqs[i].kind == HYDRA_REQ_INTEGRATE) {
            seg_off[i] = nsegs;
            nsegs += (reqs[i].nevents + kSegEvents - 1) / kSegEvents;
            int_slices += (reqs[i].nevents + kRunIntSlice - 1) / kRunIntSlice;
        } else if (reqs[i].dest == HYDRA_DEST_HOST) {
            any_host = true;
        }
    }
    const uint64_t ptiles = (int_slices < kRunIntSlicesPerWave ? int_slices : kRunIntSlicesPerWave) * (kRunIntSlice / kTileEvents);
    const int max_slices = nreq + 64 < kRunMaxSlices ? nreq + 64 : kRunMaxSlices;
    const size_t fixed = table_size(max_slices, max_slices) + ptiles * sizeof(TileSums) +
                         static_cast<size_t>(max_slices) * sizeof(hydra_integral) + nsegs * 8 * sizeof(double) + (1u << 20);
    if (budget_bytes < fixed + (16u << 20))
        return fail(HYDRA_ERR_INVALID_ARG, "budget_bytes = %zu is below the %zu bytes these requests need at least",
                    budget_bytes, fixed + (16u << 20));
    const uint64_t arena_bytes = (budget_bytes - fixed) / 256 * 256;
    const uint64_t half = any_host ? arena_bytes / 2 / 256 * 256 : arena_bytes;

    // waves: requests in order; a generate request takes arena space for [4n+1][ld] values
    // (ld = count rounded up to 4, 256-byte aligned) and is split when it exceeds a half arena;
    // device-destination requests are written in place; integrals go in 2^26-event slices
    std::vector<std::vector<Slice>> waves(1);
    uint64_t used = 0, wave_int = 0;
    auto new_wave = [&]() {
        waves.emplace_back();
        used = 0;
        wave_int = 0;
    };
    for (int i = 0; i < nreq; ++i) {
        const hydra_batch_request& r = reqs[i];
        uint64_t first = 0;
        while (first < r.nevents) {
            if (static_cast<int>(waves.back().size()) >= max_slices) new_wave();
            Slice sl{i, first, 0, 0, 0};
            if (r.kind == HYDRA_REQ_INTEGRATE) {
                if (wave_int >= kRunIntSlicesPerWave) new_wave();
                sl.count = r.nevents - first < kRunIntSlice ? r.nevents - first : kRunIntSlice;
                ++wave_int;
            } else if (r.dest == HYDRA_DEST_DEVICE) {
                sl.count = r.nevents;
            } else {
                const uint64_t per_event = static_cast<uint64_t>(4 * r.n + 1) * elem;
                const uint64_t fit_max = (half / per_event) / 4 * 4;  // events of one slice in an empty half
                if (fit_max < 4) return fail(HYDRA_ERR_INVALID_ARG, "budget too small for one group of 4 events of request %d", i);
                uint64_t avail = used < half ? (half - used) / per_event / 4 * 4 : 0;
                if (avail < 4 || (avail < r.nevents - first && avail < fit_max / 8)) {
                    new_wave();  // start a fresh half rather than leave a sliver
                    avail = fit_max;
                }
                sl.count = r.nevents - first < avail ? r.nevents - first : avail;
                sl.ld = (sl.count + 3) / 4 * 4;
                sl.arena_off = used;
                used += (per_event * sl.ld + 255) / 256 * 256;
            }
            waves.back().push_back(sl);
            first += sl.count;
        }
    }
    if (waves.back().empty()) waves.pop_back();

    // arena bytes the waves use (both halves when outputs go to the host)
    uint64_t arena_need = 0;
    for (const auto& w : waves)
        for (const Slice& sl : w)
            if (reqs[sl.req].kind == HYDRA_REQ_GENERATE && reqs[sl.req].dest != HYDRA_DEST_DEVICE) {
                const uint64_t end = sl.arena_off + (static_cast<uint64_t>(4 * reqs[sl.req].n + 1) * elem * sl.ld + 255) / 256 * 256;
                arena_need = end > arena_need ? end : arena_need;
            }
    if (any_host && arena_need) arena_need = 2 * half;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return cuda_fail(err, "cudaGetDevice");
    RunScratch* rsp = run_scratch_for(dev);
    std::lock_guard<std::mutex> lk(rsp->mu);
    RunScratch& res = *rsp;
    hydra_status st = ensure_run_scratch(rsp, max_slices, ptiles, arena_need, arena_bytes, nsegs, any_host);
    if (st != HYDRA_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // on a failure after the first wave was enqueued, wait for the work already queued (it writes
    // the kept arena) before returning, so that no later call can race with it
    auto drain = [&](hydra_status status) {
        if (any_host) cudaStreamSynchronize(res.copy);
        cudaStreamSynchronize(s);
        return status;
    };
    std::vector<hydra_request> table;
    for (size_t w = 0; w < waves.size(); ++w) {
        const int b = static_cast<int>(w & 1);
        unsigned char* base = res.arena + (any_host ? b * half : 0);
        table.assign(waves[w].size(), hydra_request{});
        bool host_copies = false;
        std::vector<int> finals;
        for (size_t j = 0; j < waves[w].size(); ++j) {
            const Slice& sl = waves[w][j];
            const hydra_batch_request& r = reqs[sl.req];
            hydra_request& q = table[j];
            q.kind = r.kind;
            q.n = r.n;
            q.dtype = r.dtype;
            q.me = r.me;
            q.M = r.M;
            std::memcpy(q.masses, r.masses, sizeof q.masses);
            std::memcpy(q.params, r.params, sizeof q.params);
            q.seed = r.seed;
            q.event_offset = r.event_offset;
            q.first = sl.first;
            q.count = sl.count;
            if (r.kind == HYDRA_REQ_INTEGRATE) {
                q.total = r.nevents;
                q.seg_partials = res.segs + seg_off[sl.req] * 8;
                if (sl.first + sl.count == r.nevents) finals.push_back(static_cast<int>(j));
            } else if (r.dest == HYDRA_DEST_DEVICE) {
                q.out = r.out;
                q.ld = r.ld;
                q.weights = r.weights;
            } else {
                q.out = base + sl.arena_off;
                q.ld = sl.ld;
                q.weights = base + sl.arena_off + static_cast<uint64_t>(4 * r.n) * sl.ld * elem;
                host_copies |= r.dest == HYDRA_DEST_HOST;
            }
        }
        // this half of the arena is free once the copies of the wave before the previous one are done
        if (any_host && w >= 2) {
            err = cudaStreamWaitEvent(s, res.copy_done[b], 0);
            if (err != cudaSuccess) return drain(cuda_fail(err, "batch run arena wait"));
        }
        st = hydra_batch_run(res.batch, table.data(), static_cast<int>(table.size()), 1, stream);
        if (st != HYDRA_OK) return drain(st);
        if (host_copies) {
            err = cudaEventRecord(res.gen_done[b], s);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(res.copy, res.gen_done[b], 0);
            for (size_t j = 0; j < waves[w].size() && err == cudaSuccess; ++j) {
                const Slice& sl = waves[w][j];
                const hydra_batch_request& r = reqs[sl.req];
                if (r.kind != HYDRA_REQ_GENERATE || r.dest != HYDRA_DEST_HOST) continue;
                const unsigned char* src = base + sl.arena_off;
                err = cudaMemcpy2DAsync(static_cast<unsigned char*>(r.out) + sl.first * elem, r.ld * elem, src,
                                        sl.ld * elem, sl.count * elem, static_cast<size_t>(4 * r.n),
                                        cudaMemcpyDeviceToHost, res.copy);
                if (err == cudaSuccess)
                    err = cudaMemcpyAsync(static_cast<unsigned char*>(r.weights) + sl.first * elem,
                                          src + static_cast<uint64_t>(4 * r.n) * sl.ld * elem, sl.count * elem,
                                          cudaMemcpyDeviceToHost, res.copy);
            }
            if (err == cudaSuccess) err = cudaEventRecord(res.copy_done[b], res.copy);
            if (err != cudaSuccess) return drain(cuda_fail(err, "batch run output copy"));
        }
        for (int j : finals) {
            st = hydra_batch_result(res.batch, j, &reqs[waves[w][j].req].result);
            if (st != HYDRA_OK) return drain(st);
        }
    }
    if (any_host) err = cudaStreamSynchronize(res.copy);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return cuda_fail(err, "batch run synchronize");
    t_last_waves = waves.size();
    for (const auto& w : waves) t_last_slices += w.size();
    return HYDRA_OK;
}

}  // extern "C"

namespace hydra {

void release_batch_run_scratch() {
    std::lock_guard<std::mutex> lk(g_run_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (size_t d = 0; d < g_run_scratch.size(); ++d) {
        if (!g_run_scratch[d]) continue;
        cudaSetDevice(static_cast<int>(d));
        g_run_scratch[d]->release();
        delete g_run_scratch[d];
        g_run_scratch[d] = nullptr;
    }
    cudaSetDevice(cur);
}

}  // namespace hydra

extern "C" {

hydra_status hydra_phsp_batch_stats(uint64_t* waves, uint64_t* slices) {
    if (!waves || !slices) return fail(HYDRA_ERR_INVALID_ARG, "NULL output");
    *waves = t_last_waves;
    *slices = t_last_slices;
    return HYDRA_OK;
}

}  // extern "C"
