// phsp_batch.cuh -- the persistent batch kernel and the tables it reads (shared by the runner
// in phsp_batch.cu and the FP32 launch-shape variants in phsp_batch_f32.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "hydra_phsp.h"
#include "phsp_device.cuh"
#include "phsp_integral.cuh"

namespace hydra {

constexpr int kBatchBlock = 256;             // threads per block of the FP64 runs and of the auxiliary kernels
constexpr int kBatchEPT = 2;                 // events per thread of integral tiles
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
    int32_t gen_ept[kNMax + 1];       // events per thread of generation tiles, by n (1, 2 or 4)
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

// Events per thread of a generation tile (each run's header carries one per n; 1, 2 or 4 for
// FP32, 1 or 2 for FP64).
template <int N, typename R, int kEPT>
__device__ __forceinline__ void generate_tile(const DecayConsts& C, const BatchEntry& e, uint64_t lt, int lane) {
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

// Events per thread a generation tile may use: FP32 1, 2 or 4 up to n = 6 and 1 or 2 above
// (four lockstep events of the longer decays would raise the register count of the whole
// persistent kernel); FP64 two.
template <int N, typename R>
__host__ __device__ constexpr bool batch_ept_allowed(int ept) {
    if constexpr (std::is_same<R, float>::value) return ept == 1 || ept == 2 || (ept == 4 && N <= 6);
    else return ept == 2;
}

template <int N, typename R>
__device__ __forceinline__ void generate_tile_e(int ept, const DecayConsts& C, const BatchEntry& e, uint64_t lt, int lane) {
    if constexpr (std::is_same<R, float>::value) {
        if constexpr (N <= 6) {
            if (ept == 4) {
                generate_tile<N, R, 4>(C, e, lt, lane);
                return;
            }
        }
        if (ept == 1) generate_tile<N, R, 1>(C, e, lt, lane);
        else generate_tile<N, R, 2>(C, e, lt, lane);
    } else {
        generate_tile<N, R, 2>(C, e, lt, lane);
    }
}

template <typename R>
__device__ __forceinline__ void generate_tile_n(int n, int ept, const DecayConsts& C, const BatchEntry& e, uint64_t lt,
                                                int lane) {
    switch (n) {
        case 2: generate_tile_e<2, R>(ept, C, e, lt, lane); break;
        case 3: generate_tile_e<3, R>(ept, C, e, lt, lane); break;
        case 4: generate_tile_e<4, R>(ept, C, e, lt, lane); break;
        case 5: generate_tile_e<5, R>(ept, C, e, lt, lane); break;
        case 6: generate_tile_e<6, R>(ept, C, e, lt, lane); break;
        case 7: generate_tile_e<7, R>(ept, C, e, lt, lane); break;
        case 8: generate_tile_e<8, R>(ept, C, e, lt, lane); break;
        case 9: generate_tile_e<9, R>(ept, C, e, lt, lane); break;
        case 10: generate_tile_e<10, R>(ept, C, e, lt, lane); break;
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

// RG: arithmetic of generation tiles (float, double or df); RI: of integral tiles; BLOCK:
// threads per block.
template <typename RG, typename RI, int BLOCK>
__global__ void __launch_bounds__(BLOCK) phsp_batch_kernel(BatchHeader* __restrict__ hdr,
                                                           TileSums* __restrict__ partials) {
    constexpr int kWarps = BLOCK / 32;
    if constexpr (std::is_same<RG, df>::value) {
        df_sincos_table_init();
        __syncthreads();
    }
    __shared__ DecayConsts sC[kWarps];
    __shared__ MEConsts sP[kWarps];
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
            generate_tile_n<RG>(e.n, hdr->gen_ept[e.n], sC[warp], e, lt, lane);
        } else {
            const TileSums ts = integrate_tile_n<RI>(e.n, e.me, sC[warp], sP[warp], e, e.first / kTileEvents + lt, lane);
            if (lane == 0) partials[e.partial_begin + lt] = ts;
        }
        __syncwarp();
    }
}

// The FP32 persistent kernel for a block of 128, 256 or 512 threads (phsp_batch_f32.cu).
const void* batch_kernel_f32(int block);
void launch_batch_kernel_f32(int block, int grid, BatchHeader* hdr, TileSums* partials, cudaStream_t s);

}  // namespace hydra
