// phsp_extras.cu -- moving parents, unweighted samples and event compaction (section 4.2:
// Listing 4's Generate(Mother, ...) and "weighted and unweighted samples").
//
//   phsp_generate_boost_kernel<N, R, EPT>  the generator of phsp.cu whose sink takes every
//                                          daughter from the parent rest frame to the lab by
//                                          the pure boost to the parent's momentum (one for
//                                          all events, or one per event read from HBM)
//   unweight_max / unweight_count / unweight_scan / unweight_write
//                                          accept-reject against w_max: event e is kept when
//                                          u_e w_max < w_e (u_e its draw 3n-4); indices of the
//                                          kept events are written in event order (stable,
//                                          deterministic: accept bits and counts per
//                                          4096-event tile, an exclusive scan, ranks by warp
//                                          ballots over the stored bits)
//   gather_events                          copies kept events into a compact SoA buffer
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

// ------------------------------------------------------------------------------------
// Moving parent
// ------------------------------------------------------------------------------------
template <typename R> __device__ __forceinline__ R from_out(typename Prec<R>::Out v);
template <> __device__ __forceinline__ float from_out<float>(float v) { return v; }
template <> __device__ __forceinline__ double from_out<double>(double v) { return v; }
template <> __device__ __forceinline__ df from_out<df>(double v) {
    const float h = __double2float_rn(v);
    return df{h, __double2float_rn(v - static_cast<double>(h))};
}

// Pure boost of each daughter from the parent rest frame to the frame where the parent has
// 4-momentum (P0, P) and mass M:  E' = (P0 E + P.p)/M,  p' = p + P (E' + E)/(P0 + M).
template <typename R, int EPT>
struct BoostSink {
    StoreSink<R, EPT> inner;
    R P0[EPT], Px[EPT], Py[EPT], Pz[EPT], invPM[EPT];
    R invM;
    __device__ __forceinline__ void subsystem_mass(int, const R (&)[EPT]) {}
    __device__ __forceinline__ void daughter(int i, const R (&E)[EPT], const R (&px)[EPT],
                                             const R (&py)[EPT], const R (&pz)[EPT]) {
        using P = Prec<R>;
        R oE[EPT], ox[EPT], oy[EPT], oz[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const R bp = P::fma_(Pz[q], pz[q], P::fma_(Py[q], py[q], Px[q] * px[q]));
            const R E1 = P::fma_(P0[q], E[q], bp) * invM;
            const R f = (E1 + E[q]) * invPM[q];
            oE[q] = E1;
            ox[q] = P::fma_(f, Px[q], px[q]);
            oy[q] = P::fma_(f, Py[q], py[q]);
            oz[q] = P::fma_(f, Pz[q], pz[q]);
        }
        inner.daughter(i, oE, ox, oy, oz);
    }
    __device__ __forceinline__ void weight(const typename Prec<R>::W (&w)[EPT]) { inner.weight(w); }
};

// Events e0 .. e0+E-1 of a moving parent: load (or take) each parent momentum, form
// P0 = sqrt(M^2 + p^2) and 1/(P0 + M), run the event group with the boosting sink.
template <int N, typename R, int E>
__device__ __forceinline__ void boosted_group(const DecayConsts& C, uint64_t e0, uint64_t event_offset,
                                              typename Prec<R>::Out* out, uint64_t ld, typename Prec<R>::Out* weights,
                                              const typename Prec<R>::Out* mothers, uint64_t mld,
                                              const R (&U)[3], R M, R M2, R invM) {
    using P = Prec<R>;
    BoostSink<R, E> sink{StoreSink<R, E>{out + e0, weights + e0, ld}};
    sink.invM = invM;
    uint64_t ev[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
        ev[q] = event_offset + e0 + q;
        R px = U[0], py = U[1], pz = U[2];
        if (mothers) {
            px = from_out<R>(mothers[e0 + q]);
            py = from_out<R>(mothers[mld + e0 + q]);
            pz = from_out<R>(mothers[2 * mld + e0 + q]);
        }
        const R P0 = P::sqrt_(P::fma_(pz, pz, P::fma_(py, py, P::fma_(px, px, M2))));
        sink.P0[q] = P0;
        sink.Px[q] = px;
        sink.Py[q] = py;
        sink.Pz[q] = pz;
        sink.invPM[q] = P::rcp(P0 + M);
    }
    raubold_lynch_group<N, R, E>(C, ev, sink);
}

// mothers: per-event parent momenta [3][mld] of the output type, or NULL for the single
// momentum (ux, uy, uz).  Groups of EPT consecutive events; the ragged tail one by one.
template <int N, typename R, int EPT>
__global__ void __launch_bounds__(512) phsp_generate_boost_kernel(
    const __grid_constant__ DecayConsts C, uint64_t nevents, uint64_t event_offset,
    typename Prec<R>::Out* __restrict__ out, uint64_t ld, typename Prec<R>::Out* __restrict__ weights,
    const typename Prec<R>::Out* __restrict__ mothers, uint64_t mld, double ux, double uy, double uz) {
    using P = Prec<R>;
    using Out = typename P::Out;
    if constexpr (std::is_same<R, df>::value) {
        df_sincos_table_init();
        __syncthreads();
    }
    const R M = P::M(C);
    const R invM = P::rcp(M);
    const R M2 = M * M;
    const R U[3] = {from_out<R>(static_cast<Out>(ux)), from_out<R>(static_cast<Out>(uy)),
                    from_out<R>(static_cast<Out>(uz))};
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t groups = nevents / EPT;
    for (uint64_t g = tid; g < groups; g += stride)
        boosted_group<N, R, EPT>(C, g * EPT, event_offset, out, ld, weights, mothers, mld, U, M, M2, invM);
    if constexpr (EPT > 1) {
        const uint64_t e = groups * EPT + tid;
        if (e < nevents)
            boosted_group<N, R, 1>(C, e, event_offset, out, ld, weights, mothers, mld, U, M, M2, invM);
    }
}

template <typename R, int EPT>
static const void* boost_kernel_n(int n) {
    switch (n) {
        case 2: return reinterpret_cast<const void*>(&phsp_generate_boost_kernel<2, R, EPT>);
        case 3: return reinterpret_cast<const void*>(&phsp_generate_boost_kernel<3, R, EPT>);
        case 4: return reinterpret_cast<const void*>(&phsp_generate_boost_kernel<4, R, EPT>);
        case 5: return reinterpret_cast<const void*>(&phsp_generate_boost_kernel<5, R, EPT>);
        case 6: return reinterpret_cast<const void*>(&phsp_generate_boost_kernel<6, R, EPT>);
        case 7: return reinterpret_cast<const void*>(&phsp_generate_boost_kernel<7, R, EPT>);
        case 8: return reinterpret_cast<const void*>(&phsp_generate_boost_kernel<8, R, EPT>);
        case 9: return reinterpret_cast<const void*>(&phsp_generate_boost_kernel<9, R, EPT>);
        case 10: return reinterpret_cast<const void*>(&phsp_generate_boost_kernel<10, R, EPT>);
    }
    return nullptr;
}

// ------------------------------------------------------------------------------------
// Unweighting
// ------------------------------------------------------------------------------------
constexpr int kUwBlock = 256;
constexpr int kUwPerThread = 16;
constexpr int kUwTile = kUwBlock * kUwPerThread;  // 4096 events per block tile
constexpr int kUwWarpRun = 32 * kUwPerThread;     // 512 consecutive events per warp within a tile

// Largest weight (order-preserving integer bits of non-negative FP32 / FP64 values).  With
// 16-byte aligned weights each thread reads four 16-byte vectors per pass (the scalar loop
// kept too few bytes in flight: 1.35 TB/s); the remainder is read element by element.
template <typename T>
__device__ __forceinline__ unsigned long long weight_bits(T v) {
    if constexpr (sizeof(T) == 4) return __float_as_uint(fmaxf(v, 0.0f));
    else return static_cast<unsigned long long>(__double_as_longlong(fmax(v, 0.0)));
}

template <typename T>
__global__ void __launch_bounds__(kUwBlock) unweight_max(const T* __restrict__ w, uint64_t nevents,
                                                         unsigned long long* __restrict__ out_bits) {
    constexpr int W = 16 / sizeof(T);  // weights per 16-byte vector
    constexpr int kU = 4;              // vectors per thread per pass
    unsigned long long best = 0;
    const uint64_t nthreads = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    uint64_t head = 0;  // weights taken by the vector loop
    if (reinterpret_cast<uintptr_t>(w) % 16 == 0) {
        const uint64_t nvec = nevents / W;
        const uint4* v = reinterpret_cast<const uint4*>(w);
        uint64_t i = tid;
        for (; i + (kU - 1) * nthreads < nvec; i += kU * nthreads) {
            uint4 q[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) q[u] = v[i + u * nthreads];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const T* x = reinterpret_cast<const T*>(&q[u]);
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    const unsigned long long b = weight_bits<T>(x[k]);
                    best = b > best ? b : best;
                }
            }
        }
        for (; i < nvec; i += nthreads) {
            const uint4 q = v[i];
            const T* x = reinterpret_cast<const T*>(&q);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const unsigned long long b = weight_bits<T>(x[k]);
                best = b > best ? b : best;
            }
        }
        head = nvec * W;
    }
    for (uint64_t e = head + tid; e < nevents; e += nthreads) {
        const unsigned long long b = weight_bits<T>(w[e]);
        best = b > best ? b : best;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
        best = o > best ? o : best;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, best);
}

// Accept decision of event e (kinematic draws 0..3n-5, the accept draw is 3n-4).
template <typename T>
__device__ __forceinline__ bool accept_event(const DecayConsts& C, int draw, uint64_t ev, T w, T w_max) {
    uint32_t x[4];
    philox4x32_10(static_cast<uint32_t>(ev), static_cast<uint32_t>(ev >> 32), draw / 4, 0u, C.rk0, C.rk1, x);
    const uint32_t xd = x[draw % 4];
    if constexpr (sizeof(T) == 4) {
        const float u = __fmaf_rn(__uint2float_rn(xd), 2.3283064365386962890625e-10f, 1.16415321826934814453125e-10f);
        return __fmul_rn(u, w_max) < w;
    } else {
        const double u = __fma_rn(__uint2double_rn(xd), 2.3283064365386962890625e-10, 1.16415321826934814453125e-10);
        return __dmul_rn(u, w_max) < w;
    }
}

template <typename T>
__device__ __forceinline__ T bits_to_value(unsigned long long b) {
    if constexpr (sizeof(T) == 4) return __uint_as_float(static_cast<uint32_t>(b));
    else return __longlong_as_double(static_cast<long long>(b));
}

// The accept decisions of one thread in a block tile, as a bit mask: warp v of the block takes
// the run of 512 consecutive events base + 512 v .. (row j: 32 events, lane l: event j*32 + l).
template <typename T>
__device__ __forceinline__ uint32_t accept_mask(const DecayConsts& C, int draw, const T* __restrict__ w,
                                                uint64_t nevents, uint64_t event_offset, T w_max, uint64_t run0,
                                                int lane) {
    uint32_t mask = 0;
#pragma unroll
    for (int j = 0; j < kUwPerThread; ++j) {
        const uint64_t e = run0 + static_cast<uint64_t>(j * 32 + lane);
        if (e < nevents && accept_event<T>(C, draw, event_offset + e, w[e], w_max)) mask |= 1u << j;
    }
    return mask;
}

template <typename T>
__global__ void __launch_bounds__(kUwBlock) unweight_count(const __grid_constant__ DecayConsts C, int draw,
                                                           const T* __restrict__ w, uint64_t nevents,
                                                           uint64_t event_offset,
                                                           const unsigned long long* __restrict__ wmax_bits,
                                                           uint32_t* __restrict__ tile_counts,
                                                           uint32_t* __restrict__ masks) {
    __shared__ uint32_t warp_cnt[kUwBlock / 32];
    const T w_max = bits_to_value<T>(*wmax_bits);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t run0 = static_cast<uint64_t>(blockIdx.x) * kUwTile + static_cast<uint64_t>(warp) * kUwWarpRun;
    const uint32_t mask = accept_mask<T>(C, draw, w, nevents, event_offset, w_max, run0, lane);
    masks[static_cast<uint64_t>(blockIdx.x) * kUwBlock + threadIdx.x] = mask;
    uint32_t cnt = __popc(mask);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if (lane == 0) warp_cnt[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int i = 0; i < kUwBlock / 32; ++i) s += warp_cnt[i];
        tile_counts[blockIdx.x] = s;
    }
}

// Exclusive scan of the tile counts by one block (each thread scans a contiguous range).
__global__ void __launch_bounds__(1024) unweight_scan(const uint32_t* __restrict__ counts, uint64_t ntiles,
                                                      uint64_t* __restrict__ offsets, uint64_t* __restrict__ total) {
    __shared__ uint64_t part[1024];
    const uint64_t per = (ntiles + blockDim.x - 1) / blockDim.x;
    const uint64_t lo = threadIdx.x * per, hi = lo + per < ntiles ? lo + per : ntiles;
    uint64_t s = 0;
    for (uint64_t i = lo; i < hi; ++i) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t acc = 0;
        for (unsigned i = 0; i < blockDim.x; ++i) {
            const uint64_t v = part[i];
            part[i] = acc;
            acc += v;
        }
        *total = acc;
    }
    __syncthreads();
    uint64_t acc = part[threadIdx.x];
    for (uint64_t i = lo; i < hi; ++i) {
        offsets[i] = acc;
        acc += counts[i];
    }
}

// Kept indices in event order, from the accept bits the count pass stored: each warp's run of
// 512 events follows the runs of the warps before it in the tile (one block-wide prefix of the
// warp totals), and within the run the rows follow each other with the lanes in order (a
// ballot per row).  (Recomputing the decisions here instead, a second Philox block and weight
// read per event, made this pass the slowest of the four.)
__global__ void __launch_bounds__(kUwBlock) unweight_write(const uint32_t* __restrict__ masks,
                                                           const uint64_t* __restrict__ offsets,
                                                           int64_t* __restrict__ indices) {
    __shared__ uint32_t warp_cnt[kUwBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t run0 = static_cast<uint64_t>(blockIdx.x) * kUwTile + static_cast<uint64_t>(warp) * kUwWarpRun;
    const uint32_t mask = masks[static_cast<uint64_t>(blockIdx.x) * kUwBlock + threadIdx.x];
    uint32_t cnt = __popc(mask);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if (lane == 0) warp_cnt[warp] = cnt;
    __syncthreads();
    uint64_t run = offsets[blockIdx.x];
    for (int i = 0; i < warp; ++i) run += warp_cnt[i];
    const uint32_t below = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kUwPerThread; ++j) {
        const bool a = (mask >> j) & 1u;
        const uint32_t ballot = __ballot_sync(0xffffffffu, a);
        if (a) indices[run + __popc(ballot & below)] = static_cast<int64_t>(run0 + static_cast<uint64_t>(j * 32 + lane));
        run += __popc(ballot);
    }
}

// dst[(i*4 + c)*dst_ld + j] = src[(i*4 + c)*src_ld + idx[j]], dst_w[j] = src_w[idx[j]].
template <typename T>
__global__ void __launch_bounds__(256) gather_events(int arrays, const T* __restrict__ src, uint64_t src_ld,
                                                     const T* __restrict__ src_w, const int64_t* __restrict__ idx,
                                                     uint64_t count, T* __restrict__ dst, uint64_t dst_ld,
                                                     T* __restrict__ dst_w) {
    for (uint64_t j = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < count;
         j += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t s = static_cast<uint64_t>(idx[j]);
        for (int a = 0; a < arrays; ++a) dst[a * dst_ld + j] = src[a * src_ld + s];
        if (src_w && dst_w) dst_w[j] = src_w[s];
    }
}

// Per-device scratch for unweighting: tile counts and offsets, the max and the total.
struct UwScratch {
    std::mutex mu;
    uint32_t* counts = nullptr;
    uint64_t* offsets = nullptr;
    uint32_t* masks = nullptr;    // accept bits of the count pass, one word per thread of a tile
    uint64_t cap = 0;
    unsigned long long* wmax = nullptr;  // [0] max bits, [1] total
    unsigned long long* h = nullptr;     // pinned copy of the two
};
static std::mutex g_uw_mu;
static std::vector<UwScratch*> g_uw;

static UwScratch* uw_scratch() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_uw_mu);
    if (static_cast<int>(g_uw.size()) <= dev) g_uw.resize(dev + 1, nullptr);
    if (!g_uw[dev]) g_uw[dev] = new UwScratch();
    return g_uw[dev];
}

// ------------------------------------------------------------------------------------
// Model evaluation on stored events: f_e = w_e |ME|^2(p_e), values and the deterministic
// integral (the tile / segment / fold tree of the generated-event integral).
// ------------------------------------------------------------------------------------
// f = w |ME|^2 from one event's components c[a][k] (daughter a = 0..2, k = E, px, py, pz), both
// evaluation kernels: FP32 events in FP32, FP64 events with K = double (native FP64) or
// K = df: there the pair masses s = E^2 - p^2 and m0^2 - s stay in native FP64 (cancellations
// that a narrow resonance amplifies several hundredfold: double-float there left ~1e-11 on
// |ME|^2 near the phi(1020)), and the well-conditioned rest of |ME|^2 runs in double-float
// from m0^2 - s split by integer operations.
template <typename R, typename K>
__device__ __forceinline__ R dalitz_value(const MEConsts& P, R we, const R (&c)[3][4]) {
    using Q = Prec<R>;
    R m2[2];
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
        R v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = c[pr][k] + c[pr + 1][k];
        m2[pr] = Q::fma_(v[0], v[0], -Q::fma_(v[3], v[3], Q::fma_(v[2], v[2], v[1] * v[1])));
    }
    if constexpr (std::is_same<K, df>::value) {
        const df xa = df_from_double(P.a_m2 - m2[0]), xb = df_from_double(P.b_m2 - m2[1]);
        return we * to_w<df>(dalitz_2bw_x<df>(P, xa, xb));
    } else {
        return we * dalitz_2bw<R>(P, m2[0], m2[1]);
    }
}

template <typename R, int ME, typename K>
__device__ __forceinline__ R eval_event(const R* __restrict__ ev, uint64_t ld, const R* __restrict__ w,
                                        const MEConsts& P, uint64_t e) {
    const R we = w[e];
    if constexpr (ME == HYDRA_ME_DALITZ_2BW) {
        R c[3][4];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int k = 0; k < 4; ++k) c[a][k] = ev[static_cast<uint64_t>(4 * a + k) * ld + e];
        return dalitz_value<R, K>(P, we, c);
    }
    return we;
}

template <typename R, int ME, typename K>
__global__ void __launch_bounds__(256) evaluate_tiles(uint64_t nevents, const R* __restrict__ ev, uint64_t ld,
                                                      const R* __restrict__ w, const __grid_constant__ MEConsts P,
                                                      R* __restrict__ values, uint64_t tile_begin, uint64_t ntiles,
                                                      TileSums* __restrict__ partials) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t t = warp; t < ntiles; t += nwarps) {
        const uint64_t base = (tile_begin + t) * kTileEvents;
        double af = 0.0, af2 = 0.0, aw = 0.0, aw2 = 0.0;
        for (int g = 0; g < kLaneIters / kGroupEvents; ++g) {
            R sf = R(0), sf2 = R(0), sw = R(0), sw2 = R(0);
            for (int i = 0; i < kGroupEvents; ++i) {
                const uint64_t e = base + static_cast<uint64_t>(32 * (g * kGroupEvents + i) + lane);
                if (e < nevents) {
                    const R we = w[e];
                    const R f = eval_event<R, ME, K>(ev, ld, w, P, e);
                    if (values) values[e] = f;
                    sf += f;
                    sf2 = Prec<R>::fma_(f, f, sf2);
                    sw += we;
                    sw2 = Prec<R>::fma_(we, we, sw2);
                }
            }
            af += static_cast<double>(sf);
            af2 += static_cast<double>(sf2);
            aw += static_cast<double>(sw);
            aw2 += static_cast<double>(sw2);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            af += __shfl_xor_sync(0xffffffffu, af, off);
            af2 += __shfl_xor_sync(0xffffffffu, af2, off);
            aw += __shfl_xor_sync(0xffffffffu, aw, off);
            aw2 += __shfl_xor_sync(0xffffffffu, aw2, off);
        }
        if (lane == 0) partials[t] = TileSums{af, af2, aw, aw2};
    }
}

// The same with 16-byte loads: lane l takes the runs of W = 16 / sizeof(R) consecutive events
// starting at base + 256 g + 32 W j + W l (j < 8 / W) of each group g of 256 events, so that a
// warp reads whole lines of every component with a quarter (FP32) or half (FP64) of the load
// instructions and several vectors in flight.  A lane still sums 8 events per group in R and
// the groups in FP64, in a fixed order (the event-to-lane assignment differs from
// evaluate_tiles, so the sums agree to rounding).  Needs 16-byte aligned events, weights and
// values and ld % W == 0; a run that crosses nevents is taken element by element.
template <typename R>
struct Vec16;
template <>
struct Vec16<float> {
    using T = float4;
    static constexpr int W = 4;
    __device__ static void get(const float* p, float (&v)[4]) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    }
    __device__ static void put(float* p, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct Vec16<double> {
    using T = double2;
    static constexpr int W = 2;
    __device__ static void get(const double* p, double (&v)[2]) {
        const double2 x = *reinterpret_cast<const double2*>(p);
        v[0] = x.x; v[1] = x.y;
    }
    __device__ static void put(double* p, const double (&v)[2]) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    }
};

template <typename R, int ME, typename K>
__global__ void __launch_bounds__(256) evaluate_tiles_vec(uint64_t nevents, const R* __restrict__ ev, uint64_t ld,
                                                          const R* __restrict__ w, const __grid_constant__ MEConsts P,
                                                          R* __restrict__ values, uint64_t tile_begin, uint64_t ntiles,
                                                          TileSums* __restrict__ partials) {
    using V = Vec16<R>;
    constexpr int W = V::W;
    constexpr int kRuns = kGroupEvents / W;       // runs of W events per lane per group
    constexpr int kGroupSpan = 32 * kGroupEvents;  // events of one group across the warp
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t t = warp; t < ntiles; t += nwarps) {
        const uint64_t base = (tile_begin + t) * kTileEvents;
        double af = 0.0, af2 = 0.0, aw = 0.0, aw2 = 0.0;
        for (int g = 0; g < kTileEvents / kGroupSpan; ++g) {
            R sf = R(0), sf2 = R(0), sw = R(0), sw2 = R(0);
#pragma unroll
            for (int j = 0; j < kRuns; ++j) {
                const uint64_t e0 = base + static_cast<uint64_t>(g * kGroupSpan + j * 32 * W + lane * W);
                R f[W], we[W];
                if (e0 + W <= nevents) {
                    V::get(w + e0, we);
                    if constexpr (ME == HYDRA_ME_DALITZ_2BW) {
                        R c[3][4][W];
#pragma unroll
                        for (int a = 0; a < 3; ++a)
#pragma unroll
                            for (int k = 0; k < 4; ++k) V::get(ev + static_cast<uint64_t>(4 * a + k) * ld + e0, c[a][k]);
#pragma unroll
                        for (int q = 0; q < W; ++q) {
                            R cq[3][4];
#pragma unroll
                            for (int a = 0; a < 3; ++a)
#pragma unroll
                                for (int k = 0; k < 4; ++k) cq[a][k] = c[a][k][q];
                            f[q] = dalitz_value<R, K>(P, we[q], cq);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < W; ++q) f[q] = we[q];
                    }
                    if (values) V::put(values + e0, f);
                } else {
#pragma unroll
                    for (int q = 0; q < W; ++q) {
                        we[q] = R(0);
                        f[q] = R(0);
                        if (e0 + q < nevents) {
                            we[q] = w[e0 + q];
                            f[q] = eval_event<R, ME, K>(ev, ld, w, P, e0 + q);
                            if (values) values[e0 + q] = f[q];
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < W; ++q) {
                    sf += f[q];
                    sf2 = Prec<R>::fma_(f[q], f[q], sf2);
                    sw += we[q];
                    sw2 = Prec<R>::fma_(we[q], we[q], sw2);
                }
            }
            af += static_cast<double>(sf);
            af2 += static_cast<double>(sf2);
            aw += static_cast<double>(sw);
            aw2 += static_cast<double>(sw2);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            af += __shfl_xor_sync(0xffffffffu, af, off);
            af2 += __shfl_xor_sync(0xffffffffu, af2, off);
            aw += __shfl_xor_sync(0xffffffffu, aw, off);
            aw2 += __shfl_xor_sync(0xffffffffu, aw2, off);
        }
        if (lane == 0) partials[t] = TileSums{af, af2, aw, aw2};
    }
}

__global__ void __launch_bounds__(kSegBlock) eval_reduce_segments(const TileSums* __restrict__ partials, uint64_t ntiles,
                                                                  uint64_t seg_begin, double* __restrict__ seg_out) {
    const uint64_t seg = blockIdx.x;  // one block per segment
    const uint64_t t0 = seg * kSegTiles;
    const uint64_t nt = ntiles - t0 < kSegTiles ? ntiles - t0 : kSegTiles;
    segment_sums_block(partials + t0, nt, seg_out + (seg_begin + seg) * 8);
}

__global__ void __launch_bounds__(32) eval_finalize(const double* __restrict__ seg, uint64_t nseg, uint64_t nevents,
                                                    hydra_integral* __restrict__ out) {
    fold_segments(seg, nseg, nevents, threadIdx.x & 31, out);
}

struct EvalScratch {
    std::mutex mu;
    TileSums* tiles = nullptr;
    double* segs = nullptr;
    uint64_t seg_cap = 0;
    hydra_integral* d_res = nullptr;
    hydra_integral* h_res = nullptr;
};
static std::mutex g_ev_mu;
static std::vector<EvalScratch*> g_ev;

static EvalScratch* eval_scratch() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_ev_mu);
    if (static_cast<int>(g_ev.size()) <= dev) g_ev.resize(dev + 1, nullptr);
    if (!g_ev[dev]) g_ev[dev] = new EvalScratch();
    return g_ev[dev];
}

// Frees the moving-parent / unweighting / evaluation scratch of every device (hydra_shutdown).
void release_extras_scratch() {
    int cur = 0;
    cudaGetDevice(&cur);
    {
        std::lock_guard<std::mutex> lk(g_uw_mu);
        for (size_t d = 0; d < g_uw.size(); ++d) {
            UwScratch* s = g_uw[d];
            if (!s) continue;
            cudaSetDevice(static_cast<int>(d));
            if (s->counts) cudaFree(s->counts);
            if (s->offsets) cudaFree(s->offsets);
            if (s->masks) cudaFree(s->masks);
            if (s->wmax) cudaFree(s->wmax);
            if (s->h) cudaFreeHost(s->h);
            delete s;
            g_uw[d] = nullptr;
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_ev_mu);
        for (size_t d = 0; d < g_ev.size(); ++d) {
            EvalScratch* s = g_ev[d];
            if (!s) continue;
            cudaSetDevice(static_cast<int>(d));
            if (s->tiles) cudaFree(s->tiles);
            if (s->segs) cudaFree(s->segs);
            if (s->d_res) cudaFree(s->d_res);
            if (s->h_res) cudaFreeHost(s->h_res);
            delete s;
            g_ev[d] = nullptr;
        }
    }
    cudaSetDevice(cur);
}

}  // namespace hydra

using namespace hydra;

extern "C" {

hydra_status hydra_phsp_generate_boosted(double M, int n, const double* masses, uint64_t nevents,
                                         uint64_t seed, uint64_t event_offset, hydra_dtype dtype,
                                         const double* mother_p, const void* mothers, uint64_t mld,
                                         void* out, uint64_t ld, void* weights, hydra_stream_t stream) {
    const NvtxRange nvtx_range("hydra_phsp_generate_boosted");
    DecayConsts C;
    hydra_status st = make_consts(M, n, masses, seed, &C);
    if (st != HYDRA_OK) return st;
    if (dtype != HYDRA_F32 && dtype != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(dtype));
    if (event_offset + nevents < event_offset) return fail(HYDRA_ERR_INVALID_ARG, "event_offset + nevents overflows 64 bits");
    if ((mother_p == nullptr) == (mothers == nullptr))
        return fail(HYDRA_ERR_INVALID_ARG, "give exactly one of mother_p (one momentum) and mothers (per event)");
    if (mother_p)
        for (int c = 0; c < 3; ++c)
            if (!std::isfinite(mother_p[c])) return fail(HYDRA_ERR_INVALID_ARG, "mother momentum is not finite");
    if (nevents == 0) return HYDRA_OK;
    if (!out || !weights) return fail(HYDRA_ERR_INVALID_ARG, "out and weights must not be NULL");
    if (ld < nevents) return fail(HYDRA_ERR_INVALID_ARG, "ld < nevents");
    if (mothers && mld < nevents) return fail(HYDRA_ERR_INVALID_ARG, "mld < nevents");
    if ((reinterpret_cast<uintptr_t>(out) & 15u) || (reinterpret_cast<uintptr_t>(weights) & 15u) || ld % 4 != 0)
        return fail(HYDRA_ERR_MISALIGNED, "out and weights must be 16-byte aligned and ld a multiple of 4");
    // the generator's tuned shape: FP32 groups of 1, 2 or 4 events (16-byte stores where the
    // generator is HBM-bound), FP64 groups of 1 or 2
    int block = 256, ept = 1;
    hydra_get_launch_config(HYDRA_KERNEL_GENERATE, n, dtype, &block, &ept);
    ept = ept >= 4 && dtype == HYDRA_F32 ? 4 : (ept >= 2 ? 2 : 1);
    const void* k = nullptr;
    if (dtype == HYDRA_F32)
        k = ept == 4 ? boost_kernel_n<float, 4>(n) : (ept == 2 ? boost_kernel_n<float, 2>(n) : boost_kernel_n<float, 1>(n));
    else if (g_fp64_arith.load() == HYDRA_FP64_NATIVE) k = ept == 2 ? boost_kernel_n<double, 2>(n) : boost_kernel_n<double, 1>(n);
    else k = ept == 2 ? boost_kernel_n<df, 2>(n) : boost_kernel_n<df, 1>(n);
    double ux = mother_p ? mother_p[0] : 0.0, uy = mother_p ? mother_p[1] : 0.0, uz = mother_p ? mother_p[2] : 0.0;
    const int grid = grid_for(k, block, (nevents + ept - 1) / ept);
    void* args[] = {&C, &nevents, &event_offset, &out, &ld, &weights, const_cast<void**>(&mothers), &mld, &ux, &uy, &uz};
    const cudaError_t err = cudaLaunchKernel(k, dim3(grid), dim3(block), args, 0, reinterpret_cast<cudaStream_t>(stream));
    if (err != cudaSuccess) return cuda_fail(err, "boosted generate launch");
    return HYDRA_OK;
}

hydra_status hydra_phsp_unweight(int n, uint64_t nevents, uint64_t seed, uint64_t event_offset, hydra_dtype dtype,
                                 const void* weights, double w_max, int64_t* indices, uint64_t* naccepted,
                                 double* w_max_used, hydra_stream_t stream) {
    const NvtxRange nvtx_range("hydra_phsp_unweight");
    if (n < 2 || n > kNMax) return fail(HYDRA_ERR_UNSUPPORTED_N, "n = %d outside [2, %d]", n, kNMax);
    if (dtype != HYDRA_F32 && dtype != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(dtype));
    if (!naccepted) return fail(HYDRA_ERR_INVALID_ARG, "naccepted is NULL");
    if (event_offset + nevents < event_offset) return fail(HYDRA_ERR_INVALID_ARG, "event_offset + nevents overflows 64 bits");
    if (!std::isfinite(w_max)) return fail(HYDRA_ERR_INVALID_ARG, "w_max is not finite");
    *naccepted = 0;
    if (nevents == 0) return HYDRA_OK;
    if (!weights || !indices) return fail(HYDRA_ERR_INVALID_ARG, "weights and indices must not be NULL");
    DecayConsts C;
    std::memset(&C, 0, sizeof C);
    uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        C.rk0[r] = k0;
        C.rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    const int draw = 3 * n - 4;
    UwScratch* s = uw_scratch();
    if (!s) return fail(HYDRA_ERR_CUDA, "no current CUDA device");
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t ntiles = (nevents + kUwTile - 1) / kUwTile;
    cudaError_t err = cudaSuccess;
    if (!s->wmax) {
        if (cudaMalloc(&s->wmax, 2 * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMallocHost(&s->h, 2 * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return fail(HYDRA_ERR_OOM, "unweighting scratch");
        }
    }
    if (ntiles > s->cap) {
        if (s->counts) cudaFree(s->counts);
        if (s->offsets) cudaFree(s->offsets);
        if (s->masks) cudaFree(s->masks);
        s->counts = nullptr;
        s->offsets = nullptr;
        s->masks = nullptr;
        s->cap = 0;
        if (cudaMalloc(&s->counts, ntiles * sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&s->offsets, ntiles * sizeof(uint64_t)) != cudaSuccess ||
            cudaMalloc(&s->masks, ntiles * kUwBlock * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return fail(HYDRA_ERR_OOM, "unweighting scratch for %llu tiles", static_cast<unsigned long long>(ntiles));
        }
        s->cap = ntiles;
    }
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long bits = 0;
    if (w_max > 0.0) {
        if (dtype == HYDRA_F32) {
            const float f = static_cast<float>(w_max);
            std::memcpy(&bits, &f, 4);
        } else {
            std::memcpy(&bits, &w_max, 8);
        }
        err = cudaMemcpyAsync(s->wmax, &bits, sizeof bits, cudaMemcpyHostToDevice, cs);
    } else {
        err = cudaMemsetAsync(s->wmax, 0, sizeof(unsigned long long), cs);
        if (err == cudaSuccess) {
            int dev = 0, sms = 148;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (dtype == HYDRA_F32)
                unweight_max<float><<<sms * 8, kUwBlock, 0, cs>>>(static_cast<const float*>(weights), nevents, s->wmax);
            else
                unweight_max<double><<<sms * 8, kUwBlock, 0, cs>>>(static_cast<const double*>(weights), nevents, s->wmax);
            err = cudaGetLastError();
        }
    }
    if (err != cudaSuccess) return cuda_fail(err, "unweighting max");
    const unsigned grid = static_cast<unsigned>(ntiles);
    if (dtype == HYDRA_F32) {
        unweight_count<float><<<grid, kUwBlock, 0, cs>>>(C, draw, static_cast<const float*>(weights), nevents, event_offset, s->wmax, s->counts, s->masks);
    } else {
        unweight_count<double><<<grid, kUwBlock, 0, cs>>>(C, draw, static_cast<const double*>(weights), nevents, event_offset, s->wmax, s->counts, s->masks);
    }
    unweight_scan<<<1, 1024, 0, cs>>>(s->counts, ntiles, s->offsets, reinterpret_cast<uint64_t*>(s->wmax + 1));
    unweight_write<<<grid, kUwBlock, 0, cs>>>(s->masks, s->offsets, indices);
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaMemcpyAsync(s->h, s->wmax, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, cs);
    if (err == cudaSuccess) err = cudaStreamSynchronize(cs);
    if (err != cudaSuccess) return cuda_fail(err, "unweighting");
    *naccepted = s->h[1];
    if (w_max_used) {
        if (dtype == HYDRA_F32) {
            float f;
            const uint32_t b32 = static_cast<uint32_t>(s->h[0]);
            std::memcpy(&f, &b32, 4);
            *w_max_used = f;
        } else {
            std::memcpy(w_max_used, &s->h[0], 8);
        }
    }
    return HYDRA_OK;
}

hydra_status hydra_phsp_evaluate(int n, uint64_t nevents, hydra_dtype dtype, hydra_me_id me, const double* params,
                                 int nparams, const void* events, uint64_t ld, const void* weights, void* values,
                                 hydra_integral* result, hydra_stream_t stream) {
    const NvtxRange nvtx_range("hydra_phsp_evaluate");
    if (n < 2 || n > kNMax) return fail(HYDRA_ERR_UNSUPPORTED_N, "n = %d outside [2, %d]", n, kNMax);
    if (dtype != HYDRA_F32 && dtype != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(dtype));
    if (!result) return fail(HYDRA_ERR_INVALID_ARG, "result is NULL");
    if (nevents == 0) return fail(HYDRA_ERR_INVALID_ARG, "nevents must be > 0");
    if (!weights || (me != HYDRA_ME_FLAT && !events)) return fail(HYDRA_ERR_INVALID_ARG, "NULL events or weights");
    if (events && ld < nevents) return fail(HYDRA_ERR_INVALID_ARG, "ld < nevents");
    MEConsts P;
    hydra_status st = make_me(me, n, params, nparams, &P);
    if (st != HYDRA_OK) return st;
    EvalScratch* s = eval_scratch();
    if (!s) return fail(HYDRA_ERR_CUDA, "no current CUDA device");
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t ntiles = (nevents + kTileEvents - 1) / kTileEvents;
    const uint64_t nseg = (ntiles + kSegTiles - 1) / kSegTiles;
    if (!s->tiles) {
        if (cudaMalloc(&s->tiles, kChunkTiles * sizeof(TileSums)) != cudaSuccess ||
            cudaMalloc(&s->d_res, sizeof(hydra_integral)) != cudaSuccess ||
            cudaMallocHost(&s->h_res, sizeof(hydra_integral)) != cudaSuccess) {
            cudaGetLastError();
            return fail(HYDRA_ERR_OOM, "evaluation scratch");
        }
    }
    if (nseg > s->seg_cap) {
        if (s->segs) cudaFree(s->segs);
        s->segs = nullptr;
        s->seg_cap = 0;
        if (cudaMalloc(&s->segs, nseg * 8 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(HYDRA_ERR_OOM, "evaluation segment scratch");
        }
        s->seg_cap = nseg;
    }
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // 16-byte loads when every array is 16-byte aligned and ld a multiple of the vector width
    const uint64_t width = dtype == HYDRA_F32 ? 4 : 2;
    const bool vec = (reinterpret_cast<uintptr_t>(weights) % 16 == 0) &&
                     (!values || reinterpret_cast<uintptr_t>(values) % 16 == 0) &&
                     (!events || (reinterpret_cast<uintptr_t>(events) % 16 == 0 && ld % width == 0));
    // FP64 events: |ME|^2 in double-float unless native FP64 arithmetic is selected
    const bool native = g_fp64_arith.load() == HYDRA_FP64_NATIVE;
    const bool dalitz = me == HYDRA_ME_DALITZ_2BW;
    const void* kern = nullptr;
    if (dtype == HYDRA_F32) {
        if (vec) kern = dalitz ? reinterpret_cast<const void*>(&evaluate_tiles_vec<float, HYDRA_ME_DALITZ_2BW, float>)
                               : reinterpret_cast<const void*>(&evaluate_tiles_vec<float, HYDRA_ME_FLAT, float>);
        else kern = dalitz ? reinterpret_cast<const void*>(&evaluate_tiles<float, HYDRA_ME_DALITZ_2BW, float>)
                           : reinterpret_cast<const void*>(&evaluate_tiles<float, HYDRA_ME_FLAT, float>);
    } else if (!dalitz) {
        kern = vec ? reinterpret_cast<const void*>(&evaluate_tiles_vec<double, HYDRA_ME_FLAT, double>)
                   : reinterpret_cast<const void*>(&evaluate_tiles<double, HYDRA_ME_FLAT, double>);
    } else if (native) {
        kern = vec ? reinterpret_cast<const void*>(&evaluate_tiles_vec<double, HYDRA_ME_DALITZ_2BW, double>)
                   : reinterpret_cast<const void*>(&evaluate_tiles<double, HYDRA_ME_DALITZ_2BW, double>);
    } else {
        kern = vec ? reinterpret_cast<const void*>(&evaluate_tiles_vec<double, HYDRA_ME_DALITZ_2BW, df>)
                   : reinterpret_cast<const void*>(&evaluate_tiles<double, HYDRA_ME_DALITZ_2BW, df>);
    }
    for (uint64_t t0 = 0; t0 < ntiles; t0 += kChunkTiles) {
        const uint64_t nt = ntiles - t0 < kChunkTiles ? ntiles - t0 : kChunkTiles;
        const uint64_t need = (nt * 32 + 255) / 256;
        const unsigned grid = static_cast<unsigned>(need < static_cast<uint64_t>(sms) * 8 ? need : static_cast<uint64_t>(sms) * 8);
        uint64_t nev = nevents, ldv = ld, tb = t0, ntv = nt;
        const void* evp = events;
        const void* wp = weights;
        void* vp = values;
        TileSums* tp = s->tiles;
        void* args[] = {&nev, const_cast<void**>(&evp), &ldv, const_cast<void**>(&wp), &P, &vp, &tb, &ntv, &tp};
        const cudaError_t lerr = cudaLaunchKernel(kern, dim3(grid), dim3(256), args, 0, cs);
        if (lerr != cudaSuccess) return cuda_fail(lerr, "evaluate launch");
        const uint64_t ns = (nt + kSegTiles - 1) / kSegTiles;
        eval_reduce_segments<<<static_cast<unsigned>(ns), kSegBlock, 0, cs>>>(s->tiles, nt, t0 / kSegTiles, s->segs);
    }
    eval_finalize<<<1, 32, 0, cs>>>(s->segs, nseg, nevents, s->d_res);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaMemcpyAsync(s->h_res, s->d_res, sizeof(hydra_integral), cudaMemcpyDeviceToHost, cs);
    if (err == cudaSuccess) err = cudaStreamSynchronize(cs);
    if (err != cudaSuccess) return cuda_fail(err, "evaluate");
    *result = *s->h_res;
    return HYDRA_OK;
}

hydra_status hydra_phsp_gather(int n, hydra_dtype dtype, const void* src, uint64_t src_ld, const void* src_weights,
                               const int64_t* indices, uint64_t count, void* dst, uint64_t dst_ld, void* dst_weights,
                               hydra_stream_t stream) {
    const NvtxRange nvtx_range("hydra_phsp_gather");
    if (n < 2 || n > kNMax) return fail(HYDRA_ERR_UNSUPPORTED_N, "n = %d outside [2, %d]", n, kNMax);
    if (dtype != HYDRA_F32 && dtype != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(dtype));
    if (count == 0) return HYDRA_OK;
    if (!src || !indices || !dst) return fail(HYDRA_ERR_INVALID_ARG, "NULL buffer");
    if (dst_ld < count) return fail(HYDRA_ERR_INVALID_ARG, "dst_ld < count");
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t need = (count + 255) / 256;
    const unsigned grid = static_cast<unsigned>(need < static_cast<uint64_t>(sms) * 8 ? need : static_cast<uint64_t>(sms) * 8);
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (dtype == HYDRA_F32)
        gather_events<float><<<grid, 256, 0, cs>>>(4 * n, static_cast<const float*>(src), src_ld, static_cast<const float*>(src_weights),
                                                   indices, count, static_cast<float*>(dst), dst_ld, static_cast<float*>(dst_weights));
    else
        gather_events<double><<<grid, 256, 0, cs>>>(4 * n, static_cast<const double*>(src), src_ld, static_cast<const double*>(src_weights),
                                                    indices, count, static_cast<double*>(dst), dst_ld, static_cast<double*>(dst_weights));
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "gather launch");
    return HYDRA_OK;
}

}  // extern "C"
