// phsp.cu -- kernels and C ABI of the B300 phase-space Monte Carlo library.
//
// Hot path of Hydra section 4.2 (Raubold-Lynch phase-space generation with weighted
// events) and of the phase-space MC integral (section 3), written for sm_103a:
//   phsp_generate_kernel<N, R>       one event per thread, grid-stride; every output
//                                    component is one fully coalesced warp store into the
//                                    structure-of-arrays buffer [n][4][ld].
//   phsp_integrate_tiles<N, R, ME>   one warp per tile of 2048 events; the kinematics stay
//                                    in registers; the tile's sums of (f, f^2, w, w^2) are
//                                    formed in a fixed order and written as FP64.
//   reduce_segments / finalize_integral   FP64 compensated (Neumaier / TwoSum) sums over
//                                    tiles, then segments, in fixed trees over the event
//                                    index, so an integral is bit-identical at every launch
//                                    shape and chunking.
// The C ABI is declared in include/hydra_phsp.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <type_traits>
#include <mutex>
#include <string>
#include <vector>

#include "hydra_phsp.h"
#include "phsp_device.cuh"
#include "phsp_host.h"
#include "phsp_integral.cuh"

namespace hydra {

// ------------------------------------------------------------------------------------
// Generation
// ------------------------------------------------------------------------------------
// Thread t takes the group of EPT consecutive events g*EPT.. (grid-stride over groups); the
// last nevents % EPT events are taken one each by the first threads of the grid.  R is the
// kinematic arithmetic (float, double, or df = pairs of floats for FP64 outputs).
template <int N, typename R, int EPT, bool kMassless = false, bool kLambda64 = false>
__global__ void __launch_bounds__(512) phsp_generate_kernel(const __grid_constant__ DecayConsts C,
                                                            uint64_t nevents, uint64_t event_offset,
                                                            typename Prec<R>::Out* __restrict__ out,
                                                            uint64_t ld,
                                                            typename Prec<R>::Out* __restrict__ weights) {
    if constexpr (std::is_same<R, df>::value) {
        df_sincos_table_init();
        __syncthreads();
    }
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t groups = nevents / EPT;
    for (uint64_t g = tid; g < groups; g += stride) {
        const uint64_t e0 = g * EPT;
        uint64_t ev[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) ev[q] = event_offset + e0 + q;
        StoreSink<R, EPT> sink{out + e0, weights + e0, ld};
        raubold_lynch_group<N, R, EPT, kMassless, kLambda64>(C, ev, sink);
    }
    if constexpr (EPT > 1) {
        const uint64_t e = groups * EPT + tid;
        if (e < nevents) {
            uint64_t ev[1] = {event_offset + e};
            StoreSink<R, 1> sink{out + e, weights + e, ld};
            raubold_lynch_group<N, R, 1, kMassless, kLambda64>(C, ev, sink);
        }
    }
}

// The 3n-4 raw Philox draws of each event, structure of arrays out[d * ld + e].
template <int N>
__global__ void __launch_bounds__(256) phsp_draws_kernel(const __grid_constant__ DecayConsts C,
                                                         uint64_t nevents, uint64_t event_offset,
                                                         uint32_t* __restrict__ out, uint64_t ld) {
    constexpr int kDraws = 3 * N - 4;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t e = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < nevents;
         e += stride) {
        const uint64_t ev = event_offset + e;
        uint32_t x[4];
#pragma unroll
        for (int d = 0; d < kDraws; ++d) {
            if (d % 4 == 0)
                philox4x32_10(static_cast<uint32_t>(ev), static_cast<uint32_t>(ev >> 32), d / 4, 0u,
                              C.rk0, C.rk1, x);
            out[static_cast<uint64_t>(d) * ld + e] = x[d % 4];
        }
    }
}

// ------------------------------------------------------------------------------------
// Integration: f = w |ME|^2
// ------------------------------------------------------------------------------------
// One warp per tile of kTileEvents events (the tile sums are in tile_sums()).
template <int N, typename R, int ME, int EPT>
__global__ void __launch_bounds__(512) phsp_integrate_tiles(const __grid_constant__ DecayConsts C,
                                                            const __grid_constant__ MEConsts P,
                                                            uint64_t nevents, uint64_t event_offset,
                                                            uint64_t tile_begin, uint64_t ntiles,
                                                            TileSums* __restrict__ partials) {
    if constexpr (std::is_same<R, df>::value) {
        df_sincos_table_init();
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t t = warp; t < ntiles; t += nwarps) {
        const TileSums ts = tile_sums<N, R, ME, EPT>(C, P, nevents, event_offset, tile_begin + t, lane);
        if (lane == 0) partials[t] = ts;
    }
}

// Segment partials: 8 doubles per segment, (s, c) for f, f^2, w, w^2.
// One block per segment of kSegTiles tiles (segment_sums_block in phsp_integral.cuh).
__global__ void __launch_bounds__(kSegBlock) reduce_segments(const TileSums* __restrict__ partials,
                                                             uint64_t ntiles, uint64_t seg_begin,
                                                             double* __restrict__ seg_out) {
    const uint64_t seg = blockIdx.x;
    const uint64_t t0 = seg * kSegTiles;
    const uint64_t nt = ntiles - t0 < kSegTiles ? ntiles - t0 : kSegTiles;
    segment_sums_block(partials + t0, nt, seg_out + (seg_begin + seg) * 8);
}

// One warp folds all segments and writes the result.
__global__ void __launch_bounds__(32) finalize_integral(const double* __restrict__ seg,
                                                        uint64_t nseg, uint64_t nevents,
                                                        hydra_integral* __restrict__ out) {
    fold_segments(seg, nseg, nevents, threadIdx.x & 31, out);
}

// ------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------
thread_local std::string g_last_error;

hydra_status fail(hydra_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

hydra_status cuda_fail(cudaError_t err, const char* what) {
    return fail(HYDRA_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(err), cudaGetErrorString(err));
}

// Validates a decay and fills the launch constants.  T = M - sum m in FP64.
hydra_status make_consts(double M, int n, const double* masses, uint64_t seed,
                                DecayConsts* C) {
    if (n < 2 || n > kNMax) return fail(HYDRA_ERR_UNSUPPORTED_N, "n = %d outside [2, %d]", n, kNMax);
    if (!masses) return fail(HYDRA_ERR_INVALID_ARG, "masses is NULL");
    if (!std::isfinite(M) || !(M > 0.0)) return fail(HYDRA_ERR_INVALID_ARG, "parent mass M = %g must be finite and > 0", M);
    std::memset(C, 0, sizeof *C);
    double sum = 0.0;
    for (int i = 0; i < n; ++i) {
        const double m = masses[i];
        if (!std::isfinite(m) || !(m >= 0.0))
            return fail(HYDRA_ERR_INVALID_ARG, "daughter mass %d = %g must be finite and >= 0", i, m);
        sum += m;
        C->m[i] = m;
        C->mu[i] = sum;
        C->m2[i] = m * m;
        C->tm[i] = 2.0 * m;
        if (m == 0.0) C->massless |= 1u << i;
    }
    const double T = M - sum;
    if (!(T > 0.0))
        return fail(HYDRA_ERR_BELOW_THRESHOLD, "sum of daughter masses %.17g >= M = %.17g", sum, M);
    // C_n = pi^(n-1) 2^(n-2) T^(n-2) / ((n-2)! M)
    double Cn = 1.0;
    for (int i = 0; i < n - 1; ++i) Cn *= M_PI;
    for (int i = 0; i < n - 2; ++i) Cn *= 2.0 * T;
    for (int i = 2; i <= n - 2; ++i) Cn /= static_cast<double>(i);
    Cn /= M;
    C->M = M;
    C->Ts = std::ldexp(T, -32);
    C->Ts_half = std::ldexp(T, -33);
    C->C = Cn;
    C->Mf = static_cast<float>(M);
    C->Tsf = static_cast<float>(C->Ts);
    C->Ts_halff = static_cast<float>(C->Ts_half);
    C->Cf = static_cast<float>(Cn);
    C->invM = 1.0 / M;
    C->halfInvM = 0.5 / M;
    C->invMf = static_cast<float>(C->invM);
    C->halfInvMf = static_cast<float>(C->halfInvM);
    C->Mm1 = M * M + masses[0] * masses[0];
    C->Mm1f = static_cast<float>(C->Mm1);
    auto split = [](double v, float* o) {
        o[0] = static_cast<float>(v);
        o[1] = static_cast<float>(v - static_cast<double>(o[0]));
    };
    split(M, C->Mdf);
    split(C->invM, C->invMdf);
    split(C->halfInvM, C->halfInvMdf);
    split(C->Mm1, C->Mm1df);
    split(C->Ts, C->Tsdf);
    split(C->Ts_half, C->Ts_halfdf);
    for (int i = 0; i < n; ++i) {
        split(C->m[i], C->mdf[i]);
        split(C->mu[i], C->mudf[i]);
        split(C->m2[i], C->m2df[i]);
        split(C->tm[i], C->tmdf[i]);
    }
    for (int i = 0; i < n; ++i) {
        C->mf[i] = static_cast<float>(C->m[i]);
        C->muf[i] = static_cast<float>(C->mu[i]);
        C->m2f[i] = static_cast<float>(C->m2[i]);
        C->tmf[i] = static_cast<float>(C->tm[i]);
    }
    uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        C->rk0[r] = k0;
        C->rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return HYDRA_OK;
}

// Grid size for a grid-stride kernel: resident blocks per SM x SM count.
int grid_for(const void* kernel, int block, uint64_t work_items) {
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
    if (per_sm < 1) per_sm = 1;
    const uint64_t full = static_cast<uint64_t>(sms) * per_sm;
    const uint64_t need = (work_items + block - 1) / block;
    return static_cast<int>(need < full ? (need ? need : 1) : full);
}

// ------------------------------------------------------------------------------------
// Kernel selection and launch configuration (block size, events per thread), settable per
// (kernel kind, n, dtype) through hydra_set_launch_config; the autotuner uses that.
// ------------------------------------------------------------------------------------
struct Launch {
    const void* kern;
    int block;
    int ept;
};

template <typename R, int EPT, bool M0, bool L64 = false>
static const void* generate_kernel_n(int n) {
    switch (n) {
        case 2: return reinterpret_cast<const void*>(&phsp_generate_kernel<2, R, EPT, M0, L64>);
        case 3: return reinterpret_cast<const void*>(&phsp_generate_kernel<3, R, EPT, M0, L64>);
        case 4: return reinterpret_cast<const void*>(&phsp_generate_kernel<4, R, EPT, M0, L64>);
        case 5: return reinterpret_cast<const void*>(&phsp_generate_kernel<5, R, EPT, M0, L64>);
        case 6: return reinterpret_cast<const void*>(&phsp_generate_kernel<6, R, EPT, M0, L64>);
        case 7: return reinterpret_cast<const void*>(&phsp_generate_kernel<7, R, EPT, M0, L64>);
        case 8: return reinterpret_cast<const void*>(&phsp_generate_kernel<8, R, EPT, M0, L64>);
        case 9: return reinterpret_cast<const void*>(&phsp_generate_kernel<9, R, EPT, M0, L64>);
        case 10: return reinterpret_cast<const void*>(&phsp_generate_kernel<10, R, EPT, M0, L64>);
    }
    return nullptr;
}

// FP32 generation with the lambda product in FP64 (hydra_set_fp32_lambda)
static const void* generate_kernel_f32_lambda64(int n, int ept) {
    switch (ept) {
        case 1: return generate_kernel_n<float, 1, false, true>(n);
        case 2: return generate_kernel_n<float, 2, false, true>(n);
        case 4: return generate_kernel_n<float, 4, false, true>(n);
    }
    return nullptr;
}

// massless: every daughter has mass 0 (the double-float generator has a variant for that case;
// it saves the square root of every two-body momentum, 7-10% of its time)
template <typename R>
static const void* generate_kernel_for(int n, int ept, bool massless) {
    constexpr bool kHasMassless = std::is_same<R, df>::value;
    if (kHasMassless && massless) {
        switch (ept) {
            case 1: return generate_kernel_n<R, 1, kHasMassless>(n);
            case 2: return generate_kernel_n<R, 2, kHasMassless>(n);
            case 4: return generate_kernel_n<R, 4, kHasMassless>(n);
        }
        return nullptr;
    }
    switch (ept) {
        case 1: return generate_kernel_n<R, 1, false>(n);
        case 2: return generate_kernel_n<R, 2, false>(n);
        case 4: return generate_kernel_n<R, 4, false>(n);
    }
    return nullptr;
}

static const void* draws_kernel_for(int n) {
    switch (n) {
        case 2: return reinterpret_cast<const void*>(&phsp_draws_kernel<2>);
        case 3: return reinterpret_cast<const void*>(&phsp_draws_kernel<3>);
        case 4: return reinterpret_cast<const void*>(&phsp_draws_kernel<4>);
        case 5: return reinterpret_cast<const void*>(&phsp_draws_kernel<5>);
        case 6: return reinterpret_cast<const void*>(&phsp_draws_kernel<6>);
        case 7: return reinterpret_cast<const void*>(&phsp_draws_kernel<7>);
        case 8: return reinterpret_cast<const void*>(&phsp_draws_kernel<8>);
        case 9: return reinterpret_cast<const void*>(&phsp_draws_kernel<9>);
        case 10: return reinterpret_cast<const void*>(&phsp_draws_kernel<10>);
    }
    return nullptr;
}

template <typename R, int ME, int EPT>
static const void* integrate_kernel_n(int n) {
    if constexpr (ME == HYDRA_ME_DALITZ_2BW) {
        return n == 3 ? reinterpret_cast<const void*>(&phsp_integrate_tiles<3, R, ME, EPT>) : nullptr;
    } else {
        switch (n) {
            case 2: return reinterpret_cast<const void*>(&phsp_integrate_tiles<2, R, ME, EPT>);
            case 3: return reinterpret_cast<const void*>(&phsp_integrate_tiles<3, R, ME, EPT>);
            case 4: return reinterpret_cast<const void*>(&phsp_integrate_tiles<4, R, ME, EPT>);
            case 5: return reinterpret_cast<const void*>(&phsp_integrate_tiles<5, R, ME, EPT>);
            case 6: return reinterpret_cast<const void*>(&phsp_integrate_tiles<6, R, ME, EPT>);
            case 7: return reinterpret_cast<const void*>(&phsp_integrate_tiles<7, R, ME, EPT>);
            case 8: return reinterpret_cast<const void*>(&phsp_integrate_tiles<8, R, ME, EPT>);
            case 9: return reinterpret_cast<const void*>(&phsp_integrate_tiles<9, R, ME, EPT>);
            case 10: return reinterpret_cast<const void*>(&phsp_integrate_tiles<10, R, ME, EPT>);
        }
        return nullptr;
    }
}

template <typename R, int ME>
static const void* integrate_kernel_for(int n, int ept) {
    switch (ept) {
        case 1: return integrate_kernel_n<R, ME, 1>(n);
        case 2: return integrate_kernel_n<R, ME, 2>(n);
        case 4: return integrate_kernel_n<R, ME, 4>(n);
    }
    return nullptr;
}

// Launch configuration table [kind][dtype][n] = block size and events per thread.  The
// defaults are the measured best on B300 (see the tuning notes); hydra_set_launch_config
// overrides them for the process.
struct LaunchCfg {
    std::atomic<int> block{256};
    std::atomic<int> ept{1};
};
static LaunchCfg g_cfg[2][2][kNMax + 1];

std::atomic<int> g_fp64_arith{HYDRA_FP64_DOUBLE_FLOAT};
std::atomic<int> g_fp32_lambda{HYDRA_LAMBDA_FACTORED_F32};

static Launch select_generate(hydra_dtype dtype, int n, const DecayConsts& C) {
    LaunchCfg& c = g_cfg[HYDRA_KERNEL_GENERATE][dtype][n];
    const int ept = c.ept.load(std::memory_order_relaxed);
    const bool massless = C.massless == (1u << n) - 1u;
    const void* k = nullptr;
    if (dtype == HYDRA_F32)
        k = g_fp32_lambda.load(std::memory_order_relaxed) == HYDRA_LAMBDA_F64 ? generate_kernel_f32_lambda64(n, ept)
                                                                               : generate_kernel_for<float>(n, ept, massless);
    else if (g_fp64_arith.load(std::memory_order_relaxed) == HYDRA_FP64_NATIVE) k = generate_kernel_for<double>(n, ept, massless);
    else k = generate_kernel_for<df>(n, ept, massless);
    return Launch{k, c.block.load(std::memory_order_relaxed), ept};
}

static Launch select_integrate(hydra_dtype dtype, hydra_me_id me, int n) {
    LaunchCfg& c = g_cfg[HYDRA_KERNEL_INTEGRATE][dtype][n];
    const int ept = c.ept.load(std::memory_order_relaxed);
    const void* k = nullptr;
    if (dtype == HYDRA_F32)
        k = me == HYDRA_ME_FLAT ? integrate_kernel_for<float, HYDRA_ME_FLAT>(n, ept)
                                : integrate_kernel_for<float, HYDRA_ME_DALITZ_2BW>(n, ept);
    else if (g_fp64_arith.load() == HYDRA_FP64_NATIVE)
        k = me == HYDRA_ME_FLAT ? integrate_kernel_for<double, HYDRA_ME_FLAT>(n, ept)
                                : integrate_kernel_for<double, HYDRA_ME_DALITZ_2BW>(n, ept);
    else
        k = me == HYDRA_ME_FLAT ? integrate_kernel_for<df, HYDRA_ME_FLAT>(n, ept)
                                : integrate_kernel_for<df, HYDRA_ME_DALITZ_2BW>(n, ept);
    return Launch{k, c.block.load(std::memory_order_relaxed), ept};
}

constexpr int kGenBlock = 256;  // the raw-draws kernel

// Per-device scratch for integrals: tile partials of one chunk, segment partials of one
// request, the device-side result and a pinned host copy.  Guarded by its mutex.
struct DeviceScratch {
    std::mutex mu;
    TileSums* tiles = nullptr;
    double* segs = nullptr;
    uint64_t seg_cap = 0;  // segments
    hydra_integral* d_result = nullptr;
    hydra_integral* h_result = nullptr;
    // host-output generation: two device staging buffers, a copy stream and events
    void* stage[2] = {nullptr, nullptr};
    size_t stage_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t gen_done[2] = {nullptr, nullptr};
    cudaEvent_t copy_done[2] = {nullptr, nullptr};
};

static std::mutex g_scratch_mu;
static std::vector<DeviceScratch*> g_scratch;

static DeviceScratch* scratch_for_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (static_cast<int>(g_scratch.size()) <= dev) g_scratch.resize(dev + 1, nullptr);
    if (!g_scratch[dev]) g_scratch[dev] = new DeviceScratch();
    return g_scratch[dev];
}

static hydra_status ensure_scratch(DeviceScratch* s, uint64_t nseg) {
    if (!s->tiles) {
        if (cudaMalloc(&s->tiles, kChunkTiles * sizeof(TileSums)) != cudaSuccess) {
            s->tiles = nullptr;
            cudaGetLastError();
            return fail(HYDRA_ERR_OOM, "cannot allocate %zu bytes of tile scratch",
                        static_cast<size_t>(kChunkTiles * sizeof(TileSums)));
        }
    }
    if (!s->d_result) {
        if (cudaMalloc(&s->d_result, sizeof(hydra_integral)) != cudaSuccess ||
            cudaMallocHost(&s->h_result, sizeof(hydra_integral)) != cudaSuccess) {
            cudaGetLastError();
            return fail(HYDRA_ERR_OOM, "cannot allocate the integral result buffers");
        }
    }
    if (nseg > s->seg_cap) {
        uint64_t cap = s->seg_cap ? s->seg_cap : 64;
        while (cap < nseg) cap *= 2;
        double* p = nullptr;
        if (cudaMalloc(&p, cap * 8 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(HYDRA_ERR_OOM, "cannot allocate segment scratch for %llu segments",
                        static_cast<unsigned long long>(nseg));
        }
        if (s->segs) cudaFree(s->segs);
        s->segs = p;
        s->seg_cap = cap;
    }
    return HYDRA_OK;
}

// Events per staging chunk of hydra_phsp_generate_host (a multiple of 4).
constexpr uint64_t kStageEvents = uint64_t(1) << 22;

static hydra_status ensure_staging(DeviceScratch* s, size_t bytes) {
    if (!s->copy_stream) {
        if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            s->copy_stream = nullptr;
            return fail(HYDRA_ERR_CUDA, "cannot create the copy stream");
        }
        for (int b = 0; b < 2; ++b) {
            if (cudaEventCreateWithFlags(&s->gen_done[b], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&s->copy_done[b], cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                return fail(HYDRA_ERR_CUDA, "cannot create staging events");
            }
        }
    }
    if (bytes > s->stage_bytes) {
        for (int b = 0; b < 2; ++b) {
            if (s->stage[b]) cudaFree(s->stage[b]);
            s->stage[b] = nullptr;
        }
        s->stage_bytes = 0;
        for (int b = 0; b < 2; ++b) {
            if (cudaMalloc(&s->stage[b], bytes) != cudaSuccess) {
                cudaGetLastError();
                return fail(HYDRA_ERR_OOM, "cannot allocate %zu bytes of staging memory", bytes);
            }
        }
        s->stage_bytes = bytes;
    }
    return HYDRA_OK;
}

hydra_status make_me(hydra_me_id me, int n, const double* params, int nparams, MEConsts* P) {
    std::memset(P, 0, sizeof *P);
    if (me == HYDRA_ME_FLAT) return HYDRA_OK;
    if (me != HYDRA_ME_DALITZ_2BW) return fail(HYDRA_ERR_INVALID_ARG, "unknown matrix element id %d", static_cast<int>(me));
    if (n != 3) return fail(HYDRA_ERR_UNSUPPORTED_N, "the Dalitz matrix element needs n = 3 (got %d)", n);
    if (!params || nparams < 6) return fail(HYDRA_ERR_INVALID_ARG, "the Dalitz matrix element needs 6 params (got %d)", nparams);
    for (int i = 0; i < 6; ++i)
        if (!std::isfinite(params[i])) return fail(HYDRA_ERR_INVALID_ARG, "param %d is not finite", i);
    P->a_m2 = params[0] * params[0];
    P->a_mg = params[0] * params[1];
    P->b_m2 = params[2] * params[2];
    P->b_mg = params[2] * params[3];
    P->c_re = params[4] * std::cos(params[5]);
    P->c_im = params[4] * std::sin(params[5]);
    P->a_m2f = static_cast<float>(P->a_m2);
    P->a_mgf = static_cast<float>(P->a_mg);
    P->b_m2f = static_cast<float>(P->b_m2);
    P->b_mgf = static_cast<float>(P->b_mg);
    P->c_ref = static_cast<float>(P->c_re);
    P->c_imf = static_cast<float>(P->c_im);
    // low parts of the double-float parameters: hi + lo = the FP64 value to ~2^-48
    P->a_m2lo = static_cast<float>(P->a_m2 - static_cast<double>(P->a_m2f));
    P->a_mglo = static_cast<float>(P->a_mg - static_cast<double>(P->a_mgf));
    P->b_m2lo = static_cast<float>(P->b_m2 - static_cast<double>(P->b_m2f));
    P->b_mglo = static_cast<float>(P->b_mg - static_cast<double>(P->b_mgf));
    P->c_relo = static_cast<float>(P->c_re - static_cast<double>(P->c_ref));
    P->c_imlo = static_cast<float>(P->c_im - static_cast<double>(P->c_imf));
    return HYDRA_OK;
}

static hydra_status launch_integrate_chunks(const Launch& L, const DecayConsts& C, const MEConsts& P,
                                            uint64_t nevents, uint64_t event_offset,
                                            DeviceScratch* s, cudaStream_t st) {
    const uint64_t ntiles = (nevents + kTileEvents - 1) / kTileEvents;
    for (uint64_t t0 = 0; t0 < ntiles; t0 += kChunkTiles) {
        const uint64_t nt = ntiles - t0 < kChunkTiles ? ntiles - t0 : kChunkTiles;
        const int grid = grid_for(L.kern, L.block, nt * 32);
        TileSums* tiles = s->tiles;
        void* args[] = {const_cast<DecayConsts*>(&C), const_cast<MEConsts*>(&P), &nevents,
                        &event_offset, const_cast<uint64_t*>(&t0), const_cast<uint64_t*>(&nt),
                        &tiles};
        cudaError_t err = cudaLaunchKernel(L.kern, dim3(grid), dim3(L.block), args, 0, st);
        if (err != cudaSuccess) return cuda_fail(err, "integrate launch");
        const uint64_t nseg = (nt + kSegTiles - 1) / kSegTiles;
        const uint64_t seg_begin = t0 / kSegTiles;
        reduce_segments<<<static_cast<unsigned>(nseg), kSegBlock, 0, st>>>(s->tiles, nt, seg_begin, s->segs);
        err = cudaGetLastError();
        if (err != cudaSuccess) return cuda_fail(err, "segment reduction launch");
    }
    return HYDRA_OK;
}

// ------------------------------------------------------------------------------------
// Integral without allocation: the scratch of hydra_phsp_integrate_noalloc lives in one
// file-scope device array, present on every device that loads this library until the
// process exits.  Layout: [tile partials of one chunk | segment partials | result].
// ------------------------------------------------------------------------------------
constexpr uint64_t kNoAllocMaxEvents = uint64_t(1) << 32;
constexpr uint64_t kNoAllocMaxSegs = kNoAllocMaxEvents / (uint64_t(kTileEvents) * kSegTiles);  // 2048
constexpr size_t kNoAllocTilesBytes = kChunkTiles * sizeof(TileSums);                  // 1 MiB
constexpr size_t kNoAllocSegsBytes = kNoAllocMaxSegs * 8 * sizeof(double);              // 128 KiB
constexpr size_t kNoAllocResultOffset = kNoAllocTilesBytes + kNoAllocSegsBytes;
constexpr size_t kNoAllocBytes = kNoAllocResultOffset + 256;
static_assert(sizeof(hydra_integral) <= 256, "result slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;

// Device address of g_noalloc_scratch on the current device, looked up on every call (the
// host-side name of the array is not a device address; a cached address could outlive the
// context it belongs to, and the lookup is cheap next to the call's own synchronisation).
static hydra_status noalloc_scratch(unsigned char** out) {
    void* ptr = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (err != cudaSuccess) return cuda_fail(err, "cudaGetSymbolAddress(no-allocation scratch)");
    *out = static_cast<unsigned char*>(ptr);
    return HYDRA_OK;
}

}  // namespace hydra

using namespace hydra;

extern "C" {

const char* hydra_last_error(void) { return g_last_error.c_str(); }

const char* hydra_status_string(hydra_status status) {
    switch (status) {
        case HYDRA_OK: return "HYDRA_OK";
        case HYDRA_ERR_INVALID_ARG: return "HYDRA_ERR_INVALID_ARG";
        case HYDRA_ERR_BELOW_THRESHOLD: return "HYDRA_ERR_BELOW_THRESHOLD";
        case HYDRA_ERR_UNSUPPORTED_N: return "HYDRA_ERR_UNSUPPORTED_N";
        case HYDRA_ERR_MISALIGNED: return "HYDRA_ERR_MISALIGNED";
        case HYDRA_ERR_OOM: return "HYDRA_ERR_OOM";
        case HYDRA_ERR_CUDA: return "HYDRA_ERR_CUDA";
        case HYDRA_ERR_TIMEOUT: return "HYDRA_ERR_TIMEOUT";
        case HYDRA_ERR_BUSY: return "HYDRA_ERR_BUSY";
    }
    return "HYDRA_ERR_UNKNOWN";
}

hydra_status hydra_phsp_volume_factor(double M, int n, const double* masses, double* C_n) {
    if (!C_n) return fail(HYDRA_ERR_INVALID_ARG, "C_n is NULL");
    DecayConsts C;
    const hydra_status st = make_consts(M, n, masses, 0, &C);
    if (st != HYDRA_OK) return st;
    *C_n = C.C;
    return HYDRA_OK;
}

hydra_status hydra_phsp_generate(double M, int n, const double* masses, uint64_t nevents,
                                 uint64_t seed, uint64_t event_offset, hydra_dtype dtype,
                                 void* out, uint64_t ld, void* weights, hydra_stream_t stream) {
    const NvtxRange nvtx_range("hydra_phsp_generate");
    DecayConsts C;
    hydra_status st = make_consts(M, n, masses, seed, &C);
    if (st != HYDRA_OK) return st;
    if (dtype != HYDRA_F32 && dtype != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(dtype));
    if (event_offset + nevents < event_offset) return fail(HYDRA_ERR_INVALID_ARG, "event_offset + nevents overflows 64 bits");
    if (nevents == 0) return HYDRA_OK;
    if (!out || !weights) return fail(HYDRA_ERR_INVALID_ARG, "out and weights must not be NULL");
    if (ld < nevents) return fail(HYDRA_ERR_INVALID_ARG, "ld = %llu < nevents = %llu", static_cast<unsigned long long>(ld), static_cast<unsigned long long>(nevents));
    if ((reinterpret_cast<uintptr_t>(out) & 15u) || (reinterpret_cast<uintptr_t>(weights) & 15u))
        return fail(HYDRA_ERR_MISALIGNED, "out and weights must be 16-byte aligned");
    if (ld % 4 != 0) return fail(HYDRA_ERR_MISALIGNED, "ld = %llu must be a multiple of 4", static_cast<unsigned long long>(ld));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const Launch L = select_generate(dtype, n, C);
    const int grid = grid_for(L.kern, L.block, (nevents + L.ept - 1) / L.ept);
    void* args[] = {&C, &nevents, &event_offset, &out, &ld, &weights};
    const cudaError_t err = cudaLaunchKernel(L.kern, dim3(grid), dim3(L.block), args, 0, s);
    if (err != cudaSuccess) return cuda_fail(err, "generate launch");
    return HYDRA_OK;
}

hydra_status hydra_phsp_generate_host(double M, int n, const double* masses, uint64_t nevents,
                                      uint64_t seed, uint64_t event_offset, hydra_dtype dtype,
                                      void* out_host, uint64_t ld, void* weights_host,
                                      hydra_stream_t stream) {
    const NvtxRange nvtx_range("hydra_phsp_generate_host");
    DecayConsts C;
    hydra_status st = make_consts(M, n, masses, seed, &C);
    if (st != HYDRA_OK) return st;
    if (dtype != HYDRA_F32 && dtype != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(dtype));
    if (event_offset + nevents < event_offset) return fail(HYDRA_ERR_INVALID_ARG, "event_offset + nevents overflows 64 bits");
    if (nevents == 0) return HYDRA_OK;
    if (!out_host || !weights_host) return fail(HYDRA_ERR_INVALID_ARG, "out and weights must not be NULL");
    if (ld < nevents) return fail(HYDRA_ERR_INVALID_ARG, "ld = %llu < nevents = %llu", static_cast<unsigned long long>(ld), static_cast<unsigned long long>(nevents));
    const size_t elem = dtype == HYDRA_F32 ? sizeof(float) : sizeof(double);
    const uint64_t chunk = nevents < kStageEvents ? (nevents + 3) / 4 * 4 : kStageEvents;
    const size_t arrays = static_cast<size_t>(4 * n + 1);
    DeviceScratch* s = scratch_for_current_device();
    if (!s) return fail(HYDRA_ERR_CUDA, "no current CUDA device");
    std::lock_guard<std::mutex> lk(s->mu);
    st = ensure_staging(s, arrays * chunk * elem);
    if (st != HYDRA_OK) return st;
    cudaStream_t gs = reinterpret_cast<cudaStream_t>(stream);
    const Launch L = select_generate(dtype, n, C);
    cudaError_t err = cudaSuccess;
    // the copy stream must not run ahead of work already queued on the caller's stream
    err = cudaEventRecord(s->gen_done[1], gs);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(s->copy_stream, s->gen_done[1], 0);
    if (err != cudaSuccess) return cuda_fail(err, "host generate ordering");
    uint64_t i = 0;
    for (uint64_t e0 = 0; e0 < nevents; e0 += chunk, ++i) {
        const int b = static_cast<int>(i & 1);
        const uint64_t cnt = nevents - e0 < chunk ? nevents - e0 : chunk;
        char* stage = static_cast<char*>(s->stage[b]);
        if (i >= 2) {
            err = cudaStreamWaitEvent(gs, s->copy_done[b], 0);  // staging buffer b is free again
            if (err != cudaSuccess) return cuda_fail(err, "staging wait");
        }
        void* dout = stage;
        void* dw = stage + static_cast<size_t>(4 * n) * chunk * elem;
        uint64_t off = event_offset + e0;
        uint64_t sld = chunk;
        uint64_t cnt_v = cnt;
        const int grid = grid_for(L.kern, L.block, (cnt + L.ept - 1) / L.ept);
        void* args[] = {&C, &cnt_v, &off, &dout, &sld, &dw};
        err = cudaLaunchKernel(L.kern, dim3(grid), dim3(L.block), args, 0, gs);
        if (err == cudaSuccess) err = cudaEventRecord(s->gen_done[b], gs);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(s->copy_stream, s->gen_done[b], 0);
        if (err == cudaSuccess)
            err = cudaMemcpy2DAsync(static_cast<char*>(out_host) + e0 * elem, ld * elem, dout, chunk * elem,
                                    cnt * elem, static_cast<size_t>(4 * n), cudaMemcpyDeviceToHost, s->copy_stream);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(static_cast<char*>(weights_host) + e0 * elem, dw, cnt * elem,
                                  cudaMemcpyDeviceToHost, s->copy_stream);
        if (err == cudaSuccess) err = cudaEventRecord(s->copy_done[b], s->copy_stream);
        if (err != cudaSuccess) return cuda_fail(err, "host generate chunk");
    }
    err = cudaStreamSynchronize(s->copy_stream);
    if (err != cudaSuccess) return cuda_fail(err, "host generate synchronize");
    return HYDRA_OK;
}

hydra_status hydra_phsp_draws(int n, uint64_t nevents, uint64_t seed, uint64_t event_offset,
                              uint32_t* out, uint64_t ld, hydra_stream_t stream) {
    const NvtxRange nvtx_range("hydra_phsp_draws");
    if (n < 2 || n > kNMax) return fail(HYDRA_ERR_UNSUPPORTED_N, "n = %d outside [2, %d]", n, kNMax);
    if (event_offset + nevents < event_offset) return fail(HYDRA_ERR_INVALID_ARG, "event_offset + nevents overflows 64 bits");
    if (nevents == 0) return HYDRA_OK;
    if (!out) return fail(HYDRA_ERR_INVALID_ARG, "out must not be NULL");
    if (ld < nevents) return fail(HYDRA_ERR_INVALID_ARG, "ld < nevents");
    DecayConsts C;
    std::memset(&C, 0, sizeof C);
    uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        C.rk0[r] = k0;
        C.rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    const void* kern = draws_kernel_for(n);
    const int grid = grid_for(kern, kGenBlock, nevents);
    void* args[] = {&C, &nevents, &event_offset, &out, &ld};
    const cudaError_t err = cudaLaunchKernel(kern, dim3(grid), dim3(kGenBlock), args, 0,
                                             reinterpret_cast<cudaStream_t>(stream));
    if (err != cudaSuccess) return cuda_fail(err, "draws launch");
    return HYDRA_OK;
}

hydra_status hydra_phsp_integrate(double M, int n, const double* masses, uint64_t nevents,
                                  uint64_t seed, uint64_t event_offset, hydra_dtype kin_dtype,
                                  hydra_me_id me, const double* params, int nparams,
                                  hydra_integral* result, hydra_stream_t stream) {
    const NvtxRange nvtx_range("hydra_phsp_integrate");
    DecayConsts C;
    hydra_status st = make_consts(M, n, masses, seed, &C);
    if (st != HYDRA_OK) return st;
    if (kin_dtype != HYDRA_F32 && kin_dtype != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(kin_dtype));
    if (!result) return fail(HYDRA_ERR_INVALID_ARG, "result is NULL");
    if (nevents == 0) return fail(HYDRA_ERR_INVALID_ARG, "nevents must be > 0");
    if (event_offset + nevents < event_offset) return fail(HYDRA_ERR_INVALID_ARG, "event_offset + nevents overflows 64 bits");
    MEConsts P;
    st = make_me(me, n, params, nparams, &P);
    if (st != HYDRA_OK) return st;
    const Launch L = select_integrate(kin_dtype, me, n);
    if (!L.kern) return fail(HYDRA_ERR_UNSUPPORTED_N, "no kernel for n = %d and me = %d", n, static_cast<int>(me));

    DeviceScratch* s = scratch_for_current_device();
    if (!s) return fail(HYDRA_ERR_CUDA, "no current CUDA device");
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t ntiles = (nevents + kTileEvents - 1) / kTileEvents;
    const uint64_t nseg = (ntiles + kSegTiles - 1) / kSegTiles;
    st = ensure_scratch(s, nseg);
    if (st != HYDRA_OK) return st;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    st = launch_integrate_chunks(L, C, P, nevents, event_offset, s, cs);
    if (st != HYDRA_OK) return st;
    finalize_integral<<<1, 32, 0, cs>>>(s->segs, nseg, nevents, s->d_result);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "finalize launch");
    err = cudaMemcpyAsync(s->h_result, s->d_result, sizeof(hydra_integral), cudaMemcpyDeviceToHost, cs);
    if (err != cudaSuccess) return cuda_fail(err, "result copy");
    err = cudaStreamSynchronize(cs);
    if (err != cudaSuccess) return cuda_fail(err, "integrate synchronize");
    *result = *s->h_result;
    return HYDRA_OK;
}

hydra_status hydra_phsp_integrate_noalloc(double M, int n, const double* masses, uint64_t nevents,
                                          uint64_t seed, uint64_t event_offset, hydra_dtype kin_dtype,
                                          hydra_me_id me, const double* params, int nparams,
                                          hydra_integral* result, hydra_stream_t stream) {
    const NvtxRange nvtx_range("hydra_phsp_integrate_noalloc");
    DecayConsts C;
    hydra_status st = make_consts(M, n, masses, seed, &C);
    if (st != HYDRA_OK) return st;
    if (kin_dtype != HYDRA_F32 && kin_dtype != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(kin_dtype));
    if (!result) return fail(HYDRA_ERR_INVALID_ARG, "result is NULL");
    if (nevents == 0) return fail(HYDRA_ERR_INVALID_ARG, "nevents must be > 0");
    if (nevents > kNoAllocMaxEvents)
        return fail(HYDRA_ERR_INVALID_ARG, "nevents = %llu exceeds the no-allocation limit of 2^32 events "
                    "(its fixed scratch holds 2048 segment partials); use hydra_phsp_integrate",
                    static_cast<unsigned long long>(nevents));
    if (event_offset + nevents < event_offset) return fail(HYDRA_ERR_INVALID_ARG, "event_offset + nevents overflows 64 bits");
    MEConsts P;
    st = make_me(me, n, params, nparams, &P);
    if (st != HYDRA_OK) return st;
    const Launch L = select_integrate(kin_dtype, me, n);
    if (!L.kern) return fail(HYDRA_ERR_UNSUPPORTED_N, "no kernel for n = %d and me = %d", n, static_cast<int>(me));

    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    unsigned char* base = nullptr;
    st = noalloc_scratch(&base);
    if (st != HYDRA_OK) return st;
    // Every tile and segment slot a call reads is written earlier in the same call, and the
    // result slot is overwritten, so nothing needs clearing between calls.
    DeviceScratch view;
    view.tiles = reinterpret_cast<TileSums*>(base);
    view.segs = reinterpret_cast<double*>(base + kNoAllocTilesBytes);
    hydra_integral* d_result = reinterpret_cast<hydra_integral*>(base + kNoAllocResultOffset);
    const uint64_t ntiles = (nevents + kTileEvents - 1) / kTileEvents;
    const uint64_t nseg = (ntiles + kSegTiles - 1) / kSegTiles;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    st = launch_integrate_chunks(L, C, P, nevents, event_offset, &view, cs);
    if (st != HYDRA_OK) return st;
    finalize_integral<<<1, 32, 0, cs>>>(view.segs, nseg, nevents, d_result);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "finalize launch");
    err = cudaMemcpyAsync(result, d_result, sizeof(hydra_integral), cudaMemcpyDeviceToHost, cs);
    if (err != cudaSuccess) return cuda_fail(err, "result copy");
    err = cudaStreamSynchronize(cs);
    if (err != cudaSuccess) return cuda_fail(err, "integrate synchronize");
    return HYDRA_OK;
}

hydra_status hydra_set_launch_config(hydra_kernel_kind kind, int n, hydra_dtype dtype, int block,
                                     int events_per_thread) {
    if (kind != HYDRA_KERNEL_GENERATE && kind != HYDRA_KERNEL_INTEGRATE)
        return fail(HYDRA_ERR_INVALID_ARG, "unknown kernel kind %d", static_cast<int>(kind));
    if (n < 2 || n > kNMax) return fail(HYDRA_ERR_UNSUPPORTED_N, "n = %d outside [2, %d]", n, kNMax);
    if (dtype != HYDRA_F32 && dtype != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(dtype));
    if (block < 32 || block > 512 || block % 32 != 0)
        return fail(HYDRA_ERR_INVALID_ARG, "block = %d must be a multiple of 32 in [32, 512]", block);
    if (events_per_thread != 1 && events_per_thread != 2 && events_per_thread != 4)
        return fail(HYDRA_ERR_INVALID_ARG, "events_per_thread = %d must be 1, 2 or 4", events_per_thread);
    LaunchCfg& c = g_cfg[kind][dtype][n];
    c.block.store(block);
    c.ept.store(events_per_thread);
    return HYDRA_OK;
}

hydra_status hydra_set_fp64_arith(hydra_fp64_arith arith) {
    if (arith != HYDRA_FP64_NATIVE && arith != HYDRA_FP64_DOUBLE_FLOAT)
        return fail(HYDRA_ERR_INVALID_ARG, "unknown FP64 arithmetic %d", static_cast<int>(arith));
    g_fp64_arith.store(arith);
    return HYDRA_OK;
}

hydra_fp64_arith hydra_get_fp64_arith(void) { return static_cast<hydra_fp64_arith>(g_fp64_arith.load()); }

hydra_status hydra_set_fp32_lambda(hydra_lambda_arith arith) {
    if (arith != HYDRA_LAMBDA_FACTORED_F32 && arith != HYDRA_LAMBDA_F64)
        return fail(HYDRA_ERR_INVALID_ARG, "unknown lambda arithmetic %d", static_cast<int>(arith));
    g_fp32_lambda.store(arith);
    return HYDRA_OK;
}

hydra_lambda_arith hydra_get_fp32_lambda(void) { return static_cast<hydra_lambda_arith>(g_fp32_lambda.load()); }

hydra_status hydra_get_launch_config(hydra_kernel_kind kind, int n, hydra_dtype dtype, int* block,
                                     int* events_per_thread) {
    if (kind != HYDRA_KERNEL_GENERATE && kind != HYDRA_KERNEL_INTEGRATE)
        return fail(HYDRA_ERR_INVALID_ARG, "unknown kernel kind %d", static_cast<int>(kind));
    if (n < 2 || n > kNMax) return fail(HYDRA_ERR_UNSUPPORTED_N, "n = %d outside [2, %d]", n, kNMax);
    if (dtype != HYDRA_F32 && dtype != HYDRA_F64) return fail(HYDRA_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(dtype));
    if (!block || !events_per_thread) return fail(HYDRA_ERR_INVALID_ARG, "NULL output");
    const LaunchCfg& c = g_cfg[kind][dtype][n];
    *block = c.block.load();
    *events_per_thread = c.ept.load();
    return HYDRA_OK;
}

hydra_status hydra_shutdown(void) {
    release_extras_scratch();
    release_vegas_scratch();
    release_batch_run_scratch();
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (size_t d = 0; d < g_scratch.size(); ++d) {
        DeviceScratch*& s = g_scratch[d];
        if (!s) continue;
        cudaSetDevice(static_cast<int>(d));
        if (s->tiles) cudaFree(s->tiles);
        if (s->segs) cudaFree(s->segs);
        if (s->d_result) cudaFree(s->d_result);
        if (s->h_result) cudaFreeHost(s->h_result);
        for (int b = 0; b < 2; ++b) {
            if (s->stage[b]) cudaFree(s->stage[b]);
            if (s->gen_done[b]) cudaEventDestroy(s->gen_done[b]);
            if (s->copy_done[b]) cudaEventDestroy(s->copy_done[b]);
        }
        if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
        delete s;
        s = nullptr;
    }
    cudaSetDevice(cur);
    return HYDRA_OK;
}

}  // extern "C"
