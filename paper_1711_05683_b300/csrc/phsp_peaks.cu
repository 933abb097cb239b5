// phsp_peaks.cu -- measured device ceilings for the rooflines the library's kernels are
// reported against: the FP32 and FP64 fused multiply-add rates (independent FMA chains in
// registers, the arithmetic peak and, for FP32, the SM instruction-issue limit: one warp FMA
// per scheduler per clock) and the write-only HBM bandwidth (16-byte stores over a buffer
// larger than L2), plus the rates of the arithmetic the generators actually run (FP32 with the
// hardware square-root and reciprocal approximations, double-float pairs, native FP64) for
// the floating-point ceiling of their rooflines.  Nothing here is part of the phase-space
// method.
#include <cuda_runtime.h>
#include <cstdint>
#include "hydra_phsp.h"
#include "phsp_df.cuh"
#include "phsp_host.h"

namespace hydra {

constexpr int kChains = 8;  // independent FMA chains per thread (covers the 4-cycle latency)

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* __restrict__ sink, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = static_cast<T>(threadIdx.x) * static_cast<T>(1e-3) + static_cast<T>(i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            if constexpr (sizeof(T) == 4) x[i] = __fmaf_rn(x[i], a, b);
            else x[i] = __fma_rn(x[i], a, b);
        }
    }
    T s = x[0];
#pragma unroll
    for (int i = 1; i < kChains; ++i) s += x[i];
    sink[static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

// U 16-byte stores per thread per pass, each warp-wide store 512 contiguous bytes.
template <int U>
__global__ void __launch_bounds__(256) fill16(uint4* __restrict__ p, uint64_t n16, uint32_t v) {
    const uint4 q = make_uint4(v, v, v, v);
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (; i + (U - 1) * stride < n16; i += U * stride) {
#pragma unroll
        for (int u = 0; u < U; ++u) p[i + u * stride] = q;
    }
    for (; i < n16; i += stride) p[i] = q;
}

// One arithmetic operation of the rate probe, in the arithmetic a generator runs: FP32 with
// the hardware approximations of its square root and reciprocal, double-float (phsp_df.cuh,
// the FP64 generator's default), or FP64 instructions.
template <typename T> struct ProbeOps;

template <> struct ProbeOps<float> {
    __device__ static float init(int t, int i) { return 1.0f + 1e-3f * static_cast<float>(t) + static_cast<float>(i); }
    __device__ static float add(float x, float a) { return __fadd_rn(x, a); }
    __device__ static float mul(float x, float a) { return __fmul_rn(x, a); }
    __device__ static float fma_(float x, float a, float b) { return __fmaf_rn(x, a, b); }
    __device__ static float sqrt_(float x) {
        float r;
        asm volatile("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    __device__ static float rcp(float x) {
        float r;
        asm volatile("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    __device__ static float fold(float x) { return x; }
};

template <> struct ProbeOps<double> {
    __device__ static double init(int t, int i) { return 1.0 + 1e-3 * t + i; }
    __device__ static double add(double x, double a) { return __dadd_rn(x, a); }
    __device__ static double mul(double x, double a) { return __dmul_rn(x, a); }
    __device__ static double fma_(double x, double a, double b) { return __fma_rn(x, a, b); }
    __device__ static double sqrt_(double x) { return __dsqrt_rn(x); }
    __device__ static double rcp(double x) { return __drcp_rn(x); }
    __device__ static double fold(double x) { return x; }
};

template <> struct ProbeOps<df> {
    __device__ static df init(int t, int i) { return df_two_sum(1.0f + 1e-3f * static_cast<float>(t), static_cast<float>(i) * 1e-9f); }
    __device__ static df add(df x, df a) { return x + a; }
    __device__ static df mul(df x, df a) { return x * a; }
    __device__ static df fma_(df x, df a, df b) { return x * a + b; }
    __device__ static df sqrt_(df x) { return df_sqrt(x); }
    __device__ static df rcp(df x) { return df_rcp(x); }
    __device__ static float fold(df x) { return __fadd_rn(x.hi, x.lo); }
};

// kChains independent chains of one operation per thread; the constants keep every chain
// finite and normal for any iteration count (x + a grows linearly, x a and x a + b stay
// near 1, the square root converges to 1, the reciprocal alternates).
template <typename T, int OP>
__global__ void __launch_bounds__(256) op_chains(float* __restrict__ sink, int iters, T a, T b) {
    using O = ProbeOps<T>;
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = O::init(threadIdx.x, i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            if constexpr (OP == HYDRA_OP_ADD) x[i] = O::add(x[i], b);
            else if constexpr (OP == HYDRA_OP_MUL) x[i] = O::mul(x[i], a);
            else if constexpr (OP == HYDRA_OP_FMA) x[i] = O::fma_(x[i], a, b);
            else if constexpr (OP == HYDRA_OP_SQRT) x[i] = O::sqrt_(x[i]);
            else x[i] = O::rcp(x[i]);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += static_cast<float>(O::fold(x[i]));
    sink[static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <typename T, int OP>
static hydra_status op_rate(int iters, T a, T b, double* per_s, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, op_chains<T, OP>, 256, 0);
    const unsigned grid = static_cast<unsigned>(sms * (per_sm > 0 ? per_sm : 1));
    float* sink = nullptr;
    cudaError_t err = cudaMalloc(&sink, static_cast<size_t>(grid) * 256 * sizeof(float));
    if (err != cudaSuccess) return cuda_fail(err, "probe sink");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    op_chains<T, OP><<<grid, 256, 0, st>>>(sink, iters / 10 + 1, a, b);  // warm-up
    cudaEventRecord(e0, st);
    op_chains<T, OP><<<grid, 256, 0, st>>>(sink, iters, a, b);
    cudaEventRecord(e1, st);
    err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return cuda_fail(err, "arithmetic-rate probe");
    *per_s = static_cast<double>(grid) * 256.0 * kChains * static_cast<double>(iters) / (ms * 1e-3);
    return HYDRA_OK;
}

template <typename T>
static hydra_status op_rate_for(hydra_probe_op op, int iters, T a, T b, double* per_s, cudaStream_t st) {
    switch (op) {
        case HYDRA_OP_ADD: return op_rate<T, HYDRA_OP_ADD>(iters, a, b, per_s, st);
        case HYDRA_OP_MUL: return op_rate<T, HYDRA_OP_MUL>(iters, a, b, per_s, st);
        case HYDRA_OP_FMA: return op_rate<T, HYDRA_OP_FMA>(iters, a, b, per_s, st);
        case HYDRA_OP_SQRT: return op_rate<T, HYDRA_OP_SQRT>(iters, a, b, per_s, st);
        case HYDRA_OP_RCP: return op_rate<T, HYDRA_OP_RCP>(iters, a, b, per_s, st);
    }
    return fail(HYDRA_ERR_INVALID_ARG, "unknown operation %d", static_cast<int>(op));
}

template <typename T>
static hydra_status fma_rate(int iters, double* per_s, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chains<T>, 256, 0);
    const unsigned grid = static_cast<unsigned>(sms * (per_sm > 0 ? per_sm : 1));
    T* sink = nullptr;
    cudaError_t err = cudaMalloc(&sink, static_cast<size_t>(grid) * 256 * sizeof(T));
    if (err != cudaSuccess) return cuda_fail(err, "probe sink");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = static_cast<T>(0.999999), b = static_cast<T>(1e-6);
    fma_chains<T><<<grid, 256, 0, st>>>(sink, iters / 10 + 1, a, b);  // warm-up
    cudaEventRecord(e0, st);
    fma_chains<T><<<grid, 256, 0, st>>>(sink, iters, a, b);
    cudaEventRecord(e1, st);
    err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return cuda_fail(err, "FMA probe");
    *per_s = static_cast<double>(grid) * 256.0 * kChains * static_cast<double>(iters) / (ms * 1e-3);
    return HYDRA_OK;
}

}  // namespace hydra

using namespace hydra;

extern "C" {

hydra_status hydra_probe_fma_rate(hydra_dtype dtype, int iterations, double* fma_per_s, hydra_stream_t stream) {
    if (!fma_per_s || iterations < 1) return fail(HYDRA_ERR_INVALID_ARG, "need iterations >= 1 and an output");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (dtype == HYDRA_F32) return fma_rate<float>(iterations, fma_per_s, st);
    if (dtype == HYDRA_F64) return fma_rate<double>(iterations, fma_per_s, st);
    return fail(HYDRA_ERR_INVALID_ARG, "unknown dtype %d", static_cast<int>(dtype));
}

hydra_status hydra_probe_op_rate(hydra_probe_arith arith, hydra_probe_op op, int iterations, double* ops_per_s,
                                 hydra_stream_t stream) {
    if (!ops_per_s || iterations < 1) return fail(HYDRA_ERR_INVALID_ARG, "need iterations >= 1 and an output");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    switch (arith) {
        case HYDRA_ARITH_F32: return op_rate_for<float>(op, iterations, 0.9999999f, 1e-7f, ops_per_s, st);
        case HYDRA_ARITH_F64: return op_rate_for<double>(op, iterations, 0.9999999999, 1e-9, ops_per_s, st);
        case HYDRA_ARITH_DOUBLE_FLOAT:
            return op_rate_for<df>(op, iterations, df{0.99999988f, 1e-15f}, df{1e-7f, 1e-16f}, ops_per_s, st);
    }
    return fail(HYDRA_ERR_INVALID_ARG, "unknown arithmetic %d", static_cast<int>(arith));
}

hydra_status hydra_probe_write_bandwidth(void* buffer, uint64_t bytes, int reps, double* gb_per_s,
                                         hydra_stream_t stream) {
    if (!buffer || !gb_per_s || reps < 1 || bytes < 16) return fail(HYDRA_ERR_INVALID_ARG, "bad probe arguments");
    if (reinterpret_cast<uintptr_t>(buffer) % 16 != 0) return fail(HYDRA_ERR_MISALIGNED, "buffer must be 16-byte aligned");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t n16 = bytes / 16;
    uint4* p = static_cast<uint4*>(buffer);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 0.0f;
    cudaError_t err = cudaSuccess;
    // the best over a few launch shapes: 4..32 blocks of 256 threads per SM, 1 or 4 stores in flight
    const int per_sm[4] = {4, 8, 16, 32};
    for (int c = 0; c < 8 && err == cudaSuccess; ++c) {
        const unsigned grid = static_cast<unsigned>(sms * per_sm[c % 4]);
        const bool unroll = c >= 4;
        if (unroll) fill16<4><<<grid, 256, 0, st>>>(p, n16, 0u);  // warm-up of the shape
        else fill16<1><<<grid, 256, 0, st>>>(p, n16, 0u);
        for (int r = 0; r < reps && err == cudaSuccess; ++r) {
            cudaEventRecord(e0, st);
            if (unroll) fill16<4><<<grid, 256, 0, st>>>(p, n16, static_cast<uint32_t>(r + 1));
            else fill16<1><<<grid, 256, 0, st>>>(p, n16, static_cast<uint32_t>(r + 1));
            cudaEventRecord(e1, st);
            err = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err == cudaSuccess && (best == 0.0f || ms < best)) best = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "write-bandwidth probe");
    *gb_per_s = static_cast<double>(n16 * 16) / (best * 1e-3) / 1e9;
    return HYDRA_OK;
}

}  // extern "C"
