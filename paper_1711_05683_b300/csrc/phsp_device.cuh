// phsp_device.cuh -- device building blocks of the phase-space Monte Carlo hot path.
//
// One event of the Raubold-Lynch generator (Hydra section 4.2; F. James, CERN 68-15) held
// entirely in registers: Philox4x32-10 draws, a sorting network over the intermediate-mass
// draws, intermediate masses from exact integer gaps, two-body momenta, the event weight,
// isotropic directions and the top-down chain of two-body decays with pure boosts.  The
// caller supplies a Sink that receives daughters and the weight; unused outputs are removed
// by the compiler (an integral over a flat matrix element never computes an angle).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "phsp_df.cuh"

namespace hydra {

constexpr int kNMax = 10;

// Per-decay constants, computed once per call on the host in FP64 and passed by value.
struct DecayConsts {
    // FP64 copies
    double M;           // parent mass
    double Ts;          // T * 2^-32 (T = M - sum m)
    double Ts_half;     // T * 2^-33
    double C;           // weight constant C_n
    double invM, halfInvM;  // 1/M and 1/(2M) (the parent's decay, the same for every event)
    double Mm1;             // M^2 + m_1^2 (s23 = M^2 + m_1^2 - 2 M E_1 of the Dalitz variables)
    double m[kNMax];    // daughter masses m_1..m_n at [0..n-1]
    double mu[kNMax];   // mu[k-1] = m_1 + ... + m_k
    double m2[kNMax];   // m_i^2
    double tm[kNMax];   // 2 m_i
    // FP32 copies (rounded from the FP64 values)
    float Mf, Tsf, Ts_halff, Cf, invMf, halfInvMf, Mm1f;
    float mf[kNMax], muf[kNMax], m2f[kNMax], tmf[kNMax];
    // double-float copies (hi, lo) for the df kinematics of the FP64 generator
    float Mdf[2], Tsdf[2], Ts_halfdf[2], invMdf[2], halfInvMdf[2], Mm1df[2];
    float mdf[kNMax][2], mudf[kNMax][2], m2df[kNMax][2], tmdf[kNMax][2];
    // Philox round keys: key + r * (W0, W1), r = 0..9
    uint32_t rk0[10], rk1[10];
    uint32_t massless;  // bit i set when daughter i+1 has mass 0
};

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter (c0..c3), round keys rk*.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              const uint32_t* __restrict__ rk0,
                                              const uint32_t* __restrict__ rk1, uint32_t out[4]) {
    constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = static_cast<uint64_t>(kM0) * c0;
        const uint64_t p1 = static_cast<uint64_t>(kM1) * c2;
        const uint32_t hi0 = static_cast<uint32_t>(p0 >> 32), lo0 = static_cast<uint32_t>(p0);
        const uint32_t hi1 = static_cast<uint32_t>(p1 >> 32), lo1 = static_cast<uint32_t>(p1);
        c0 = hi1 ^ c1 ^ rk0[r];
        c1 = lo1;
        c2 = hi0 ^ c3 ^ rk1[r];
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// ------------------------------------------------------------------------------------
// Ascending sort of the first K draws: Batcher's odd-even merge network for 8 inputs,
// with comparators that touch an index >= K removed (equivalent to padding with +inf).
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void compare_exchange(uint32_t& a, uint32_t& b) {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

__device__ __forceinline__ void compare_exchange(uint64_t& a, uint64_t& b) {
    const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}

template <int K, typename T>
__device__ __forceinline__ void sort_mass_draws(T* x) {
    constexpr int kPairs[19][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3}, {4, 6},
                                   {5, 7}, {1, 2}, {5, 6}, {0, 4}, {1, 5}, {2, 6}, {3, 7},
                                   {2, 4}, {3, 5}, {1, 2}, {3, 4}, {5, 6}};
#pragma unroll
    for (int i = 0; i < 19; ++i)
        if (kPairs[i][1] < K) compare_exchange(x[kPairs[i][0]], x[kPairs[i][1]]);
}

// ------------------------------------------------------------------------------------
// Precision traits.  FP32 kinematics use the hardware approximations sqrt.approx,
// rcp.approx and __sincosf (errors of a few units of 2^-24, far inside the FP32 tolerance);
// FP64 uses correctly rounded sqrt, division and sincospi.  Conversions of 32-bit draws
// are exact in FP64.
// ------------------------------------------------------------------------------------
template <typename R> struct Prec;

template <> struct Prec<float> {
    __device__ static float u32(uint32_t v) { return __uint2float_rn(v); }
    __device__ static float i32(int32_t v) { return __int2float_rn(v); }
    // Hardware approximations (a few ulp of 2^-24): the FP32 path's tolerance is 2e-5.
    __device__ static float sqrt_(float v) {  // sqrt.approx: exact 0 at 0, rel. error ~2^-23
        float r;
        asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
        return r;
    }
    __device__ static float rcp(float v) {  // rcp.approx: ~1 ulp for normal v
        float r;
        asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
        return r;
    }
    __device__ static float div(float a, float b) { return a * rcp(b); }
    __device__ static float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    // sums of terms that cannot cancel (the same operations in FP32)
    __device__ static float add_pos(float a, float b) { return a + b; }
    __device__ static float fma_pos(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    __device__ static float fma_lazy(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    __device__ static float sub_lazy(float a, float b) { return a - b; }
    __device__ static float sub_le(float a, float b) { return a - b; }
    // sin and cos of phi = 2 pi (x + 1/2) 2^-32: __sincosf is accurate (|err| < 2^-21.4) on
    // (-pi, pi), so evaluate it at phi - pi and flip both signs.
    __device__ static void sincos_2pi_u(uint32_t x, float* s, float* c) {
        constexpr float kTwoPiScale = 1.46291807926715968e-09f;              // 2 pi 2^-32
        constexpr float kShift = 7.31459039633579841e-10f - 3.14159265358979323846f;  // pi 2^-32 - pi
        float sn, cs;
        __sincosf(__fmaf_rn(__uint2float_rn(x), kTwoPiScale, kShift), &sn, &cs);
        *s = -sn;
        *c = -cs;
    }
    // cos(2 pi (xa - xb) 2^-32): the difference of two phi draws, exact modulo 2^32, in (-pi, pi]
    __device__ static float cos_2pi_diff(uint32_t xa, uint32_t xb) {
        return __cosf(__int2float_rn(static_cast<int32_t>(xa - xb)) * 1.46291807926715968e-09f);
    }
    __device__ static float scale(float x, float pow2) { return x * pow2; }
    __device__ static float half_odd(uint32_t y) { return __uint2float_rn(y) + 0.5f; }  // y + 1/2
    // 1 + cos(theta), 1 - cos(theta), cos(theta) of a cos(theta) draw x (u = (x + 1/2) 2^-32)
    __device__ static float one_plus_cos(uint32_t x) { return __fmaf_rn(__uint2float_rn(x), 4.656612873077392578125e-10f, 2.3283064365386962890625e-10f); }
    __device__ static float one_minus_cos(uint32_t x) { return one_plus_cos(~x); }
    __device__ static float cos_of(uint32_t x) { return __fmaf_rn(__int2float_rn(static_cast<int32_t>(x ^ 0x80000000u)), 4.656612873077392578125e-10f, 2.3283064365386962890625e-10f); }
    using W = float;    // weight type
    using Out = float;  // stored type
    using Wacc = float;  // weight product while it accumulates
    __device__ static Wacc w_one() { return 1.0f; }
    __device__ static Wacc w_mul(Wacc w, float p) { return w * p; }
    __device__ static W w_final(Wacc w, const DecayConsts& C) { return w * C.Cf; }
    __device__ static Out out(float v) { return v; }
    __device__ static float M(const DecayConsts& C) { return C.Mf; }
    __device__ static float Ts(const DecayConsts& C) { return C.Tsf; }
    __device__ static float Ts_half(const DecayConsts& C) { return C.Ts_halff; }
    __device__ static float Cn(const DecayConsts& C) { return C.Cf; }
    __device__ static float m(const DecayConsts& C, int i) { return C.mf[i]; }
    __device__ static float mu(const DecayConsts& C, int i) { return C.muf[i]; }
    __device__ static float m2(const DecayConsts& C, int i) { return C.m2f[i]; }
    __device__ static float twom(const DecayConsts& C, int i) { return C.tmf[i]; }
    __device__ static float invM(const DecayConsts& C) { return C.invMf; }
    __device__ static float halfInvM(const DecayConsts& C) { return C.halfInvMf; }
    __device__ static float Mm1(const DecayConsts& C) { return C.Mm1f; }
};

template <> struct Prec<double> {
    __device__ static double u32(uint32_t v) { return __uint2double_rn(v); }
    __device__ static double i32(int32_t v) { return __int2double_rn(v); }
    __device__ static double sqrt_(double v) { return sqrt(v); }
    __device__ static double rcp(double v) { return 1.0 / v; }
    __device__ static double div(double a, double b) { return a / b; }
    __device__ static double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
    __device__ static double add_pos(double a, double b) { return a + b; }
    __device__ static double fma_pos(double a, double b, double c) { return __fma_rn(a, b, c); }
    __device__ static double fma_lazy(double a, double b, double c) { return __fma_rn(a, b, c); }
    __device__ static double sub_lazy(double a, double b) { return a - b; }
    __device__ static double sub_le(double a, double b) { return a - b; }
    // sin and cos of phi = 2 pi u with u = (x + 1/2) 2^-32: sincospi(2u), argument exact.
    __device__ static void sincos_2pi_u(uint32_t x, double* s, double* c) {
        sincospi(__fma_rn(__uint2double_rn(x), 4.656612873077392578125e-10, 2.3283064365386962890625e-10), s, c);
    }
    __device__ static double cos_2pi_diff(uint32_t xa, uint32_t xb) {
        return cospi(__int2double_rn(static_cast<int32_t>(xa - xb)) * 4.656612873077392578125e-10);
    }
    __device__ static double scale(double x, double pow2) { return x * pow2; }
    __device__ static double half_odd(uint32_t y) { return __uint2double_rn(y) + 0.5; }
    __device__ static double one_plus_cos(uint32_t x) { return __fma_rn(__uint2double_rn(x), 4.656612873077392578125e-10, 2.3283064365386962890625e-10); }
    __device__ static double one_minus_cos(uint32_t x) { return one_plus_cos(~x); }
    __device__ static double cos_of(uint32_t x) { return __fma_rn(__int2double_rn(static_cast<int32_t>(x ^ 0x80000000u)), 4.656612873077392578125e-10, 2.3283064365386962890625e-10); }
    using W = double;
    using Out = double;
    using Wacc = double;
    __device__ static Wacc w_one() { return 1.0; }
    __device__ static Wacc w_mul(Wacc w, double p) { return w * p; }
    __device__ static W w_final(Wacc w, const DecayConsts& C) { return w * C.C; }
    __device__ static Out out(double v) { return v; }
    __device__ static double M(const DecayConsts& C) { return C.M; }
    __device__ static double Ts(const DecayConsts& C) { return C.Ts; }
    __device__ static double Ts_half(const DecayConsts& C) { return C.Ts_half; }
    __device__ static double Cn(const DecayConsts& C) { return C.C; }
    __device__ static double m(const DecayConsts& C, int i) { return C.m[i]; }
    __device__ static double mu(const DecayConsts& C, int i) { return C.mu[i]; }
    __device__ static double m2(const DecayConsts& C, int i) { return C.m2[i]; }
    __device__ static double twom(const DecayConsts& C, int i) { return C.tm[i]; }
    __device__ static double invM(const DecayConsts& C) { return C.invM; }
    __device__ static double halfInvM(const DecayConsts& C) { return C.halfInvM; }
    __device__ static double Mm1(const DecayConsts& C) { return C.Mm1; }
};

// Double-float kinematics for the FP64 generator: arithmetic on the FP32 pipe with ~48
// significand bits (phsp_df.cuh); the weight product and the stored values are FP64.
template <> struct Prec<df> {
    using W = double;
    using Out = double;
    __device__ static df scale(df x, float pow2) { return df_scale(x, pow2); }
    __device__ static df half_odd(uint32_t y) { return df_half_odd_raw(y); }
    __device__ static df one_plus_cos(uint32_t x) { return df_half_odd_u32(x); }
    __device__ static df one_minus_cos(uint32_t x) { return df_half_odd_u32(~x); }
    __device__ static df cos_of(uint32_t x) { return df_half_odd_centered(x); }
    __device__ static df u32(uint32_t v) { return df_from_u32(v); }
    __device__ static df i32(int32_t v) { return df_from_i32(v); }
    __device__ static df sqrt_(df v) { return df_sqrt(v); }
    __device__ static df rcp(df v) { return df_rcp(v); }
    __device__ static df div(df a, df b) { return df_div(a, b); }
    __device__ static df fma_(df a, df b, df c) { return a * b + c; }
    // a + b and a b + c whose terms are >= 0 (no cancellation): left unnormalised, the larger
    // high part first (FastTwoSum)
    __device__ static df add_pos(df a, df b) { return df_add_pos_lazy(a, b); }
    __device__ static df fma_pos(df a, df b, df c) { return df_add_pos_lazy(a * b, c); }
    // sums whose result only feeds products, sums and the conversion to double (the absolute
    // error at the scale of the terms is what matters): left unnormalised
    __device__ static df fma_lazy(df a, df b, df c) { return df_add_lazy(a * b, c); }
    __device__ static df sub_lazy(df a, df b) { return df_add_lazy(a, -b); }
    // a - b for 0 <= b <= a (an energy less a part of it), left unnormalised
    __device__ static df sub_le(df a, df b) { return df_sub_le_lazy(a, b); }
    __device__ static void sincos_2pi_u(uint32_t x, df* s, df* c) { df_sincos_2pi_u(x, s_sincos_table, s, c); }
    // cos(phi_a - phi_b) = cos(2 pi (xa - xb) 2^-32), the integer difference taken mod 2^32
    __device__ static df cos_2pi_diff(uint32_t xa, uint32_t xb) {
        df sv, cv;
        df_sincos_2pi_int(xa - xb, s_sincos_table, &sv, &cv);
        return cv;
    }
    using Wacc = DfWeight;  // double-float mantissa and binary exponent: no FP64 until the end
    __device__ static Wacc w_one() { return df_weight_one(); }
    __device__ static Wacc w_mul(Wacc w, df p) { return df_weight_mul(w, p); }
    __device__ static W w_final(Wacc w, const DecayConsts& C) { return df_weight_final(w, C.C); }
    __device__ static Out out(df v) { return df_to_double(v); }
    __device__ static df M(const DecayConsts& C) { return df{C.Mdf[0], C.Mdf[1]}; }
    __device__ static df Ts(const DecayConsts& C) { return df{C.Tsdf[0], C.Tsdf[1]}; }
    __device__ static df Ts_half(const DecayConsts& C) { return df{C.Ts_halfdf[0], C.Ts_halfdf[1]}; }
    __device__ static df m(const DecayConsts& C, int i) { return df{C.mdf[i][0], C.mdf[i][1]}; }
    __device__ static df mu(const DecayConsts& C, int i) { return df{C.mudf[i][0], C.mudf[i][1]}; }
    __device__ static df m2(const DecayConsts& C, int i) { return df{C.m2df[i][0], C.m2df[i][1]}; }
    __device__ static df twom(const DecayConsts& C, int i) { return df{C.tmdf[i][0], C.tmdf[i][1]}; }
    __device__ static df invM(const DecayConsts& C) { return df{C.invMdf[0], C.invMdf[1]}; }
    __device__ static df halfInvM(const DecayConsts& C) { return df{C.halfInvMdf[0], C.halfInvMdf[1]}; }
    __device__ static df Mm1(const DecayConsts& C) { return df{C.Mm1df[0], C.Mm1df[1]}; }
};

// Direction of subsystem k in the rest frame of subsystem k+1 for the double-float generators
// with N >= 6, as one out-of-line function: p (sin theta cos phi, sin theta sin phi, cos theta)
// from the cos(theta) draw xc and the phi draw xp.  Their unrolled bodies are long enough that a
// single copy of this code (sin(theta) by its square root, the sin/cos table step for phi and the
// five products) saves more in instruction fetch than the call costs.  Measured over the FP64
// sweep, against the sin/cos step alone out of line with its results through pointers (itself 3%
// faster than all inline): 2.2% faster, 3.5-4.5% at N = 9, 10, with bit-identical results; below
// N = 6 the inline code is faster.  The six FP32 parts come back by value, in registers.
struct DfDirection {
    float v[6];  // px, py, pz as (hi, lo) pairs
};

// The direction in double-float.  1 - cos(theta), 1 + cos(theta) and cos(theta) are the exact
// integers ~x + 1/2, x + 1/2 and x - 2^31 + 1/2 times 2^-31; the factor 2^-31 is applied once,
// to p, instead of to each of them (an exact power of two either way).  x + 1/2 is the exact
// pair a + b, a = x & ~0xFF and b = (x & 0xFF) + 1/2, and the other two follow from a and b by
// exact FP32 subtractions: ~x + 1/2 = (2^32 - 256 - a) + (256 - b) and
// x - 2^31 + 1/2 = (a - 2^31) + b (every result a multiple of 256 below 2^32 in magnitude, or
// below 256: representable, so the subtractions round nothing and the pairs are the ones the
// integer conversions give).  (~x + 1/2)(x + 1/2) >= 2^31, so the square root needs no zero test.
__device__ __forceinline__ DfDirection df_direction(df p, uint32_t xc, uint32_t xp) {
    const df p31 = df_scale(p, 4.656612873077392578125e-10f);  // p 2^-31
    const float a = __uint2float_rz(xc & 0xFFFFFF00u);
    const float b = __fadd_rn(__uint2float_rz(xc & 0xFFu), 0.5f);
    const df one_p31 = df_fast_two_sum(a, b);                                        // x + 1/2
    const df one_m31 = df_fast_two_sum(__fsub_rn(4294967040.0f, a), __fsub_rn(256.0f, b));  // ~x + 1/2
    const df cos_t31 = df_fast_two_sum(__fsub_rn(a, 2147483648.0f), b);              // cos(theta) 2^31
    const df sin_t31 = df_sqrt_pos(one_m31 * one_p31);                               // sin(theta) 2^31
    df sphi, cphi;
    df_sincos_2pi_u(xp, s_sincos_table, &sphi, &cphi);
    const df ps = p31 * sin_t31;
    const df px = ps * cphi, py = ps * sphi, pz = p31 * cos_t31;
    return DfDirection{{px.hi, px.lo, py.hi, py.lo, pz.hi, pz.lo}};
}

static __device__ __noinline__ DfDirection df_direction_outlined(df p, uint32_t xc, uint32_t xp) {
    return df_direction(p, xc, xp);
}

// ------------------------------------------------------------------------------------
// A group of EPT Raubold-Lynch events computed in lockstep (EPT independent dependency
// chains per thread).  The library is compiled with -fmad=false and every fused
// multiply-add is written out, so the rounding of each event is fixed by this source and
// results are bit-identical whatever the group size, block size or batch composition.
//
// Draws: d = 0..n-3 intermediate masses; for top-down step j = 0..n-2 (j = 0 is the
// parent's decay) cos(theta) from draw n-2+2j and phi from draw n-1+2j.  Draw d is word
// d%4 of Philox block d/4; each block is generated when a draw first needs it (live state:
// the sorted mass draws and one block).
//
// With y_1 <= ... <= y_{n-2} the sorted mass draws, r_j = (y_j + 1/2) 2^-32, r_0 = 0,
// r_{n-1} = 1:  M_1 = m_1, M_k = mu_k + r_{k-1} T, M_n = M, and the kinetic gaps
// Delta_k = T (r_k - r_{k-1}) are formed from exact 32-bit integer differences.
// p_k = sqrt(Delta (Delta + 2 M_k)(Delta + 2 m_{k+1})(Delta + 2 M_k + 2 m_{k+1})) / (2 M_{k+1})
// (Kallen's lambda, factorised; no cancellation near threshold).  w = (prod p_k) C_n.
// Subsystem k's energy in the rest frame of k+1 is M_k + Delta (Delta + 2 m_{k+1}) / (2 M_{k+1})
// (the two-body energy (M_{k+1}^2 + M_k^2 - m_{k+1}^2) / (2 M_{k+1}) rewritten with the gap),
// which reuses a factor of lambda instead of a square root of p^2 + M_k^2.
//
// Top-down: Q = lab 4-momentum of subsystem k+1 (daughters 1..k+1), Q = (M, 0) for k = n-1.
// In its rest frame subsystem k moves along +p_k n and daughter k+1 along -p_k n.  The
// subsystem is boosted to the lab, E' = (Q0 E + Q.p)/M_{k+1},
// p' = p + Q (E' + E)/(Q0 + M_{k+1}); daughter k+1 = Q - Q' by 4-momentum conservation.
//
// Sink interface (arrays hold one value per event of the group):
//   sink.daughter(i, E, px, py, pz)  daughter index i = 0..n-1 (daughter i+1)
//   sink.subsystem_mass(k, Mk)       M_k for k = 1..n-1
//   sink.weight(w)
// kMassless: a variant for decays whose daughters are all massless (chosen by the host), where
// lambda(M_{k+1}^2, M_k^2, 0) = (Delta (Delta + 2 M_k))^2 and the momentum needs no square root.
// kLambda64 (FP32 kinematics only): the four factors of lambda multiplied in FP64 and the
// product rounded once to FP32 before its square root.
// ------------------------------------------------------------------------------------
template <int N, typename R, int EPT, bool kMassless = false, bool kLambda64 = false, typename Sink>
__device__ __forceinline__ void raubold_lynch_group(const DecayConsts& C, const uint64_t (&ev)[EPT],
                                                    Sink& sink) {
    using P = Prec<R>;
    constexpr int kMass = N - 2;
    constexpr int kMassBlocks = (kMass + 3) / 4;
    constexpr int kY = kMass > 0 ? kMass : 1;

    uint32_t y[EPT][kY];
    uint32_t blk[EPT][4];
#pragma unroll
    for (int b = 0; b < kMassBlocks; ++b) {
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            philox4x32_10(static_cast<uint32_t>(ev[q]), static_cast<uint32_t>(ev[q] >> 32), b, 0u,
                          C.rk0, C.rk1, blk[q]);
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (4 * b + t < kMass) y[q][4 * b + t] = blk[q][t];
        }
    }
    if constexpr (N > 3) {
#pragma unroll
        for (int q = 0; q < EPT; ++q) sort_mass_draws<N - 2>(y[q]);
    }

    const R M = P::M(C);
    const R Ts = P::Ts(C);

    using W = typename P::W;
    typename P::Wacc w[EPT];
    R Q0[EPT], Qx[EPT], Qy[EPT], Qz[EPT], Mnext[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        w[q] = P::w_one();  // prod p_k; C_n is applied last so only the final product can leave the normal range
        Q0[q] = M; Qx[q] = R(0); Qy[q] = R(0); Qz[q] = R(0);
        Mnext[q] = M;  // M_{k+1}
    }

    // double-float only: the parts of the previous step's draw and its (y + 1/2) T 2^-32
    float draw_a[EPT], draw_b[EPT];
    df draw_T[EPT];
    int cur = kMassBlocks - 1;  // Philox block held in blk (-1: none); known at compile time
#pragma unroll
    for (int k = N - 1; k >= 1; --k) {
        const int j = N - 1 - k;
        const int dc = N - 2 + 2 * j;  // cos(theta) draw; the phi draw dc + 1 may open the next block
        uint32_t xcs[EPT], xps[EPT];
        if (dc / 4 != cur) {
#pragma unroll
            for (int q = 0; q < EPT; ++q)
                philox4x32_10(static_cast<uint32_t>(ev[q]), static_cast<uint32_t>(ev[q] >> 32), dc / 4, 0u,
                              C.rk0, C.rk1, blk[q]);
            cur = dc / 4;
        }
#pragma unroll
        for (int q = 0; q < EPT; ++q) xcs[q] = blk[q][dc % 4];
        if ((dc + 1) / 4 != cur) {
#pragma unroll
            for (int q = 0; q < EPT; ++q)
                philox4x32_10(static_cast<uint32_t>(ev[q]), static_cast<uint32_t>(ev[q] >> 32), (dc + 1) / 4,
                              0u, C.rk0, C.rk1, blk[q]);
            cur = (dc + 1) / 4;
        }
#pragma unroll
        for (int q = 0; q < EPT; ++q) xps[q] = blk[q][(dc + 1) % 4];
        R dE[EPT], dx[EPT], dy[EPT], dz[EPT], Mk_out[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            // intermediate mass M_k
            R Mk;
            // kinetic gap Delta_k = T (r_k - r_{k-1}) from integer differences
            R gap;
            if constexpr (std::is_same<R, df>::value && N > 2) {
                // Double-float: each sorted draw's y + 1/2 as the exact pair a + b, a = y & ~0xFF,
                // b = (y & 0xFF) + 1/2, converted once.  The gaps follow from neighbouring parts by
                // exact FP32 subtractions (multiples of 256 below 2^32, or below 256 in magnitude):
                // y_k - y_{k-1} = (a_k - a_{k-1}) + (b_k - b_{k-1}) and 2^32 - 1 - y + 1/2 =
                // (2^32 - 256 - a) + (256 - b); FastTwoSum then gives the same pair as converting
                // the integer difference.
                float a = 0.0f, b = 0.0f;
                df hT{0.0f, 0.0f};
                if (k >= 2) {
                    const uint32_t yv = y[q][k - 2];
                    a = __uint2float_rz(yv & 0xFFFFFF00u);
                    b = __fadd_rn(__uint2float_rz(yv & 0xFFu), 0.5f);
                    hT = df_fast_two_sum(a, b) * Ts;  // (y + 1/2) T 2^-32
                    Mk = df_add_pos_lazy(hT, P::mu(C, k - 1));
                } else {
                    Mk = P::m(C, 0);
                }
                if (k == N - 1) gap = df_fast_two_sum(__fsub_rn(4294967040.0f, a), __fsub_rn(256.0f, b)) * Ts;
                else if (k == 1) gap = draw_T[q];
                else gap = df_fast_two_sum(__fsub_rn(draw_a[q], a), __fsub_rn(draw_b[q], b)) * Ts;
                draw_a[q] = a; draw_b[q] = b; draw_T[q] = hT;
            } else {
            if (k == 1) Mk = P::m(C, 0);
            else Mk = P::fma_pos(P::half_odd(y[q][k - 2]), Ts, P::mu(C, k - 1));
            if constexpr (N == 2) {
                gap = Ts * R(4294967296.0);  // T exactly: Ts = T * 2^-32
            } else if (k == 1) {
                gap = P::half_odd(y[q][0]) * Ts;
            } else if (k == N - 1) {
                gap = P::half_odd(~y[q][kY - 1]) * Ts;
            } else {
                gap = P::u32(y[q][k - 1] - y[q][k - 2]) * Ts;
            }
            }
            Mk_out[q] = Mk;
            // two-body momentum
            const R twoMk = k == 1 ? P::twom(C, 0) : P::scale(Mk, 2.0f);  // 2 M_1 = 2 m_1
            // 1/M_{k+1}; for the parent's decay a host constant
            const R invM = k == N - 1 ? P::invM(C) : P::rcp(Mnext[q]);
            const R halfInvM = k == N - 1 ? P::halfInvM(C) : P::scale(invM, 0.5f);
            R p, gm;  // gm = Delta (Delta + 2 m_{k+1})
            if constexpr (kMassless) {
                // every daughter massless: lambda = (Delta (Delta + 2 M_k))^2, no square root;
                // the last step has M_1 = 0, so p = Delta^2 / (2 M_2) (the same operations with
                // the zero terms dropped: bit-identical)
                gm = gap * gap;
                if (k == 1) p = gm * halfInvM;
                else p = (gap * P::add_pos(gap, twoMk)) * halfInvM;
            } else {
                const R twom = P::twom(C, k);
                const R a = P::add_pos(gap, twoMk);
                const R gpm = P::add_pos(gap, twom);
                gm = gap * gpm;
                R lam;
                if constexpr (kLambda64) {
                    static_assert(std::is_same<R, float>::value, "the FP64 lambda product is an FP32-kinematics mode");
                    lam = __double2float_rn(__dmul_rn(__dmul_rn(__dmul_rn(static_cast<double>(gap), static_cast<double>(gpm)),
                                                                static_cast<double>(a)),
                                                      static_cast<double>(P::add_pos(a, twom))));
                } else {
                    lam = (gm * a) * P::add_pos(a, twom);
                }
                p = P::sqrt_(lam) * halfInvM;
            }
            w[q] = P::w_mul(w[q], p);
            // isotropic direction of subsystem k in the rest frame of subsystem k+1
            const uint32_t xc = xcs[q];
            const uint32_t xp = xps[q];
            R px, py, pz;
            if constexpr (std::is_same<R, df>::value) {
                DfDirection d;
                if constexpr (N >= 6) d = df_direction_outlined(p, xc, xp);  // one copy of the code
                else d = df_direction(p, xc, xp);
                px = df{d.v[0], d.v[1]}; py = df{d.v[2], d.v[3]}; pz = df{d.v[4], d.v[5]};
            } else {
                const R cos_t = P::cos_of(xc);         // 2u - 1
                const R one_m = P::one_minus_cos(xc);  // 1 - cos(theta)
                const R one_p = P::one_plus_cos(xc);   // 1 + cos(theta)
                const R sin_t = P::sqrt_(one_m * one_p);
                R sphi, cphi;
                P::sincos_2pi_u(xp, &sphi, &cphi);  // phi = 2 pi u
                const R ps = p * sin_t;
                px = ps * cphi; py = ps * sphi; pz = p * cos_t;
            }
            // energy of subsystem k in the rest frame of k+1: (M_{k+1}^2 + M_k^2 - m_{k+1}^2) / (2 M_{k+1})
            // = M_k + Delta (Delta + 2 m_{k+1}) / (2 M_{k+1}), a sum of positive terms
            // (massless last step: M_1 = 0 and Es = p, the energy of a massless daughter)
            const R Es = (kMassless && k == 1) ? p : P::fma_pos(gm, halfInvM, Mk);
            if (k == N - 1) {
                // parent at rest: no boost
                dE[q] = P::sub_le(M, Es); dx[q] = -px; dy[q] = -py; dz[q] = -pz;
                Q0[q] = Es; Qx[q] = px; Qy[q] = py; Qz[q] = pz;
            } else {
                // Q.p and the lab momentum n: their sums may cancel and are left unnormalised.
                // The lab energy E1 is renormalised: it feeds the next step's product Q0 Es and
                // the reciprocal of Q0 + M, and an unnormalised low part carried along the chain
                // of boosts grows until the product's dropped lo x lo term and the reciprocal's
                // FP32 residual reach ~2^-40 of the event scale (measured: 9.4e-13 worst error
                // against the oracle over 3.6e6 events with E1 lazy, 8.4e-14 renormalised).
                const R qp = P::fma_lazy(Qz[q], pz, P::fma_lazy(Qy[q], py, Qx[q] * px));
                const R E1 = P::fma_(Q0[q], Es, qp) * invM;
                const R f = P::div(P::add_pos(E1, Es), P::add_pos(Q0[q], Mnext[q]));
                const R nx = P::fma_lazy(f, Qx[q], px), ny = P::fma_lazy(f, Qy[q], py), nz = P::fma_lazy(f, Qz[q], pz);
                // the daughter by 4-momentum conservation (stored: left unnormalised)
                dE[q] = P::sub_le(Q0[q], E1); dx[q] = P::sub_lazy(Qx[q], nx);
                dy[q] = P::sub_lazy(Qy[q], ny); dz[q] = P::sub_lazy(Qz[q], nz);
                Q0[q] = E1; Qx[q] = nx; Qy[q] = ny; Qz[q] = nz;
            }
            Mnext[q] = Mk;
        }
        sink.subsystem_mass(k, Mk_out);
        sink.daughter(k, dE, dx, dy, dz);
    }
    sink.daughter(0, Q0, Qx, Qy, Qz);
    W wout[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) wout[q] = P::w_final(w[q], C);
    sink.weight(wout);
}

// ------------------------------------------------------------------------------------
// Generation sink: structure-of-arrays stores out[(i*4 + c)*ld + e], weights[e].
// ------------------------------------------------------------------------------------
// Store EPT consecutive values (16-byte vectors where the group allows it).
template <typename R, int EPT>
__device__ __forceinline__ void store_group(R* __restrict__ p, const R (&v)[EPT]) {
    if constexpr (EPT == 1) {
        p[0] = v[0];
    } else if constexpr (sizeof(R) == 4 && EPT == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    } else if constexpr (sizeof(R) == 4 && EPT == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        static_assert(sizeof(R) == 8 && EPT % 2 == 0, "double groups are pairs");
#pragma unroll
        for (int q = 0; q < EPT; q += 2) *reinterpret_cast<double2*>(p + q) = make_double2(v[q], v[q + 1]);
    }
}

template <typename R, int EPT>
struct StoreSink {
    using Out = typename Prec<R>::Out;
    using W = typename Prec<R>::W;
    Out* __restrict__ base;  // out + e0
    Out* __restrict__ wout;  // weights + e0
    uint64_t ld;
    __device__ __forceinline__ void subsystem_mass(int, const R (&)[EPT]) {}
    __device__ __forceinline__ void put(Out* p, const R (&v)[EPT]) {
        Out o[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) o[q] = Prec<R>::out(v[q]);
        store_group<Out, EPT>(p, o);
    }
    __device__ __forceinline__ void daughter(int i, const R (&E)[EPT], const R (&px)[EPT],
                                             const R (&py)[EPT], const R (&pz)[EPT]) {
        Out* p = base + static_cast<uint64_t>(4 * i) * ld;
        put(p, E);
        put(p + ld, px);
        put(p + 2 * ld, py);
        put(p + 3 * ld, pz);
    }
    __device__ __forceinline__ void weight(const W (&w)[EPT]) {
        Out o[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) o[q] = static_cast<Out>(w[q]);
        store_group<Out, EPT>(wout, o);
    }
};

}  // namespace hydra
