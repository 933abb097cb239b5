// phsp_integral.cuh -- device side of the phase-space integral (section 3, "phase-space
// Monte Carlo integration"): the integrand f = w |ME|^2 over Raubold-Lynch events, the
// fixed-order tile sums, and the compensated FP64 accumulators of the reduction tree.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hydra_phsp.h"
#include "phsp_device.cuh"

namespace hydra {

// ------------------------------------------------------------------------------------
// Fixed reduction geometry of the integral (part of the result's definition).
// ------------------------------------------------------------------------------------
constexpr int kTileEvents = 2048;                         // events per warp tile
constexpr int kGroupEvents = 8;                           // events a lane sums in R before FP64
constexpr int kLaneIters = kTileEvents / 32;              // 64 events per lane per tile
constexpr int kSegTiles = 1024;                           // tiles per segment (2^21 events)
constexpr uint64_t kChunkTiles = 32768;                   // tiles per launch (2^26 events)
static_assert(kChunkTiles % kSegTiles == 0, "a chunk holds whole segments");
static_assert(kLaneIters % kGroupEvents == 0, "groups tile the lane's events");

struct TileSums {
    double f, f2, w, w2;
};

// Matrix-element parameters in both precisions.
struct MEConsts {
    double a_m2, a_mg, b_m2, b_mg, c_re, c_im;  // m0^2, m0*Gamma, Re c, Im c
    float a_m2f, a_mgf, b_m2f, b_mgf, c_ref, c_imf;           // FP32 values (double-float high parts)
    float a_m2lo, a_mglo, b_m2lo, b_mglo, c_relo, c_imlo;     // double-float low parts
};

template <typename R, int EPT>
struct IntegrandSink {
    using W = typename Prec<R>::W;  // weights: FP32, or FP64 for double and double-float kinematics
    R E1[EPT], M2[EPT];
    W w[EPT];
    __device__ __forceinline__ void subsystem_mass(int k, const R (&Mk)[EPT]) {
        if (k == 2) {
#pragma unroll
            for (int q = 0; q < EPT; ++q) M2[q] = Mk[q];
        }
    }
    __device__ __forceinline__ void daughter(int i, const R (&E)[EPT], const R (&)[EPT],
                                             const R (&)[EPT], const R (&)[EPT]) {
        if (i == 0) {
#pragma unroll
            for (int q = 0; q < EPT; ++q) E1[q] = E[q];
        }
    }
    __device__ __forceinline__ void weight(const W (&wv)[EPT]) {
#pragma unroll
        for (int q = 0; q < EPT; ++q) w[q] = wv[q];
    }
};

// A matrix-element parameter in arithmetic R: the FP32 value, the FP64 value, or the
// double-float pair (hi, lo).
template <typename R> __device__ __forceinline__ R me_param(double d, float f, float lo);
template <> __device__ __forceinline__ float me_param<float>(double, float f, float) { return f; }
template <> __device__ __forceinline__ double me_param<double>(double d, float, float) { return d; }
template <> __device__ __forceinline__ df me_param<df>(double, float f, float lo) { return df{f, lo}; }

// A value of arithmetic R in the weights' type (the double-float result rounded to FP64).
template <typename R>
__device__ __forceinline__ typename Prec<R>::W to_w(R v) {
    if constexpr (std::is_same<R, df>::value) return df_to_double(v);
    else return v;
}

// |BW(s12; a) + c BW(s23; b)|^2, BW(s) = (m0^2 - s + i m0 G) / ((m0^2 - s)^2 + (m0 G)^2), from
// xa = m0a^2 - s12 and xb = m0b^2 - s23 (near a narrow resonance the subtraction is the
// ill-conditioned step; what follows is well conditioned).
template <typename R>
__device__ __forceinline__ R dalitz_2bw_x(const MEConsts& P, R xa, R xb) {
    const R ya = me_param<R>(P.a_mg, P.a_mgf, P.a_mglo);
    const R yb = me_param<R>(P.b_mg, P.b_mgf, P.b_mglo);
    using Q = Prec<R>;
    const R ia = Q::rcp(Q::fma_(xa, xa, ya * ya));
    const R ib = Q::rcp(Q::fma_(xb, xb, yb * yb));
    const R cr = me_param<R>(P.c_re, P.c_ref, P.c_relo), ci = me_param<R>(P.c_im, P.c_imf, P.c_imlo);
    const R re = Q::fma_(xa, ia, Q::fma_(cr, xb, -(ci * yb)) * ib);
    const R im = Q::fma_(ya, ia, Q::fma_(cr, yb, ci * xb) * ib);
    return Q::fma_(re, re, im * im);
}

template <typename R>
__device__ __forceinline__ R dalitz_2bw(const MEConsts& P, R s12, R s23) {
    return dalitz_2bw_x<R>(P, me_param<R>(P.a_m2, P.a_m2f, P.a_m2lo) - s12, me_param<R>(P.b_m2, P.b_m2f, P.b_m2lo) - s23);
}

// The N = 3 integrand from the event's five draws without its 4-vectors.  Same event as
// raubold_lynch_group<3>: draw 0 gives M_2 = mu_2 + r T, the gaps T (1 - r) and T r, the
// momenta p2 (parent -> (12) + 3) and p1 ((12) -> 1 + 2) and the weight (p2 p1) C_3; draws
// (1, 2) and (3, 4) are the directions n_a of subsystem (12) in the parent frame and n_b of
// daughter 1 in the (12) frame, both in the parent's axes (pure boosts), so the boost gives
//   E1 = (Q0 E1* + p2 p1 cos alpha) / M_2,  Q0 = sqrt(p2^2 + M_2^2),  E1* = sqrt(p1^2 + m1^2)
//   (both energies taken from the gap factors of lambda, without a square root),
//   cos alpha = n_a . n_b = c_a c_b + s_a s_b cos(phi_a - phi_b),
// with phi_a - phi_b from the integer difference of the two phi draws.  Then s12 = M_2^2 and
// s23 = M^2 + m1^2 - 2 M E1 as in the general path; one cosine instead of two sin/cos pairs
// and no 3-vectors.
template <typename R>
__device__ __forceinline__ void dalitz3_point(const DecayConsts& C, const MEConsts& P, uint64_t e,
                                              typename Prec<R>::W& f, typename Prec<R>::W& wout) {
    using Q = Prec<R>;
    using W = typename Q::W;
    uint32_t b0[4], b1[4];
    philox4x32_10(static_cast<uint32_t>(e), static_cast<uint32_t>(e >> 32), 0u, 0u, C.rk0, C.rk1, b0);
    philox4x32_10(static_cast<uint32_t>(e), static_cast<uint32_t>(e >> 32), 1u, 0u, C.rk0, C.rk1, b1);
    const uint32_t y = b0[0], xca = b0[1], xpa = b0[2], xcb = b0[3], xpb = b1[0];
    const R M = Q::M(C), Ts = Q::Ts(C);
    const R m1 = Q::m(C, 0);
    const R M2 = Q::fma_(Q::half_odd(y), Ts, Q::mu(C, 1));
    const R gap2 = Q::half_odd(~y) * Ts;  // T (1 - r)
    const R gap1 = Q::half_odd(y) * Ts;   // T r
    const R twoM2 = Q::scale(M2, 2.0f), twom3 = Q::twom(C, 2);
    const R a2 = gap2 + twoM2, g2 = gap2 * (gap2 + twom3);  // g2 = Delta2 (Delta2 + 2 m3)
    const R lam2 = (g2 * a2) * (a2 + twom3);
    const R twom1 = Q::twom(C, 0), twom2 = Q::twom(C, 1);
    const R a1 = gap1 + twom1, g1 = gap1 * (gap1 + twom2);  // g1 = Delta1 (Delta1 + 2 m2)
    const R lam1 = (g1 * a1) * (a1 + twom2);
    const R invM2 = Q::rcp(M2);
    const R halfInvM = Q::halfInvM(C), halfInvM2 = Q::scale(invM2, 0.5f);
    const R p2 = Q::sqrt_(lam2) * halfInvM;
    const R p1 = Q::sqrt_(lam1) * halfInvM2;
    const W w = Q::w_final(Q::w_mul(Q::w_mul(Q::w_one(), p2), p1), C);
    const R ssq = (Q::one_minus_cos(xca) * Q::one_plus_cos(xca)) * (Q::one_minus_cos(xcb) * Q::one_plus_cos(xcb));
    const R cos_alpha = Q::fma_(Q::cos_of(xca), Q::cos_of(xcb), Q::sqrt_(ssq) * Q::cos_2pi_diff(xpa, xpb));
    // two-body energies from the gap factors of lambda (as in the generator):
    // Q0 = (M^2 + M2^2 - m3^2) / (2 M) = M2 + g2 / (2 M), E1* = (M2^2 + m1^2 - m2^2) / (2 M2) = m1 + g1 / (2 M2)
    const R Q0 = Q::fma_(g2, halfInvM, M2);
    const R E1s = Q::fma_(g1, halfInvM2, m1);
    const R E1 = Q::fma_(Q0, E1s, (p2 * p1) * cos_alpha) * invM2;
    const R s12 = M2 * M2;
    const R s23 = Q::fma_(R(-2) * M, E1, Q::Mm1(C));
    wout = w;
    f = w * to_w<R>(dalitz_2bw<R>(P, s12, s23));
}

template <int N, typename R, int ME, int EPT>
__device__ __forceinline__ void integrand_group(const DecayConsts& C, const MEConsts& P, const uint64_t (&ev)[EPT],
                                                typename Prec<R>::W (&f)[EPT], typename Prec<R>::W (&w)[EPT]) {
    if constexpr (ME == HYDRA_ME_DALITZ_2BW && N == 3) {
#pragma unroll
        for (int q = 0; q < EPT; ++q) dalitz3_point<R>(C, P, ev[q], f[q], w[q]);
        return;
    }
    IntegrandSink<R, EPT> s;
    raubold_lynch_group<N, R, EPT>(C, ev, s);
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        w[q] = s.w[q];
        if constexpr (ME == HYDRA_ME_DALITZ_2BW) {
            // s12 = M_2^2 (subsystem of daughters 1, 2); s23 = (P - p1)^2 = M^2 + m1^2 - 2 M E1
            const R M = Prec<R>::M(C);
            const R s12 = s.M2[q] * s.M2[q];
            const R s23 = Prec<R>::fma_(R(-2) * M, s.E1[q], Prec<R>::Mm1(C));
            f[q] = s.w[q] * to_w<R>(dalitz_2bw<R>(P, s12, s23));
        } else {
            f[q] = s.w[q];
        }
    }
}


// One warp per tile of kTileEvents events.  Lane l takes events tile*2048 + 32*i + l,
// i = 0..63, sums them in R in groups of 8 (fixed order), folds each group into FP64, and
// the warp combines lanes by a fixed xor butterfly; lane 0's total is the tile partial.
// Sums of (f, f^2, w, w^2) over tile `tile` (events tile*2048 .. tile*2048+2047 of a
// request; events >= nevents are skipped).  Lane l takes events 32 i + l, i = 0..63, sums
// them in R in groups of 8 (fixed order), folds each group into FP64, and the warp combines
// lanes by a fixed xor butterfly; lane 0's value is the tile partial.  Every integral entry
// point uses this routine, so a request gives the same bits alone or in a batch.
template <int N, typename R, int ME, int EPT>
__device__ __forceinline__ TileSums tile_sums(const DecayConsts& C, const MEConsts& P, uint64_t nevents,
                                              uint64_t event_offset, uint64_t tile, int lane) {
    static_assert(kGroupEvents % EPT == 0, "a group holds whole event groups");
    using W = typename Prec<R>::W;  // the group sums' type: FP32 kinematics sum in FP32, FP64 ones in FP64
    const uint64_t base = tile * kTileEvents;
    double af = 0.0, af2 = 0.0, aw = 0.0, aw2 = 0.0;
#pragma unroll 1
    for (int g = 0; g < kLaneIters / kGroupEvents; ++g) {
        W sf = W(0), sf2 = W(0), sw = W(0), sw2 = W(0);
#pragma unroll 1
        for (int i0 = 0; i0 < kGroupEvents; i0 += EPT) {
            uint64_t ev[EPT];
            bool valid[EPT];
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const uint64_t e = base + static_cast<uint64_t>(32 * (g * kGroupEvents + i0 + q) + lane);
                valid[q] = e < nevents;
                ev[q] = event_offset + e;
            }
            W f[EPT], w[EPT];
            integrand_group<N, R, ME, EPT>(C, P, ev, f, w);
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                if (valid[q]) {
                    sf += f[q];
                    sf2 = Prec<W>::fma_(f[q], f[q], sf2);
                    sw += w[q];
                    sw2 = Prec<W>::fma_(w[q], w[q], sw2);
                }
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
    return TileSums{af, af2, aw, aw2};
}

// Compensated FP64 accumulator (Neumaier's variant of Kahan summation).
struct Comp {
    double s = 0.0, c = 0.0;
    __device__ __forceinline__ void add(double x) {
        const double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    // Combine with another accumulator: TwoSum of the leading parts, compensations added.
    __device__ __forceinline__ void merge(double s2, double c2) {
        const double t = s + s2;
        const double bb = t - s;
        const double err = (s - (t - bb)) + (s2 - bb);
        s = t;
        c = c + c2 + err;
    }
};

__device__ __forceinline__ void warp_merge(Comp& a) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double s2 = __shfl_xor_sync(0xffffffffu, a.s, off);
        const double c2 = __shfl_xor_sync(0xffffffffu, a.c, off);
        a.merge(s2, c2);
    }
}

// Compensated sums of nt (<= kSegTiles) consecutive tile partials by one block of kSegWarps
// warps (every thread of the block calls it): warp v takes tiles [v 128, (v + 1) 128), its
// lane l tiles v 128 + l + 32 i (i = 0..3) in order; a fixed TwoSum butterfly merges the
// lanes, thread 0 merges the warps in order v = 0..7 and writes 8 doubles (s, c) for f, f^2,
// w, w^2 to out.  (One warp per segment left a 2^26-event chunk on 8 SMs, each lane with 128
// dependent compensated FP64 additions on B300's narrow FP64 pipe.)
constexpr int kSegWarps = 8;
constexpr int kSegBlock = 32 * kSegWarps;

__device__ __forceinline__ void segment_sums_block(const TileSums* __restrict__ partials, uint64_t nt,
                                                   double* __restrict__ out) {
    constexpr int kPerWarp = kSegTiles / kSegWarps;
    constexpr int kPerLane = kPerWarp / 32;
    __shared__ double part[kSegWarps][8];
    const int lane = threadIdx.x & 31, v = threadIdx.x >> 5;
    TileSums p[kPerLane];
#pragma unroll
    for (int i = 0; i < kPerLane; ++i) {
        const uint64_t t = static_cast<uint64_t>(v * kPerWarp + i * 32 + lane);
        p[i] = t < nt ? partials[t] : TileSums{0.0, 0.0, 0.0, 0.0};
    }
    Comp f, f2, w, w2;
#pragma unroll
    for (int i = 0; i < kPerLane; ++i) {
        if (static_cast<uint64_t>(v * kPerWarp + i * 32 + lane) < nt) {
            f.add(p[i].f);
            f2.add(p[i].f2);
            w.add(p[i].w);
            w2.add(p[i].w2);
        }
    }
    warp_merge(f);
    warp_merge(f2);
    warp_merge(w);
    warp_merge(w2);
    if (lane == 0) {
        part[v][0] = f.s; part[v][1] = f.c; part[v][2] = f2.s; part[v][3] = f2.c;
        part[v][4] = w.s; part[v][5] = w.c; part[v][6] = w2.s; part[v][7] = w2.c;
    }
    __syncthreads();
    if (threadIdx.x < 4) {  // lane k merges quantity k over the warps in order (FP64 pipe: 4 lanes, one pass)
        const int k = threadIdx.x;
        Comp q;
        q.s = part[0][2 * k];
        q.c = part[0][2 * k + 1];
        for (int u = 1; u < kSegWarps; ++u) q.merge(part[u][2 * k], part[u][2 * k + 1]);
        out[2 * k] = q.s;
        out[2 * k + 1] = q.c;
    }
    __syncthreads();  // part is reused by the block's next segment
}

// One warp folds nseg segment partials (lane l: segments l, l+32, ...), merges lanes and
// lane 0 writes mean, variance of the mean and the sums.
__device__ __forceinline__ void fold_segments(const double* __restrict__ seg, uint64_t nseg, uint64_t nevents,
                                              int lane, hydra_integral* __restrict__ out) {
    Comp q[4];
    for (uint64_t s = lane; s < nseg; s += 32) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            q[k].add(seg[s * 8 + 2 * k]);
            q[k].add(seg[s * 8 + 2 * k + 1]);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) warp_merge(q[k]);
    if (lane == 0) {
        const double n = static_cast<double>(nevents);
        const double sf = q[0].s + q[0].c, sf2 = q[1].s + q[1].c;
        const double sw = q[2].s + q[2].c, sw2 = q[3].s + q[3].c;
        const double mean = sf / n;
        const double var = nevents > 1 ? (sf2 / n - mean * mean) / (n - 1.0) : 0.0;
        out->mean = mean;
        out->var_mean = var;
        out->sum_f = sf;
        out->sum_f2 = sf2;
        out->sum_w = sw;
        out->sum_w2 = sw2;
        out->n = nevents;
    }
}

}  // namespace hydra
