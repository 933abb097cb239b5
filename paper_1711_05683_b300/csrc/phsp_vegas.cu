// phsp_vegas.cu -- VEGAS importance sampling over the Raubold-Lynch variables (section 3,
// "self-adaptive importance sampling"; section 4.1; G. P. Lepage, J. Comput. Phys. 27 (1978)
// 192).  The integrand is F(u) = w(u) |ME|^2(event(u)) on the unit cube of the D = 3n-4
// variables of one event (n-2 intermediate-mass uniforms, then one (cos theta, phi) pair per
// top-down two-body step), so that Int F du = Int |ME|^2 dR_n.  Each dimension has a grid of
// K bins refined after every iteration; sampling, kinematics, sums and the grid refinement all
// run on the GPU (FP64: native or double-float, hydra_set_fp64_arith).
//
// Per iteration i (Philox stream i + 1):
//   vegas_eval  point s: y_d = (x + 1/2) 2^-32 from Philox word d%4 of counter (s low, s high,
//               d/4, i + 1); bin and position from exact integers (below); the event's
//               weight and |ME|^2; f = F(u) J and the point's D bins (one byte each, four
//               to a word: word q of point s at [q][calls]) stored;
//               the deterministic tile sums of f and f^2 (the integral's group / tile /
//               segment tree, with tiles of 512 points); the largest f^2.
//   vegas_hist  per-bin sums of f^2 in 64-bit fixed point (order-independent integer adds)
//               from the stored values and bins.
//   vegas_refine  refinement of every dimension's grid and cells (one block per dimension).
//   host        the per-iteration estimates and variances (copied back without waiting) and
//               their combination, after one synchronisation at the end.
//
// Grid arithmetic.  With P = (2x + 1) K (< 2^41), the bin is b = floor(y K) = P >> 33 and the
// position inside it is y K - b = rho 2^-33 with rho = P mod 2^33, both exact (y K has at
// most 42 significant bits, so these are also what an FP64 evaluation of floor(y K) and
// y K - b gives).  Edges are held as 64-bit fixed point G_b = g_b 2^64 (G_K = 2^64 - 1) and
// widths W_b = G_{b+1} - G_b, so u 2^64 = G_b + floor(rho W_b 2^-33) to within one unit of
// 2^-64; the Jacobian factor K (g_{b+1} - g_b) is the host's FP64 value.  A cell is 16 bytes
// (K + 1 per dimension in shared memory).  Sorting the mass variables and forming the kinetic
// gaps T (r_k - r_{k-1}) work on exact integers, as in the generator.
#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>
#include "hydra_phsp.h"
#include "phsp_device.cuh"
#include "phsp_df.cuh"
#include "phsp_host.h"
#include "phsp_integral.cuh"

namespace hydra {

__global__ void eval_reduce_segments(const TileSums* __restrict__ partials, uint64_t ntiles, uint64_t seg_begin,
                                     double* __restrict__ seg_out);
__global__ void eval_finalize(const double* __restrict__ seg, uint64_t nseg, uint64_t nevents,
                              hydra_integral* __restrict__ out);

constexpr int kVegasMaxCells = 6144;  // D * K bins (D * (K + 1) cells of 16 B in shared memory)
constexpr int kVegasMaxD = 3 * kNMax - 4;
constexpr int kVegasBlock = 256;
// A VEGAS tile is 512 points (16 per lane, two groups of 8): a quarter of the integral's tile,
// because a VEGAS point over the 3n - 4 variables costs up to ~2500 instructions (n = 10) and
// an iteration of 1e7 points must still spread over every resident warp several times (with
// 2048-point tiles it was 1.4 waves of warps, run as two rounds).
constexpr int kVegasTileEvents = 512;
constexpr int kVegasLaneIters = kVegasTileEvents / 32;
static_assert(kVegasLaneIters % kGroupEvents == 0, "groups tile the lane's points");
constexpr uint64_t kVegasChunkTiles = kChunkTiles * (kTileEvents / kVegasTileEvents);  // 2^26 points per launch
static_assert(kVegasChunkTiles % kSegTiles == 0, "a chunk holds whole segments");
constexpr int kVegasMaxChunks = static_cast<int>((1ull << 36) / (kVegasChunkTiles * kVegasTileEvents));  // tile counters

struct VegasCell {
    uint64_t G;  // left edge g_b 2^64 (the cell after the last bin holds 2^64 - 1)
    double J;    // Jacobian factor K (g_{b+1} - g_b)
};
static_assert(sizeof(VegasCell) == 16, "cells are 16 bytes");

// Matrix-element constants (m0a^2, m0a Ga, m0b^2, m0b Gb, Re c, Im c) in FP64 and as
// double-float pairs.
struct VegasME {
    double v[6];
    float hi[6], lo[6];
};

template <typename R> struct VegasArith;

// Native FP64: u = U 2^-64 rounded to double.
template <> struct VegasArith<double> {
    __device__ static double frac(uint64_t v) { return __ull2double_rn(v) * 5.42101086242752217003726400434970855712890625e-20; }
    __device__ static double comp(uint64_t v) { return v == 0 ? 1.0 : frac(0 - v); }  // 1 - v 2^-64
    __device__ static void sincos(uint64_t v, double* s, double* c) { sincospi(2.0 * frac(v), s, c); }
    __device__ static double T(const DecayConsts& C) { return C.Ts * 4294967296.0; }
    __device__ static double me(const VegasME& P, int i) { return P.v[i]; }
    __device__ static double to_double(double x) { return x; }
};

template <> struct VegasArith<df> {
    __device__ static df frac(uint64_t v) { return df_frac_u64(v); }
    __device__ static df comp(uint64_t v) { return v == 0 ? df{1.0f, 0.0f} : df_frac_u64(0 - v); }
    // phi = 2 pi v 2^-64 = 2 pi (X + 1/2) 2^-32 + delta, X = v >> 32, delta = 2 pi 2^-64 (L - 2^31)
    // with L the low 32 bits (|delta| <= pi 2^-32): the table sin/cos of the first angle, then
    // sin(a + delta) = s + c delta, cos(a + delta) = c - s delta (the delta^2 terms are below
    // 3e-19).
    __device__ static void sincos(uint64_t v, df* s, df* c) {
        df s0, c0;
        df_sincos_2pi_u(static_cast<uint32_t>(v >> 32), s_sincos_table, &s0, &c0);
        const float delta = __fmul_rn(__int2float_rn(static_cast<int32_t>(static_cast<uint32_t>(v) ^ 0x80000000u)),
                                      3.40612158008655459e-19f);
        *s = df_add_f(s0, __fmul_rn(c0.hi, delta));
        *c = df_add_f(c0, -__fmul_rn(s0.hi, delta));
    }
    __device__ static df T(const DecayConsts& C) { return df_scale(Prec<df>::Ts(C), 4294967296.0f); }
    __device__ static df me(const VegasME& P, int i) { return df{P.hi[i], P.lo[i]}; }
    __device__ static double to_double(df x) { return df_to_double(x); }
};

// Raubold-Lynch event of fixed-point uniforms U[0..3n-5] in arithmetic R (the generator's
// construction: sorted mass variables, exact integer gaps, factorised Kallen lambda, top-down
// pure boosts).  Returns the weight (FP64, C_n included); E1 = lab energy of daughter 1 and
// M2 = mass of the (1, 2) subsystem, which fix s12 and s23.
template <int N, typename R>
__device__ __forceinline__ double vegas_event(const DecayConsts& C, const uint64_t (&U)[3 * N - 4], R& E1, R& M2) {
    using P = Prec<R>;
    using A = VegasArith<R>;
    constexpr int kY = N > 2 ? N - 2 : 1;
    uint64_t y[kY];
#pragma unroll
    for (int j = 0; j < N - 2; ++j) y[j] = U[j];
    if constexpr (N > 3) sort_mass_draws<N - 2>(y);
    const R M = P::M(C);
    const R T = A::T(C);
    typename P::Wacc w = P::w_one();
    R Q0 = M, Qx = R(0.0f), Qy = R(0.0f), Qz = R(0.0f), Mnext = M;
    M2 = M;
#pragma unroll
    for (int k = N - 1; k >= 1; --k) {
        const int j = N - 1 - k;
        R Mk;
        if (k == 1) Mk = P::m(C, 0);
        else Mk = P::fma_(A::frac(y[k - 2]), T, P::mu(C, k - 1));
        if (k == 2) M2 = Mk;
        R gap;
        if constexpr (N == 2) gap = T;
        else if (k == 1) gap = A::frac(y[0]) * T;
        else if (k == N - 1) gap = A::comp(y[kY - 1]) * T;
        else gap = A::frac(y[k - 1] - y[k - 2]) * T;
        const R mk1 = P::m(C, k);
        const R twoMk = P::scale(Mk, 2.0f), twom = P::scale(mk1, 2.0f);
        const R a = gap + twoMk;
        const R gm = gap * (gap + twom);  // Delta (Delta + 2 m_{k+1})
        const R lam = (gm * a) * (a + twom);
        const R invM = P::rcp(Mnext);
        const R halfInvM = P::scale(invM, 0.5f);
        const R p = P::sqrt_(lam) * halfInvM;
        w = P::w_mul(w, p);
        const uint64_t uc = U[N - 2 + 2 * j], up = U[N - 1 + 2 * j];
        const R one_p = P::scale(A::frac(uc), 2.0f);  // 1 + cos(theta) = 2u
        const R one_m = P::scale(A::comp(uc), 2.0f);  // 1 - cos(theta) = 2(1 - u)
        const R cos_t = A::frac(uc) - A::comp(uc);            // 2u - 1
        const R sin_t = P::sqrt_(one_m * one_p);
        R sphi, cphi;
        A::sincos(up, &sphi, &cphi);
        const R ps = p * sin_t;
        const R px = ps * cphi, py = ps * sphi, pz = p * cos_t;
        const R Es = P::fma_(gm, halfInvM, Mk);  // (M_{k+1}^2 + M_k^2 - m_{k+1}^2) / (2 M_{k+1})
        if (k == N - 1) {
            Q0 = Es; Qx = px; Qy = py; Qz = pz;
        } else {
            const R qp = P::fma_(Qz, pz, P::fma_(Qy, py, Qx * px));
            const R E1v = P::fma_(Q0, Es, qp) * invM;
            const R f = P::div(E1v + Es, Q0 + Mnext);
            Qx = P::fma_(f, Qx, px);
            Qy = P::fma_(f, Qy, py);
            Qz = P::fma_(f, Qz, pz);
            Q0 = E1v;
        }
        Mnext = Mk;
    }
    E1 = Q0;
    return P::w_final(w, C);
}

// The N = 3 event of the same uniforms in closed form (the integrand's construction): the
// weight, M2 and the lab energy E1 of daughter 1 without the event's 4-vectors.  Step 1 (parent
// -> (12) + 3): gap T (1 - u0), momentum p2, direction n_a from (U1, U2); step 2 ((12) -> 1 + 2):
// gap T u0, momentum p1, direction n_b from (U3, U4).  With the two-body energies from the gap
// factors of lambda, Q0 = M2 + D2 (D2 + 2 m3) / (2 M) and E1* = m1 + D1 (D1 + 2 m2) / (2 M2),
// the pure boost gives E1 = (Q0 E1* + p2 p1 n_a.n_b) / M2 with
// n_a.n_b = c_a c_b + s_a s_b cos(phi_a - phi_b), the angle difference from U2 - U4 (mod 2^64).
template <typename R>
__device__ __forceinline__ double vegas_event3(const DecayConsts& C, const uint64_t (&U)[5], R& E1, R& M2) {
    using P = Prec<R>;
    using A = VegasArith<R>;
    const R M = P::M(C), T = A::T(C);
    const R m1 = P::m(C, 0), m2 = P::m(C, 1), m3 = P::m(C, 2);
    M2 = P::fma_(A::frac(U[0]), T, P::mu(C, 1));
    const R gap2 = A::comp(U[0]) * T, gap1 = A::frac(U[0]) * T;
    const R twoM2 = P::scale(M2, 2.0f), twom3 = P::scale(m3, 2.0f);
    const R a2 = gap2 + twoM2, g2 = gap2 * (gap2 + twom3);
    const R twom1 = P::scale(m1, 2.0f), twom2 = P::scale(m2, 2.0f);
    const R a1 = gap1 + twom1, g1 = gap1 * (gap1 + twom2);
    const R invM2 = P::rcp(M2);
    const R halfInvM = P::scale(P::rcp(M), 0.5f), halfInvM2 = P::scale(invM2, 0.5f);
    const R p2 = P::sqrt_((g2 * a2) * (a2 + twom3)) * halfInvM;
    const R p1 = P::sqrt_((g1 * a1) * (a1 + twom2)) * halfInvM2;
    const R ca = A::frac(U[1]) - A::comp(U[1]), cb = A::frac(U[3]) - A::comp(U[3]);
    const R sab2 = (P::scale(A::comp(U[1]), 2.0f) * P::scale(A::frac(U[1]), 2.0f)) *
                   (P::scale(A::comp(U[3]), 2.0f) * P::scale(A::frac(U[3]), 2.0f));
    R sd, cd;
    A::sincos(U[2] - U[4], &sd, &cd);
    const R cos_alpha = P::fma_(ca, cb, P::sqrt_(sab2) * cd);
    const R Q0 = P::fma_(g2, halfInvM, M2);
    const R E1s = P::fma_(g1, halfInvM2, m1);
    E1 = P::fma_(Q0, E1s, (p2 * p1) * cos_alpha) * invM2;
    return P::w_final(P::w_mul(P::w_mul(P::w_one(), p2), p1), C);
}

// |BW(s12; a) + c BW(s23; b)|^2 in arithmetic R (the integral's formula).
template <typename R>
__device__ __forceinline__ R vegas_dalitz(const VegasME& PM, R s12, R s23) {
    using A = VegasArith<R>;
    using Q = Prec<R>;
    const R xa = A::me(PM, 0) - s12, ya = A::me(PM, 1);
    const R xb = A::me(PM, 2) - s23, yb = A::me(PM, 3);
    const R ia = Q::rcp(Q::fma_(xa, xa, ya * ya));
    const R ib = Q::rcp(Q::fma_(xb, xb, yb * yb));
    const R cr = A::me(PM, 4), ci = A::me(PM, 5);
    const R re = Q::fma_(xa, ia, Q::fma_(cr, xb, -(ci * yb)) * ib);
    const R im = Q::fma_(ya, ia, Q::fma_(cr, yb, ci * xb) * ib);
    return Q::fma_(re, re, im * im);
}

// Bins of point s: calls visit(d, b, rho) for d = 0..D-1 (one Philox block per four
// dimensions), b = P >> 33 and rho = P mod 2^33 with P = (2x + 1) K.
template <typename Visit>
__device__ __forceinline__ void vegas_bins(const DecayConsts& C, uint64_t s, uint32_t stream, int D, int K,
                                           Visit visit) {
#pragma unroll
    for (int q = 0; q < (D + 3) / 4; ++q) {
        uint32_t x[4];
        philox4x32_10(static_cast<uint32_t>(s), static_cast<uint32_t>(s >> 32), static_cast<uint32_t>(q), stream,
                      C.rk0, C.rk1, x);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int d = 4 * q + j;
            if (d < D) {
                const uint64_t Pv = (2ull * x[j] + 1ull) * static_cast<uint64_t>(K);
                visit(d, static_cast<int>(Pv >> 33), Pv & 0x1FFFFFFFFull);
            }
        }
    }
}

template <int N, typename R, int ME>
__global__ void __launch_bounds__(kVegasBlock) vegas_eval(const __grid_constant__ DecayConsts C,
                                                          const __grid_constant__ VegasME PM,
                                                          const VegasCell* __restrict__ grid, int K, uint32_t stream,
                                                          uint64_t calls, uint64_t tile_begin, uint64_t ntiles,
                                                          TileSums* __restrict__ partials, double* __restrict__ fvals,
                                                          uint32_t* __restrict__ bins,
                                                          unsigned long long* __restrict__ max_f2,
                                                          unsigned int* __restrict__ next_tile) {
    constexpr int D = 3 * N - 4;
    extern __shared__ VegasCell cells[];
    if constexpr (std::is_same_v<R, df>) df_sincos_table_init();
    for (int i = threadIdx.x; i < D * (K + 1); i += blockDim.x) cells[i] = grid[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    unsigned long long mx = 0;
    // Tiles are taken from a counter (a persistent grid stays balanced across SMs whatever
    // the tile count); each tile's sums land at its own index, so the result does not depend
    // on which warp took it.
    for (;;) {
        unsigned int tn = 0;
        if (lane == 0) tn = atomicAdd(next_tile, 1u);
        const uint64_t t = __shfl_sync(0xffffffffu, tn, 0);
        if (t >= ntiles) break;
        const uint64_t base = (tile_begin + t) * kVegasTileEvents;
        double af = 0.0, af2 = 0.0;
        for (int g = 0; g < kVegasLaneIters / kGroupEvents; ++g) {
            double sf = 0.0, sf2 = 0.0;
            for (int i = 0; i < kGroupEvents; ++i) {
                const uint64_t s = base + static_cast<uint64_t>(32 * (g * kGroupEvents + i) + lane);
                if (s < calls) {
                    uint64_t U[D];
                    uint32_t packed[(D + 3) / 4] = {};
                    double jac = 1.0;
                    vegas_bins(C, s, stream, D, K, [&](int d, int b, uint64_t rho) {
                        packed[d / 4] |= static_cast<uint32_t>(b) << (8 * (d % 4));
                        const VegasCell c = cells[d * (K + 1) + b];
                        const uint64_t W = cells[d * (K + 1) + b + 1].G - c.G;
                        U[d] = c.G + ((__umul64hi(rho, W) << 31) | ((rho * W) >> 33));
                        jac *= c.J;
                    });
#pragma unroll
                    for (int q = 0; q < (D + 3) / 4; ++q) bins[static_cast<uint64_t>(q) * calls + s] = packed[q];
                    R E1, M2;
                    double w;
                    if constexpr (ME == HYDRA_ME_DALITZ_2BW && N == 3) w = vegas_event3<R>(C, U, E1, M2);
                    else w = vegas_event<N, R>(C, U, E1, M2);
                    double me2 = 1.0;
                    if constexpr (ME == HYDRA_ME_DALITZ_2BW) {
                        // s12 = M_2^2; s23 = (P - p1)^2 = M^2 + m1^2 - 2 M E1
                        const R M = Prec<R>::M(C);
                        const R s12 = M2 * M2;
                        const R s23 = Prec<R>::fma_(Prec<R>::scale(M, -2.0f), E1,
                                                    Prec<R>::fma_(M, M, Prec<R>::m2(C, 0)));
                        me2 = VegasArith<R>::to_double(vegas_dalitz<R>(PM, s12, s23));
                    }
                    const double f = (w * me2) * jac;
                    fvals[s] = f;
                    sf += f;
                    sf2 = __fma_rn(f, f, sf2);
                    const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(f * f));
                    mx = bits > mx ? bits : mx;
                }
            }
            af += sf;
            af2 += sf2;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            af += __shfl_xor_sync(0xffffffffu, af, off);
            af2 += __shfl_xor_sync(0xffffffffu, af2, off);
        }
        if (lane == 0) partials[t] = TileSums{af, af2, 0.0, 0.0};
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, off);
        mx = o > mx ? o : mx;
    }
    if (lane == 0) atomicMax(max_f2, mx);
}

// Per-bin sums of f^2 in 64-bit fixed point, one unit = (largest f^2 of the iteration) / qnum
// with qnum = 2^(62 - ceil(log2 calls)), so no bin can overflow: integer additions are order
// independent, so the histogram and the refined grid are reproducible bit for bit.
template <int D>
__global__ void __launch_bounds__(kVegasBlock) vegas_hist(int K, uint64_t calls, double qnum,
                                                          const double* __restrict__ fvals,
                                                          const uint32_t* __restrict__ bins,
                                                          const unsigned long long* __restrict__ max_f2,
                                                          unsigned long long* __restrict__ hist) {
    constexpr int kWords = (D + 3) / 4;
    // each bin's 64-bit sum as two 32-bit words: the low word's atomic returns the old value,
    // from which the carry into the high word follows (exact modulo 2^64, so the same integer
    // sums as 64-bit atomics, mostly with one 32-bit atomic per update)
    extern __shared__ uint32_t sh32[];
    uint32_t* lo = sh32;
    uint32_t* hi = sh32 + D * K;
    for (int i = threadIdx.x; i < 2 * D * K; i += blockDim.x) sh32[i] = 0u;
    __syncthreads();
    const double mx = __longlong_as_double(static_cast<long long>(*max_f2));
    const double scale = mx > 0.0 ? qnum / mx : 0.0;
    for (uint64_t s = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < calls;
         s += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const double f = fvals[s];
        uint32_t wd[kWords];
#pragma unroll
        for (int q = 0; q < kWords; ++q) wd[q] = bins[static_cast<uint64_t>(q) * calls + s];
        const unsigned long long qf = static_cast<unsigned long long>(f * f * scale);
        if (qf == 0ull) continue;
        const uint32_t ql = static_cast<uint32_t>(qf), qh = static_cast<uint32_t>(qf >> 32);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int i = d * K + static_cast<int>((wd[d / 4] >> (8 * (d % 4))) & 0xFFu);
            const uint32_t old = atomicAdd(&lo[i], ql);
            const uint32_t up = qh + (old + ql < old ? 1u : 0u);
            if (up) atomicAdd(&hi[i], up);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < D * K; i += blockDim.x) {
        const unsigned long long v = (static_cast<unsigned long long>(hi[i]) << 32) | lo[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

static const void* vegas_hist_for(int n) {
    switch (n) {
        case 2: return reinterpret_cast<const void*>(&vegas_hist<2>);
        case 3: return reinterpret_cast<const void*>(&vegas_hist<5>);
        case 4: return reinterpret_cast<const void*>(&vegas_hist<8>);
        case 5: return reinterpret_cast<const void*>(&vegas_hist<11>);
        case 6: return reinterpret_cast<const void*>(&vegas_hist<14>);
        case 7: return reinterpret_cast<const void*>(&vegas_hist<17>);
        case 8: return reinterpret_cast<const void*>(&vegas_hist<20>);
        case 9: return reinterpret_cast<const void*>(&vegas_hist<23>);
        case 10: return reinterpret_cast<const void*>(&vegas_hist<26>);
    }
    return nullptr;
}

template <typename R, int ME>
static const void* vegas_eval_for(int n) {
    if constexpr (ME == HYDRA_ME_DALITZ_2BW) {
        return n == 3 ? reinterpret_cast<const void*>(&vegas_eval<3, R, ME>) : nullptr;
    } else {
        switch (n) {
            case 2: return reinterpret_cast<const void*>(&vegas_eval<2, R, ME>);
            case 3: return reinterpret_cast<const void*>(&vegas_eval<3, R, ME>);
            case 4: return reinterpret_cast<const void*>(&vegas_eval<4, R, ME>);
            case 5: return reinterpret_cast<const void*>(&vegas_eval<5, R, ME>);
            case 6: return reinterpret_cast<const void*>(&vegas_eval<6, R, ME>);
            case 7: return reinterpret_cast<const void*>(&vegas_eval<7, R, ME>);
            case 8: return reinterpret_cast<const void*>(&vegas_eval<8, R, ME>);
            case 9: return reinterpret_cast<const void*>(&vegas_eval<9, R, ME>);
            case 10: return reinterpret_cast<const void*>(&vegas_eval<10, R, ME>);
        }
        return nullptr;
    }
}

// Refinement of every dimension on the device (one block per dimension): smoothed bin sums (1,2,1)/4 inside and (1,1)/2 at the ends,
// weights ((r - 1)/ln r)^alpha of each bin's share r, and new edges at equal shares of the
// total weight, linear inside a bin; then the dimension's fixed-point cells.  The sums and the
// redistribution run on one thread in bin order, the weights on one thread per bin, so the
// grid is the host rule's to the last bit of pow and log.  No refinement when K = 1 or all
// sums are zero.  (On the host this took ~0.15 ms per iteration at 26 x 100 bins, plus a
// synchronisation: a tenth of a 1e7-point N = 10 iteration.)
__global__ void __launch_bounds__(256) vegas_refine(int K, double alpha, const unsigned long long* __restrict__ hist,
                                                    double* __restrict__ grid, VegasCell* __restrict__ cells) {
    __shared__ double sm[256], wt[256], g[257], ng[257];
    __shared__ double tot_s;
    const int d = blockIdx.x;
    const unsigned long long* hd = hist + static_cast<size_t>(d) * K;
    double* gd = grid + static_cast<size_t>(d) * (K + 1);
    VegasCell* cd = cells + static_cast<size_t>(d) * (K + 1);
    for (int t = threadIdx.x; t <= K; t += blockDim.x) g[t] = gd[t];
    if (K > 1) {
        for (int t = threadIdx.x; t < K; t += blockDim.x) {
            const double c = static_cast<double>(hd[t]);
            if (t == 0) sm[t] = (c + static_cast<double>(hd[1])) / 2.0;
            else if (t == K - 1) sm[t] = (static_cast<double>(hd[K - 2]) + c) / 2.0;
            else sm[t] = (static_cast<double>(hd[t - 1]) + 2.0 * c + static_cast<double>(hd[t + 1])) / 4.0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int t = 0; t < K; ++t) tot += sm[t];
            tot_s = tot;
        }
        __syncthreads();
        const double tot = tot_s;
        if (tot > 0.0) {
            for (int t = threadIdx.x; t < K; t += blockDim.x) {
                const double r = sm[t] / tot;
                wt[t] = (r > 0.0 && r < 1.0) ? pow((r - 1.0) / log(r), alpha) : (r >= 1.0 ? 1.0 : 0.0);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double wsum = 0.0;
                for (int t = 0; t < K; ++t) wsum += wt[t];
                if (wsum > 0.0) {
                    const double share = wsum / K;
                    double acc = 0.0;
                    int j = 0;
                    ng[0] = 0.0;
                    for (int i = 1; i < K; ++i) {
                        const double need = share * i;
                        while (j < K - 1 && acc + wt[j] < need) acc += wt[j++];
                        double frac = wt[j] > 0.0 ? (need - acc) / wt[j] : 0.0;
                        frac = frac < 0.0 ? 0.0 : (frac > 1.0 ? 1.0 : frac);
                        ng[i] = g[j] + frac * (g[j + 1] - g[j]);
                    }
                    ng[K] = 1.0;
                    for (int i = 0; i <= K; ++i) g[i] = ng[i];
                }
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t <= K; t += blockDim.x) {
        gd[t] = g[t];
        if (t < K) {
            cd[t].G = g[t] < 1.0 ? static_cast<uint64_t>(ldexp(g[t], 64)) : ~uint64_t{0};  // exact below 2^64
            cd[t].J = K * (g[t + 1] - g[t]);
        } else {
            cd[t].G = ~uint64_t{0};
            cd[t].J = 0.0;
        }
    }
}

// Fixed-point cells of one dimension's edges g[0..K] (K + 1 cells).
static void grid_cells(const double* g, int K, VegasCell* out) {
    for (int b = 0; b < K; ++b) {
        out[b].G = g[b] < 1.0 ? static_cast<uint64_t>(std::ldexp(g[b], 64)) : ~uint64_t{0};  // exact below 2^64
        out[b].J = K * (g[b + 1] - g[b]);
    }
    out[K].G = ~uint64_t{0};  // 2^64 - 1: the last width is short by 2^-64
    out[K].J = 0.0;
}

struct VegasScratch {
    std::mutex mu;
    TileSums* tiles = nullptr;
    double* segs = nullptr;
    uint64_t seg_cap = 0;
    double* fvals = nullptr;
    uint32_t* bins = nullptr;  // [ceil(D/4)][calls]
    uint64_t fcap = 0;
    int bins_d = 0;
    VegasCell* cells = nullptr;
    double* grid = nullptr;              // [D][K+1] edges (refined on the device)
    unsigned long long* hist = nullptr;  // [D*K] bin sums, the largest f^2 (as bits), tile counters
    hydra_integral* d_res = nullptr;
    void* h_pin = nullptr;               // pinned: result, histogram, cells
    hydra_integral* h_res_all = nullptr; // pinned: every iteration's result
    int res_cap = 0;
};
static std::mutex g_vg_mu;
static std::vector<VegasScratch*> g_vg;

static VegasScratch* vegas_scratch() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_vg_mu);
    if (static_cast<int>(g_vg.size()) <= dev) g_vg.resize(dev + 1, nullptr);
    if (!g_vg[dev]) g_vg[dev] = new VegasScratch();
    return g_vg[dev];
}

// Frees the VEGAS scratch of every device (hydra_shutdown).
void release_vegas_scratch() {
    int cur = 0;
    cudaGetDevice(&cur);
    std::lock_guard<std::mutex> lk(g_vg_mu);
    for (size_t d = 0; d < g_vg.size(); ++d) {
        VegasScratch* s = g_vg[d];
        if (!s) continue;
        cudaSetDevice(static_cast<int>(d));
        if (s->tiles) cudaFree(s->tiles);
        if (s->segs) cudaFree(s->segs);
        if (s->fvals) cudaFree(s->fvals);
        if (s->bins) cudaFree(s->bins);
        if (s->cells) cudaFree(s->cells);
        if (s->grid) cudaFree(s->grid);
        if (s->hist) cudaFree(s->hist);
        if (s->d_res) cudaFree(s->d_res);
        if (s->h_pin) cudaFreeHost(s->h_pin);
        if (s->h_res_all) cudaFreeHost(s->h_res_all);
        delete s;
        g_vg[d] = nullptr;
    }
    cudaSetDevice(cur);
}

}  // namespace hydra

using namespace hydra;

extern "C" {

hydra_status hydra_phsp_vegas(double M, int n, const double* masses, uint64_t seed, hydra_me_id me, const double* params,
                              int nparams, uint64_t calls, int iterations, int bins, double alpha, int skip,
                              double* est, double* var, double* result, double* grid_out, hydra_stream_t stream) {
    const NvtxRange nvtx_range("hydra_phsp_vegas");
    DecayConsts C;
    hydra_status st = make_consts(M, n, masses, seed, &C);
    if (st != HYDRA_OK) return st;
    MEConsts P;
    st = make_me(me, n, params, nparams, &P);
    if (st != HYDRA_OK) return st;
    const int D = 3 * n - 4, K = bins;
    if (iterations < 1 || calls < 2 || calls > (uint64_t{1} << 36) || !est || !var || !result)
        return fail(HYDRA_ERR_INVALID_ARG, "need iterations >= 1, 2 <= calls <= 2^36 and est/var/result arrays");
    if (K < 1 || K > 256 || D * K > kVegasMaxCells)
        return fail(HYDRA_ERR_INVALID_ARG, "bins = %d: need 1 <= bins <= 256 and (3n-4) bins <= %d", K, kVegasMaxCells);
    if (!(alpha >= 0.0) || skip < 0 || skip >= iterations) return fail(HYDRA_ERR_INVALID_ARG, "bad alpha or skip");
    const bool use_df = g_fp64_arith.load() == HYDRA_FP64_DOUBLE_FLOAT;
    const void* kern = use_df ? (me == HYDRA_ME_FLAT ? vegas_eval_for<df, HYDRA_ME_FLAT>(n)
                                                     : vegas_eval_for<df, HYDRA_ME_DALITZ_2BW>(n))
                              : (me == HYDRA_ME_FLAT ? vegas_eval_for<double, HYDRA_ME_FLAT>(n)
                                                     : vegas_eval_for<double, HYDRA_ME_DALITZ_2BW>(n));
    if (!kern) return fail(HYDRA_ERR_UNSUPPORTED_N, "no VEGAS kernel for n = %d", n);
    VegasME PM;
    const double pv[6] = {P.a_m2, P.a_mg, P.b_m2, P.b_mg, P.c_re, P.c_im};
    for (int i = 0; i < 6; ++i) {
        PM.v[i] = pv[i];
        PM.hi[i] = static_cast<float>(pv[i]);
        PM.lo[i] = static_cast<float>(pv[i] - static_cast<double>(PM.hi[i]));
    }
    VegasScratch* s = vegas_scratch();
    if (!s) return fail(HYDRA_ERR_CUDA, "no current CUDA device");
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t ntiles = (calls + kVegasTileEvents - 1) / kVegasTileEvents;
    const uint64_t nseg = (ntiles + kSegTiles - 1) / kSegTiles;
    const size_t hist_words = static_cast<size_t>(kVegasMaxCells) + 1 + kVegasMaxChunks;
    const size_t cell_bytes = static_cast<size_t>(kVegasMaxCells + kVegasMaxD) * sizeof(VegasCell);
    if (!s->tiles) {
        if (cudaMalloc(&s->tiles, kVegasChunkTiles * sizeof(TileSums)) != cudaSuccess ||
            cudaMalloc(&s->cells, cell_bytes) != cudaSuccess ||
            cudaMalloc(&s->grid, static_cast<size_t>(kVegasMaxCells + kVegasMaxD) * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&s->hist, hist_words * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMalloc(&s->d_res, sizeof(hydra_integral)) != cudaSuccess ||
            cudaMallocHost(&s->h_pin, sizeof(hydra_integral) + hist_words * sizeof(unsigned long long) + cell_bytes) !=
                cudaSuccess) {
            cudaGetLastError();
            return fail(HYDRA_ERR_OOM, "VEGAS scratch");
        }
    }
    if (nseg > s->seg_cap) {
        if (s->segs) cudaFree(s->segs);
        s->segs = nullptr;
        s->seg_cap = 0;
        if (cudaMalloc(&s->segs, nseg * 8 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(HYDRA_ERR_OOM, "VEGAS segment scratch");
        }
        s->seg_cap = nseg;
    }
    if (calls > s->fcap || D > s->bins_d) {
        const uint64_t cap = calls > s->fcap ? calls : s->fcap;
        const int dcap = D > s->bins_d ? D : s->bins_d;
        if (s->fvals) cudaFree(s->fvals);
        if (s->bins) cudaFree(s->bins);
        s->fvals = nullptr;
        s->bins = nullptr;
        s->fcap = 0;
        s->bins_d = 0;
        if (cudaMalloc(&s->fvals, cap * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&s->bins, cap * static_cast<uint64_t>((dcap + 3) / 4) * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return fail(HYDRA_ERR_OOM, "VEGAS point values and bins (%llu calls, %d dimensions)",
                        static_cast<unsigned long long>(calls), D);
        }
        s->fcap = cap;
        s->bins_d = dcap;
    }
    if (iterations > s->res_cap) {
        if (s->h_res_all) cudaFreeHost(s->h_res_all);
        s->h_res_all = nullptr;
        s->res_cap = 0;
        if (cudaMallocHost(&s->h_res_all, static_cast<size_t>(iterations) * sizeof(hydra_integral)) != cudaSuccess) {
            cudaGetLastError();
            return fail(HYDRA_ERR_OOM, "VEGAS results (%d iterations)", iterations);
        }
        s->res_cap = iterations;
    }
    const size_t smem = static_cast<size_t>(D) * (K + 1) * sizeof(VegasCell);
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(cell_bytes));
    if (err != cudaSuccess) return cuda_fail(err, "VEGAS shared-memory limit");
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kVegasBlock, smem);
    per_sm = per_sm < 1 ? 1 : per_sm;
    std::vector<double> g(static_cast<size_t>(D) * (K + 1));
    for (int d = 0; d < D; ++d)
        for (int b = 0; b <= K; ++b) g[static_cast<size_t>(d) * (K + 1) + b] = static_cast<double>(b) / K;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* h_hist = reinterpret_cast<unsigned long long*>(static_cast<char*>(s->h_pin) + sizeof(hydra_integral));
    VegasCell* h_cells = reinterpret_cast<VegasCell*>(h_hist + hist_words);
    unsigned long long* d_max = s->hist + kVegasMaxCells;
    int lg = 0;
    while ((uint64_t{1} << lg) < calls) ++lg;
    const double qnum = std::ldexp(1.0, 62 - lg);
    // the uniform grid and its cells; later grids are refined on the device
    for (int d = 0; d < D; ++d)
        grid_cells(&g[static_cast<size_t>(d) * (K + 1)], K, h_cells + static_cast<size_t>(d) * (K + 1));
    err = cudaMemcpyAsync(s->cells, h_cells, smem, cudaMemcpyHostToDevice, cs);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(s->grid, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice, cs);
    if (err != cudaSuccess) return cuda_fail(err, "VEGAS grid upload");
    for (int it = 0; it < iterations; ++it) {
        const uint32_t stream_id = static_cast<uint32_t>(it + 1);
        err = cudaMemsetAsync(s->hist, 0, hist_words * sizeof(unsigned long long), cs);
        if (err != cudaSuccess) return cuda_fail(err, "VEGAS histogram reset");
        for (uint64_t t0 = 0; t0 < ntiles; t0 += kVegasChunkTiles) {
            const uint64_t nt = ntiles - t0 < kVegasChunkTiles ? ntiles - t0 : kVegasChunkTiles;
            const uint64_t need = (nt * 32 + kVegasBlock - 1) / kVegasBlock;
            const uint64_t cap = static_cast<uint64_t>(sms) * per_sm;  // one persistent wave
            const unsigned grid = static_cast<unsigned>(need < cap ? need : cap);
            const VegasCell* gp = s->cells;
            int Kv = K;
            uint32_t sid = stream_id;
            uint64_t cl = calls, tb = t0, ntv = nt;
            TileSums* tp = s->tiles;
            double* fv = s->fvals;
            uint32_t* bp = s->bins;
            unsigned long long* mp = d_max;
            unsigned int* ctr = reinterpret_cast<unsigned int*>(d_max + 1 + t0 / kVegasChunkTiles);
            void* args[] = {&C, &PM, &gp, &Kv, &sid, &cl, &tb, &ntv, &tp, &fv, &bp, &mp, &ctr};
            err = cudaLaunchKernel(kern, dim3(grid), dim3(kVegasBlock), args, smem, cs);
            if (err != cudaSuccess) return cuda_fail(err, "VEGAS evaluation launch");
            const uint64_t ns = (nt + kSegTiles - 1) / kSegTiles;
            eval_reduce_segments<<<static_cast<unsigned>(ns), kSegBlock, 0, cs>>>(s->tiles, nt, t0 / kSegTiles, s->segs);
        }
        eval_finalize<<<1, 32, 0, cs>>>(s->segs, nseg, calls, s->d_res);
        if (it < iterations - 1) {
            const uint64_t hneed = (calls + kVegasBlock - 1) / kVegasBlock;
            const uint64_t hcap = static_cast<uint64_t>(sms) * 4;
            const unsigned hgrid = static_cast<unsigned>(hneed < hcap ? hneed : hcap);
            const double* fv = s->fvals;
            const uint32_t* bp = s->bins;
            const unsigned long long* mp = d_max;
            unsigned long long* hp = s->hist;
            int Kv = K;
            uint64_t cl = calls;
            double qn = qnum;
            void* hargs[] = {&Kv, &cl, &qn, &fv, &bp, &mp, &hp};
            err = cudaLaunchKernel(vegas_hist_for(n), dim3(hgrid), dim3(kVegasBlock), hargs,
                                   static_cast<size_t>(D) * K * sizeof(unsigned long long), cs);
            if (err != cudaSuccess) return cuda_fail(err, "VEGAS histogram launch");
            vegas_refine<<<static_cast<unsigned>(D), 256, 0, cs>>>(K, alpha, s->hist, s->grid, s->cells);
        }
        err = cudaGetLastError();
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(s->h_res_all + it, s->d_res, sizeof(hydra_integral), cudaMemcpyDeviceToHost, cs);
        if (err != cudaSuccess) return cuda_fail(err, "VEGAS iteration");
    }
    err = cudaStreamSynchronize(cs);
    if (err == cudaSuccess && grid_out)
        err = cudaMemcpy(grid_out, s->grid, g.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) return cuda_fail(err, "VEGAS iterations");
    double sw = 0.0, swi = 0.0, swi2 = 0.0;
    for (int it = 0; it < iterations; ++it) {
        est[it] = s->h_res_all[it].mean;
        var[it] = s->h_res_all[it].var_mean;
        if (it >= skip && var[it] > 0.0) {
            sw += 1.0 / var[it];
            swi += est[it] / var[it];
            swi2 += est[it] * est[it] / var[it];
        }
    }
    const double res = sw > 0.0 ? swi / sw : est[iterations - 1];
    const int used = iterations - skip;
    result[0] = res;
    result[1] = sw > 0.0 ? 1.0 / std::sqrt(sw) : std::sqrt(var[iterations - 1]);
    result[2] = used > 1 ? (swi2 - res * res * sw) / (used - 1) : 0.0;
    return HYDRA_OK;
}

}  // extern "C"
