// phsp_df.cuh -- double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significand bits.  On B300 the FP32
// pipe is ~64x wider than the FP64 pipe, so the FP64 generator computes its kinematics in
// df and converts to double only when it stores.
//
// Building blocks (error-free transformations):
//   TwoSum (Knuth):        s = fl(a+b), e = exact a + b - s                (6 FP32 ops)
//   FastTwoSum (Dekker):   same when |a| >= |b|                            (3 ops)
//   TwoProd (with FMA):    p = fl(a*b), e = fma(a, b, -p) exact            (2 ops)
// Addition is the "sloppy" double-word sum (TwoSum of the high parts, low parts added,
// renormalised): its error is bounded by ~2^-46 (|x| + |y|), i.e. relative to the operands,
// which is the measure the generator's tolerance uses (error at the event scale).
// Multiplication is the FMA-based double-word product (relative error ~2^-46).  Sums that
// cannot cancel, and sums whose result only feeds products, sums and the conversion to double,
// may skip the final renormalisation (df_add_lazy): the low part then exceeds ulp(hi)/2 by a
// few ulp, which products, sums and conversions absorb at ~2^-48 of the terms' scale.  The
// limit is a value carried through a chain of products and reciprocals (the boosted lab energy
// from step to step, the weight's running product): unnormalised there, its low part grows
// link by link until the product's dropped lo x lo term costs precision, so those are
// renormalised.
// Reciprocal, division and square root take an FP32 hardware approximation as the seed (of
// the pair rounded to FP32, so an unnormalised operand still gives a seed within ~1 ulp) and
// apply one Newton-Raphson correction evaluated in double-word arithmetic, which squares
// the seed's ~2^-23 relative error to ~2^-46.
//
// Range: full ~48-bit precision needs |hi| >= ~2^-100 (the low part must stay a normal
// FP32 number); values whose FP32 part underflows lose precision or flush to zero, an
// absolute error below 2^-126 -- negligible at the event scale of GeV-range kinematics.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hydra {

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h) : hi(h), lo(0.0f) {}
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}

__device__ __forceinline__ df df_from_float(float a) { return df{a, 0.0f}; }

// x + y
__device__ __forceinline__ df operator+(df x, df y) {
    const df s = df_two_sum(x.hi, y.hi);
    const float l = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return df_fast_two_sum(s.hi, l);
}

// x + y without the final renormalisation: (fl(x.hi + y.hi), its exact error + x.lo + y.lo).
// For operands that cannot cancel (both >= 0) the low part stays within a few ulp of the
// high part, which every consumer here tolerates (products and sums fold the low part in
// with its own rounding, reciprocal and square root form their residual from both parts,
// the conversion to double adds both); 3 FP32 operations fewer than operator+.  Also used
// where only the absolute error matters (sin/cos values that multiply momenta).
__device__ __forceinline__ df df_add_lazy(df x, df y) {
    const df s = df_two_sum(x.hi, y.hi);
    return df{s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}

// x + y for x, y >= 0, unnormalised like df_add_lazy.  With the larger high part first, Dekker's
// FastTwoSum yields the same exact pair (fl(x.hi + y.hi), its rounding error) as TwoSum, so the
// result is bit-identical to df_add_lazy in one FP32 instruction fewer (a max and a min on the
// ALU pipe replace two dependent additions).
__device__ __forceinline__ df df_add_pos_lazy(df x, df y) {
    const df s = df_fast_two_sum(fmaxf(x.hi, y.hi), fminf(x.hi, y.hi));
    return df{s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}

// x - y for 0 <= y <= x (up to the rounding of either), unnormalised like df_add_lazy(x, -y) and
// bit-identical to it: FastTwoSum(x.hi, -y.hi) is exact when y.hi <= x.hi, and when rounding
// leaves y.hi above x.hi the two lie within a factor of two, where the difference itself is
// exact (Sterbenz) and so is the zero error term.  Three FP32 instructions fewer than TwoSum.
__device__ __forceinline__ df df_sub_le_lazy(df x, df y) {
    const df s = df_fast_two_sum(x.hi, -y.hi);
    return df{s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, -y.lo))};
}

__device__ __forceinline__ df operator-(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }

// x * y.  The result (p, e) is left unnormalised: p = fl(x.hi y.hi) and |e| is a few ulp(p)
// (the exact rounding error of p plus the cross terms).  Every consumer takes such pairs:
// additions renormalise, products fold e into their own cross terms, and reciprocal and
// square root form their residual from both parts; the error stays ~2^-46 relative.
__device__ __forceinline__ df operator*(df x, df y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return df{p, e};
}

// x * a for an FP32 a (unnormalised like the product above)
__device__ __forceinline__ df operator*(df x, float a) {
    const float p = __fmul_rn(x.hi, a);
    float e = __fmaf_rn(x.hi, a, -p);
    e = __fmaf_rn(x.lo, a, e);
    return df{p, e};
}

// 1/y: seed r = rcp.approx(fl(hi + lo)); e = 1 - y r (exact to first order in df); r (1 + e),
// returned as the unnormalised pair (r, r e): |r e| is ~2^-23 |r| (the seed's error), every
// consumer is a product, and the pair has the value FastTwoSum would renormalise it to.
__device__ __forceinline__ df df_rcp(df y) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(__fadd_rn(y.hi, y.lo)));
    float e = __fmaf_rn(-y.hi, r, 1.0f);
    e = __fmaf_rn(-y.lo, r, e);
    return df{r, __fmul_rn(r, e)};
}

__device__ __forceinline__ df df_div(df x, df y) { return x * df_rcp(y); }

__device__ __forceinline__ df& operator*=(df& x, df y) {
    x = x * y;
    return x;
}

// sqrt(x), x >= 0: with xh = fl(hi + lo), s0 = xh rsqrt(xh); s = s0 + (x - s0^2) / (2 s0), the
// residual formed from both parts with an exact product; 0 for x = 0.  Returned as the
// unnormalised pair (s0, correction), |correction| ~2^-23 s0, like the reciprocal.
// The square root of an x known to be positive and normal (no zero test).
__device__ __forceinline__ df df_sqrt_pos(df x) {
    const float xh = __fadd_rn(x.hi, x.lo);
    float r;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(xh));
    const float s0 = __fmul_rn(xh, r);
    const float p = __fmul_rn(s0, s0);
    const float pe = __fmaf_rn(s0, s0, -p);
    const float res = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), pe), x.lo);
    return df{s0, __fmul_rn(res, __fmul_rn(0.5f, r))};
}

__device__ __forceinline__ df df_sqrt(df x) {
    if (!(__fadd_rn(x.hi, x.lo) > 0.0f)) return df{0.0f, 0.0f};
    return df_sqrt_pos(x);
}

// Exact conversion of a 32-bit unsigned / signed integer: v = (v & ~0xFF) + (v & 0xFF), both
// parts exact in FP32.  The high part is 0 or at least 256 in magnitude and the low part below
// 256, so Dekker's FastTwoSum gives the same exact pair as TwoSum.
__device__ __forceinline__ df df_from_u32(uint32_t v) {
    return df_fast_two_sum(__uint2float_rz(v & 0xFFFFFF00u), __uint2float_rz(v & 0xFFu));
}

__device__ __forceinline__ df df_from_i32(int32_t v) {
    const int32_t high = static_cast<int32_t>(static_cast<uint32_t>(v) & 0xFFFFFF00u);
    return df_fast_two_sum(__int2float_rz(high), __uint2float_rz(static_cast<uint32_t>(v) & 0xFFu));
}

// FP32 -> FP64 by bit manipulation on the integer pipe (exact for normal numbers; zero and
// FP32 subnormals, below 2^-126, become a signed zero).  Keeps conversions off B300's narrow
// FP64 pipe: a stored value costs one DADD instead of two conversions and a DADD.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t sign = b & 0x80000000u;
    uint32_t hi = (((b & 0x7FFFFFFFu) >> 3) + 0x38000000u) | sign;  // exponent rebias 127 -> 1023
    uint32_t lo = b << 29;
    if ((b & 0x7F800000u) == 0u) {
        hi = sign;
        lo = 0u;
    }
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

// The same rebias without the zero / subnormal case: exact for normal numbers; a zero or an
// FP32 subnormal maps to a value of magnitude in [2^-127, 2^-126) with its sign.
//
// The high word sign | (e + 896) << 20 | m >> 3 from an arithmetic shift: xs = b >> 3 (signed)
// copies the sign into bits 31..28, so xs & 0x90000000 is 0x90000000 times the sign, and
// xs + (xs & 0x90000000) + 0x38000000 = ((b & 0x7FFFFFFF) >> 3) + 0x38000000 + sign (mod 2^32):
// a shift, a logic operation and a three-input addition (checked against the masked form for
// all 2^32 bit patterns).
__device__ __forceinline__ double f32_to_f64_bits_fast(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t xs = static_cast<uint32_t>(static_cast<int32_t>(b) >> 3);
    const uint32_t hi = xs + (xs & 0x90000000u) + 0x38000000u;
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(b << 29));
}

// Nearest double to hi + lo for the stored kinematics, to within 2^-125 absolute: parts below
// 2^-126 in magnitude (zero, FP32 subnormals) are not special-cased, so an exact double-float
// zero is stored as 0 or +-2^-126.  Momenta and energies of a decay above threshold are never
// below that scale (they carry a ~2^-46 relative error at the event scale), and the check
// would cost three integer instructions per stored value.
__device__ __forceinline__ double df_to_double(df x) {
    return __dadd_rn(f32_to_f64_bits_fast(x.hi), f32_to_f64_bits_fast(x.lo));
}

// Nearest double to hi + lo with zeros exact (for values whose zero has a meaning).
__device__ __forceinline__ double df_to_double_exact(df x) {
    return __dadd_rn(f32_to_f64_bits(x.hi), f32_to_f64_bits(x.lo));
}

// x * 2^k for an exact power of two (both parts scale exactly).
__device__ __forceinline__ df df_scale(df x, float pow2) { return df{__fmul_rn(x.hi, pow2), __fmul_rn(x.lo, pow2)}; }

// (x + 1/2) 2^-31 for a 32-bit unsigned x (= 1 + cos(theta) when x is a cos(theta) draw):
// x + 1/2 = (x & ~0xFF) + ((x & 0xFF) + 1/2), both parts exact in FP32 (the first 0 or >= 256,
// the second in (0, 256): FastTwoSum is exact), then an exact scale.
__device__ __forceinline__ df df_half_odd_raw(uint32_t x) {  // x + 1/2, unscaled
    const float a = __uint2float_rz(x & 0xFFFFFF00u);
    const float b = __fadd_rn(__uint2float_rz(x & 0xFFu), 0.5f);
    return df_fast_two_sum(a, b);
}

__device__ __forceinline__ df df_half_odd_u32(uint32_t x) {
    return df_scale(df_half_odd_raw(x), 4.656612873077392578125e-10f);
}

// x - 2^31 + 1/2 for a 32-bit unsigned x, exact (cos(theta) 2^31 of a cos(theta) draw x)
__device__ __forceinline__ df df_half_odd_centered_raw(uint32_t x) {
    const int32_t c = static_cast<int32_t>(x ^ 0x80000000u);
    const float a = __int2float_rz(static_cast<int32_t>(static_cast<uint32_t>(c) & 0xFFFFFF00u));
    const float b = __fadd_rn(__uint2float_rz(x & 0xFFu), 0.5f);
    return df_fast_two_sum(a, b);
}

// (x - 2^31 + 1/2) 2^-31 for a 32-bit unsigned x (= cos(theta) = 2u - 1 exactly)
__device__ __forceinline__ df df_half_odd_centered(uint32_t x) {
    return df_scale(df_half_odd_centered_raw(x), 4.656612873077392578125e-10f);
}

// An FP64 value as a double-float pair by integer operations (an FP64-to-FP32 conversion would
// run on the narrow FP64 pipe): hi = x truncated to 24 significant bits, lo = the remaining 29
// bits of the significand converted to FP32 (rounded to 24 bits) and scaled by an exact power
// of two, so |x - (hi + lo)| < 2^-47 |x|, with 0 <= |lo| < ulp(hi), for 2^-74 <= |x| < 2^128.
// Below 2^-74 the low part is dropped (absolute error under 2^-98) and below 2^-126 the value
// is a signed zero: far under any kinematic scale of these events.
__device__ __forceinline__ df df_from_double(double x) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const uint32_t bh = static_cast<uint32_t>(b >> 32);
    const uint32_t sign = bh & 0x80000000u;
    const int ef = static_cast<int>((bh >> 20) & 0x7FFu) - 896;  // FP32 biased exponent of hi
    if (ef <= 0) return df{__uint_as_float(sign), 0.0f};
    const float hi = __uint_as_float(sign | (static_cast<uint32_t>(ef) << 23) |
                                     (static_cast<uint32_t>(b >> 29) & 0x7FFFFFu));
    const int el = ef - 52;                                       // FP32 biased exponent of 2^(e - 52)
    const float mag = el > 0 ? __fmul_rn(__uint2float_rn(static_cast<uint32_t>(b) & 0x1FFFFFFFu),
                                         __uint_as_float(static_cast<uint32_t>(el) << 23))
                             : 0.0f;
    return df{hi, sign ? -mag : mag};
}

// x + f for an FP32 f with |f| <= |x.hi|, left unnormalised (df_add_small without its final
// FastTwoSum), for a result that only feeds products.
__device__ __forceinline__ df df_add_small_lazy(df x, float f) {
    const float s = __fadd_rn(x.hi, f);
    return df{s, __fadd_rn(__fsub_rn(f, __fsub_rn(s, x.hi)), x.lo)};
}

// x + f for an FP32 f with |f| <= |x.hi| (a correction term): FastTwoSum and renormalise.
__device__ __forceinline__ df df_add_small(df x, float f) {
    const float s = __fadd_rn(x.hi, f);
    const float e = __fadd_rn(__fsub_rn(f, __fsub_rn(s, x.hi)), x.lo);
    return df_fast_two_sum(s, e);
}

// v 2^-64 as a double-float: the top 48 significant bits of v (the rest truncated, relative
// error < 2^-47), hi built from the bits directly; 0 for v = 0.
__device__ __forceinline__ df df_frac_u64(uint64_t v) {
    if (v == 0) return df{0.0f, 0.0f};
    const int lz = __clzll(static_cast<long long>(v));
    const uint64_t m = v << lz;                                            // bit 63 set
    const uint32_t t1 = static_cast<uint32_t>(m >> 40);                    // bits 63..40
    const uint32_t t2 = static_cast<uint32_t>(m >> 16) & 0xFFFFFFu;        // bits 39..16
    const float hi = __int_as_float(((126 - lz) << 23) | static_cast<int>(t1 & 0x7FFFFFu));  // t1 2^(-24-lz)
    const float lo = __fmul_rn(__uint2float_rz(t2), __int_as_float((79 - lz) << 23));         // t2 2^(-48-lz)
    return df_fast_two_sum(hi, lo);
}

// x + f for any FP32 f (TwoSum, then the low parts).
__device__ __forceinline__ df df_add_f(df x, float f) {
    const df s = df_two_sum(x.hi, f);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

// ------------------------------------------------------------------------------------
// Weight product prod_k p_k without the FP64 pipe: a double-float mantissa times 2^e.  Each
// factor is scaled by an exact power of two into [1, 2) (its exponent read from the bits of
// its high part) before the double-float product, so the mantissa stays below 2^(n-1) and the
// range is the integer exponent's; one conversion to double at the end.
// ------------------------------------------------------------------------------------
struct DfWeight {
    df m;
    int e;
};

__device__ __forceinline__ DfWeight df_weight_one() { return DfWeight{df{1.0f, 0.0f}, 0}; }

__device__ __forceinline__ DfWeight df_weight_mul(DfWeight w, df p) {
    // p >= 0; 0 and FP32 subnormals read as exponent -127 (a zero stays zero, a subnormal is
    // scaled into the normal range).  With b the biased exponent field of p.hi, the scale
    // 2^(127 - b) has the field 254 - b: one subtraction from the masked bits.
    const uint32_t field = __float_as_uint(p.hi) & 0x7F800000u;
    const float s = __uint_as_float(0x7F000000u - field);  // 2^-ep, ep = b - 127
    // the running product is renormalised after each factor: carried unnormalised, its low part
    // grows factor by factor and the product's dropped lo x lo term with it (worst weight error
    // over a 3.6e6-event survey 6.1e-13 unnormalised, 2.7e-13 renormalised)
    const df m = w.m * df{__fmul_rn(p.hi, s), __fmul_rn(p.lo, s)};
    return DfWeight{df_fast_two_sum(m.hi, m.lo), w.e + static_cast<int>(field >> 23) - 127};
}

// w as the nearest double, times an FP64 factor c.  The power 2^e is applied to the bits of
// the product's exponent when the result stays a normal double (two FP64 instructions in all);
// otherwise by two FP64 multiplications with normal powers of two, so that a result below the
// double range rounds to a subnormal or zero as a plain product would.  A zero factor (a tie
// in the mass draws) gives exactly 0.
__device__ __forceinline__ double df_weight_final(DfWeight w, double c) {
    const double v = df_to_double_exact(w.m) * c;
    const long long bits = __double_as_longlong(v);
    const int ev = static_cast<int>((bits >> 52) & 0x7FF);  // biased exponent of v
    if (ev != 0 && ev + w.e > 0 && ev + w.e < 0x7FF)          // v normal and v 2^e normal
        return __longlong_as_double(bits + (static_cast<long long>(w.e) << 52));
    if (ev == 0 && v == 0.0) return v;
    const int e1 = w.e < -1022 ? -1022 : (w.e > 1023 ? 1023 : w.e);
    int e2 = w.e - e1;
    e2 = e2 < -1022 ? -1022 : (e2 > 1023 ? 1023 : e2);
    const double p1 = __longlong_as_double(static_cast<long long>(e1 + 1023) << 52);
    const double p2 = __longlong_as_double(static_cast<long long>(e2 + 1023) << 52);
    return (v * p1) * p2;
}

// ------------------------------------------------------------------------------------
// sin and cos of phi = 2 pi u, u = (x + 1/2) 2^-32 for a 32-bit x, in df.
//
// They multiply momenta bounded by the event scale, so the target is an absolute error of
// ~1e-15.  Reduction is exact integer arithmetic: phi = theta_k + delta with theta_k = k pi/1024,
// k = the top 11 bits of x (a 2048-entry table of sin/cos(theta_k) in df over the whole
// circle), and delta = pi (2r + 1) 2^-32 in (0, pi/1024), r = the low 21 bits:
//   sin(delta) = delta - delta^3/6 (1 - delta^2/20)      (the correction, <= 4.9e-9, in FP32:
//                                                          absolute error < 1e-15)
//   cos(delta) = 1 - delta^2/2 + delta^4/24             (delta^2 from an exact product)
// then the angle-sum identities.
// ------------------------------------------------------------------------------------
struct SinCosTable {
    float4 e[2048];  // (sin hi, sin lo, cos hi, cos lo) of k pi/1024: one 16-byte load
};

// The table lives in shared memory (32 KB) of the kernels that compute in df.  Each block
// fills it before its first event: entries 0..256 (angles 0..pi/4) from FP64 sincospi, the
// rest from those by the exact symmetries sin(pi/2 - b) = cos b and quarter-turn rotations.
// Every thread of the block must call it (it synchronises the block).
static __shared__ SinCosTable s_sincos_table;

__device__ __forceinline__ void df_sincos_table_init() {
    for (int k = threadIdx.x; k <= 256; k += blockDim.x) {
        double sv, cv;
        sincospi(static_cast<double>(k) / 1024.0, &sv, &cv);
        const float sh = __double2float_rn(sv), ch = __double2float_rn(cv);
        s_sincos_table.e[k] = make_float4(sh, __double2float_rn(sv - static_cast<double>(sh)), ch,
                                          __double2float_rn(cv - static_cast<double>(ch)));
    }
    __syncthreads();
    for (int k = 257 + threadIdx.x; k < 2048; k += blockDim.x) {
        const int j = k >> 9, m = k & 511;  // k pi/1024 = j pi/2 + m pi/1024
        float4 b = s_sincos_table.e[m <= 256 ? m : 512 - m];
        if (m > 256) b = make_float4(b.z, b.w, b.x, b.y);  // sin(pi/2 - a) = cos a, cos(pi/2 - a) = sin a
        float4 r;
        if (j == 0) r = b;
        else if (j == 1) r = make_float4(b.z, b.w, -b.x, -b.y);   // (cos, -sin)
        else if (j == 2) r = make_float4(-b.x, -b.y, -b.z, -b.w); // (-sin, -cos)
        else r = make_float4(-b.z, -b.w, b.x, b.y);               // (-cos, sin)
        s_sincos_table.e[k] = r;
    }
}

// sin and cos of theta_k + delta with delta = pi rem2 2^-32 (rem2 < 2^22) and k < 2048.
__device__ __forceinline__ void df_sincos_table_step(uint32_t k, uint32_t rem2, const SinCosTable& T, df* s,
                                                     df* c) {
    const df pi_scaled{7.31459059988282e-10f, -2.035470133961082e-17f};  // pi 2^-32 (hi + lo)
    const df d = pi_scaled * __uint2float_rn(rem2);                       // delta
    const float d2f = __fmul_rn(d.hi, d.hi);
    // sin(delta)
    const float corr = __fmul_rn(__fmul_rn(d.hi, __fmul_rn(d2f, 0.16666667163372039795f)),
                                 __fmaf_rn(d2f, -0.05f, 1.0f));
    const df sd = df_add_small_lazy(d, -corr);
    // cos(delta): delta^2 = p + e exactly (TwoProd) plus 2 hi lo
    const float p2 = d2f;
    const float e2 = __fmaf_rn(2.0f * d.hi, d.lo, __fmaf_rn(d.hi, d.hi, -p2));
    const df one_minus = df_fast_two_sum(1.0f, -0.5f * p2);
    const float tail = __fmaf_rn(__fmul_rn(p2, p2), 1.0f / 24.0f, -0.5f * e2);
    const df cd{one_minus.hi, __fadd_rn(one_minus.lo, tail)};  // feeds products: unnormalised
    const float4 t = T.e[k];
    const df sk{t.x, t.y}, ck{t.z, t.w};
    // sin(theta_k + delta), cos(theta_k + delta); near a zero of either the two products
    // cancel and the pair is left unnormalised: its absolute error (what a direction
    // component needs) stays at ~2^-48
    *s = df_add_lazy(sk * cd, ck * sd);
    *c = df_add_lazy(ck * cd, -(sk * sd));
}

__device__ __forceinline__ void df_sincos_2pi_u(uint32_t x, const SinCosTable& T, df* s, df* c) {
    // k = top 11 bits; delta = pi (2r + 1) 2^-32 with r the low 21 bits (2r + 1 < 2^22, exact in FP32)
    df_sincos_table_step(x >> 21, ((x & 0x1FFFFFu) << 1) | 1u, T, s, c);
}

// sin and cos of 2 pi d 2^-32 for a 32-bit integer d (no half-step offset: the difference of
// two phi draws, whose offsets cancel).
__device__ __forceinline__ void df_sincos_2pi_int(uint32_t d, const SinCosTable& T, df* s, df* c) {
    df_sincos_table_step(d >> 21, (d & 0x1FFFFFu) << 1, T, s, c);
}

}  // namespace hydra
