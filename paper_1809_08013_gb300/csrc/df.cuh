// df.cuh -- double-float arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats (about 48 significant
// bits). The building blocks are the classical error-free transformations:
// Knuth's TwoSum, Dekker's Fast2Sum (|a| >= |b|) and the FMA-based TwoProd
// (a b = p + e exactly). Every operation uses the explicitly rounded
// intrinsics so the compiler cannot contract or reassociate them.
//
// Error model used by the pair kernels: add and mul return a result within
// about 2^-47 (|x| + |y|) and 2^-47 |x y| of the exact one, so a chain of a few
// tens of operations stays near 1e-14 relative to the magnitudes involved.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sph {
namespace dfl {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ df neg(df x) { return {-x.hi, -x.lo}; }

// x + y with the low parts folded in once (error ~2^-47 (|x| + |y|)).
__device__ __forceinline__ df add(df x, df y) {
    const df s = two_sum(x.hi, y.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df sub(df x, df y) { return add(x, neg(y)); }

// x + y for operands of the same sign (no cancellation), left unnormalised:
// the low part may reach ~1.5 ulp of the high one. Only for a sum whose
// consumer is a normalising add: a product of an unnormalised value rounds
// its larger low part in FP32 (measured: up to 5x the error of the force
// sums), and a running sum's low part would keep growing.
__device__ __forceinline__ df add_same(df x, df y) {
    const df s = two_sum(x.hi, y.hi);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}

__device__ __forceinline__ df addf(df x, float b) {
    const df s = two_sum(x.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

// Products return (p, e) without the final Fast2Sum: that step is exact (it
// does not change hi + lo), and every consumer here -- another product, a
// sum, a sign or range test of hi, the conversion to double -- accepts a low
// part of a few ulps of hi at ~2^-46 relative error.
__device__ __forceinline__ df mul(df x, df y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return {p, e};
}

__device__ __forceinline__ df mulf(df x, float b) {
    const float p = __fmul_rn(x.hi, b);
    float e = __fmaf_rn(x.hi, b, -p);
    e = __fmaf_rn(x.lo, b, e);
    return {p, e};
}

__device__ __forceinline__ df sqr(df x) {
    const float p = __fmul_rn(x.hi, x.hi);
    float e = __fmaf_rn(x.hi, x.hi, -p);
    e = __fmaf_rn(__fadd_rn(x.hi, x.hi), x.lo, e);
    return {p, e};
}

// exact scaling by a power of two (no overflow/underflow in use)
__device__ __forceinline__ df scale2(df x, float p2) { return {__fmul_rn(x.hi, p2), __fmul_rn(x.lo, p2)}; }

// 1/sqrt(x), x > 0: FP32 approximation y0, then one Newton step
// y1 = y0 + y0 e / 2 with e = 1 - x y0^2 (error ~2^-46 from the ~2^-23 seed).
// e is small (~2^-22), so the FMAs below give it to a few units of 2^-46
// absolutely: y0^2 = p + pe exactly, then 1 - x_hi p, - x_hi pe, - x_lo p.
// The correction y0 e / 2 is below 2^-22 y0 and joins y0 by Fast2Sum.
__device__ __forceinline__ df rsqrt(df x) {
    float y0;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(x.hi));
    const float p = __fmul_rn(y0, y0);
    const float pe = __fmaf_rn(y0, y0, -p);
    float e = __fmaf_rn(-x.hi, p, 1.0f);
    e = __fmaf_rn(-x.hi, pe, e);
    e = __fmaf_rn(-x.lo, p, e);
    const float hy = __fmul_rn(0.5f, y0);
    const float c = __fmul_rn(hy, e);
    const float cl = __fmaf_rn(hy, e, -c);
    const df r = fast_two_sum(y0, c);
    return {r.hi, __fadd_rn(r.lo, cl)};
}

// 1/x, x > 0: FP32 approximation y0, one Newton step y1 = y0 + y0 e with
// e = 1 - x y0 (~2^-22), formed by FMAs as in rsqrt.
__device__ __forceinline__ df rcp(df x) {
    float y0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(x.hi));
    float e = __fmaf_rn(-x.hi, y0, 1.0f);
    e = __fmaf_rn(-x.lo, y0, e);
    const float c = __fmul_rn(y0, e);
    const float cl = __fmaf_rn(y0, e, -c);
    const df r = fast_two_sum(y0, c);
    return {r.hi, __fadd_rn(r.lo, cl)};
}

// Per-particle conversion to double-float with the FP64 pipe (exact to 2^-48).
__device__ __forceinline__ df from_double_fp64(double d) {
    const float hi = __double2float_rn(d);
    const float lo = __double2float_rn(d - (double)hi);
    return {hi, lo};
}

// Split of a double into hi + lo (error <= 2^-47 |d|) using integer and FP32
// operations only: on GB300 FP64 arithmetic, int/float conversions and the
// leading-zero count all issue on the narrow FP64 pipe, so none is used.
// hi takes the top 24 significand bits. The remaining 29 bits R = Rh 2^23 + Rl
// become floats exactly by the 2^23 trick (the bits of an integer m < 2^23
// ORed into 2^23's mantissa give 2^23 + m; subtracting 2^23 is exact), then
// lo = (Rh 2^23 + Rl) 2^(e-1075) rounded once. lo may exceed half an ulp of
// hi, which the double-float operations accept. Meant for pair differences:
// |d| < 2^-60 maps to 0 (an absolute error far below any use here) and |d|
// is assumed below 2^60 (larger magnitudes saturate).
// With sh, the result is d 2^sh (sh moves the exponent; the thresholds then
// apply to d 2^sh): how a difference in the caller's units enters the pair
// kernels' units.
__device__ __forceinline__ df from_double(double d, int sh = 0) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return {0.0f, 0.0f};  // zero (and subnormal differences: below any use)
    e += sh;
    if (e < 1023 - 60) return {0.0f, 0.0f};
    e = e > 1023 + 60 ? 1023 + 60 : e;
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) |
                                     (unsigned)((b >> 29) & 0x7fffffu));
    const unsigned R = (unsigned)(b & 0x1fffffffull);
    const float fl = __fsub_rn(__uint_as_float(0x4b000000u | (R & 0x7fffffu)), 8388608.0f);
    const float fh = __fsub_rn(__uint_as_float(0x4b000000u | (R >> 23)), 8388608.0f);
    const float r = __fmaf_rn(fh, 8388608.0f, fl);                     // R rounded to float
    const float lo = __fmul_rn(r, __uint_as_float((unsigned)(e - 948) << 23));  // R 2^(e-1075)
    return {hi, __uint_as_float(__float_as_uint(lo) | sign)};
}

// ---- Exact coordinate differences without the FP64 pipe.
// Once per step each coordinate becomes a 64-bit fixed-point number
// X = rint(x 2^k), with k per instance such that |X| < 2^61 (x is exact in it
// wherever ulp(x) >= 2^-k; elsewhere rounded by at most 2^-(k+1), a
// negligible absolute error), split as X = c2 2^42 + c1 2^21 + c0 with c2
// signed and c1, c0 in [0, 2^21). The chunks are stored pre-scaled as floats
// c2 2^(42-f), c1 2^(21-f), c0 2^-f with f = k + uL (the coordinate in the
// length unit 2^uL of the pair kernels), each exact. For two particles the
// three chunkwise differences are exact floats too (at most 21 significant
// bits), and their double-float sum is (x_i - x_j) 2^-uL to within ~2^-48 of
// its size: the only rounding of the whole difference.
struct fx3 {
    float c2, c1, c0;
};

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// k in [-1000, 1000], f in [-60, 100] (so every scaled chunk is a normal float)
__device__ __forceinline__ fx3 to_fx(double x, int k, int f) {
    const double sc = __longlong_as_double((long long)(1023 + k) << 52);  // 2^k
    const long long X = __double2ll_rn(x * sc);
    return {(float)(X >> 42) * pow2f(42 - f), (float)((X >> 21) & 0x1fffffLL) * pow2f(21 - f),
            (float)(X & 0x1fffffLL) * pow2f(-f)};
}

// The double-float value of the exact chunk differences a2 + a1 + a0
// (a2, a1, a0 multiples of 2^(42-k), 2^(21-k), 2^-k; |a1| < 2^(43-k),
// |a0| < 2^(22-k)). Fast2Sum is exact for (a2, a1): either |a2| >= |a1| in
// exponent, or a2 = 0, or 2^(42-k) <= |a2| < |a1| and a2 + a1 is a multiple
// of 2^(21-k) below 2^(44-k), i.e. representable, in which case Fast2Sum
// returns it with a zero error term. Then t = lo + a0 is rounded once (|t| <
// ulp(hi)/2 + 2^(22-k) <= |hi| unless hi = 0) and folded in by Fast2Sum:
// the result is within ~2^-48 of the exact difference.
__device__ __forceinline__ df fx_sum(float a2, float a1, float a0) {
    const df s = fast_two_sum(a2, a1);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a0));
}

// Per-particle conversion back to FP64 (two conversions and one FP64 add).
__device__ __forceinline__ double to_double(df x) { return (double)x.hi + (double)x.lo; }

// Sum over groups of T consecutive lanes (T a power of two <= 32), returned to
// every lane of the group: a fixed butterfly, independent of timing.
template <int T>
__device__ __forceinline__ df lane_sum(df v) {
#pragma unroll
    for (int o = 1; o < T; o <<= 1) {
        const df w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = add(v, w);
    }
    return v;
}

// The pair kernels' units (length 2^uL, mass 2^uM, velocity 2^uV) of one
// instance, as the exact power-of-two factors that take each packed quantity
// from the caller's units into them (a quantity of dimension L^a M^b V^c is
// multiplied by 2^-(a uL + b uM + c uV)).
struct PairUnits {
    double L;     // lengths (h):              2^-uL
    double iL;    // inverse lengths (1/h):    2^uL
    double M;     // masses:                   2^-uM
    double V;     // velocities (c, v):        2^-uV
    double rho;   // densities, M L^-3:        2^(3 uL - uM)
    double A;     // p / rho^2, L^3 V^2 M^-1:  2^(uM - 3 uL - 2 uV)
};

__host__ __device__ __forceinline__ double pow2(int e) {
    union { long long i; double d; } u;
    u.i = (long long)(1023 + e) << 52;
    return u.d;
}

__host__ __device__ __forceinline__ PairUnits pair_units(int uL, int uM, int uV) {
    return {pow2(-uL), pow2(uL), pow2(-uM), pow2(-uV), pow2(3 * uL - uM), pow2(uM - 3 * uL - 2 * uV)};
}

// The range every float-pair quantity of a pack must lie in, in the pair
// kernels' units, for the kernel arithmetic to stay within the normal float
// range with ample room (no product of pair terms overflows, and the low
// parts of the terms that carry the sums stay normal): h within 2^15 of the
// instance's mean h (so 1/h^4 stays within 2^+-60); rho in [2^-60, 2^60];
// alpha c below 2^60; |p/rho^2| below 2^64 (a stiff equation of state far
// from rho0 makes it the quantity with the widest range).
__device__ __forceinline__ bool pack_in_range(double hinv_u, double rho_u, double A_u, double ac_u) {
    return hinv_u >= 0x1p-15 && hinv_u <= 0x1p15 && rho_u >= 0x1p-60 && rho_u <= 0x1p60 &&
           fabs(A_u) <= 0x1p64 && ac_u <= 0x1p60;
}

// Per-particle pack of the double-float force kernel (48 B per particle), in
// the pair kernels' units:
//   dpk[3k] = (1/h, 1/h^4), dpk[3k+1] = (p/rho^2, h/2), dpk[3k+2] = (rho/2, alpha c/2).
// A particle outside pack_in_range sets `range_bit` in *status. The float
// pairs are split with integer operations (from_double: within 2^-47 of each
// value, no FP64 pipe), which in range hold every value but p/rho^2; that one
// is split on the FP64 pipe (from_double_fp64), which holds any float.
__device__ __forceinline__ void write_pack(float4* __restrict__ dpk, int64_t k, double hinv,
                                           double A, double h, double rho, double alpha, double c,
                                           const PairUnits& U, unsigned* status,
                                           unsigned range_bit) {
    const double hu = hinv * U.iL;
    const double h2 = hu * hu;
    const double Au = A * U.A;
    const double ru = rho * (0.5 * U.rho);
    const double cu = (alpha * c) * (0.5 * U.V);
    if (!pack_in_range(hu, 2.0 * ru, Au, 2.0 * cu)) atomicOr(status, range_bit);
    const df a = from_double(hu), b = from_double(h2 * h2);
    const df cA = from_double_fp64(Au), d = from_double(h * (0.5 * U.L));
    const df e = from_double(ru), f = from_double(cu);
    dpk[3 * k + 0] = make_float4(a.hi, a.lo, b.hi, b.lo);
    dpk[3 * k + 1] = make_float4(cA.hi, cA.lo, d.hi, d.lo);
    dpk[3 * k + 2] = make_float4(e.hi, e.lo, f.hi, f.lo);
}

}  // namespace dfl
}  // namespace sph
