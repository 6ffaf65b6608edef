// lbmhd_ff.cuh -- double-word ("float-float") arithmetic on the FP32 units.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2: 48 significand bits, unit roundoff u^2 = 2^-48, at
// FP32 issue rates.  On GB300 the FP64 pipe is a small fraction of the FP32
// one, so the double-word collision runs several times faster than the FP64
// collision, at 2^5 times its rounding error.
//
// Building blocks (all error-free transformations of IEEE binary32):
//   TwoSum      (Knuth, TAOCP vol. 2, Sec. 4.2.2): s + e = a + b exactly;
//   FastTwoSum  (Dekker 1971): the same in 3 operations when |a| >= |b|;
//   TwoProd     with a fused multiply-add: p + e = a b exactly.
// Sum and product are the "sloppy" double-word sum and the FMA double-word
// product analysed by Joldes, Muller and Popescu (ACM TOMS 44(2), 2017):
// the sum's error is bounded relative to |x| + |y| (not |x + y|), which is
// the bound the rounded FP64 arithmetic of a stencil update effectively has
// as well, at 11 operations instead of 20 for the accurate variant.
// Reciprocal: one Newton-Raphson step from the correctly rounded FP32
// reciprocal, whose residual 1 - b y is exact with an FMA (Markstein), plus
// the quadratic term of the series.  Square root: Dekker's sqrt2 -- the
// correctly rounded FP32 root s corrected by (x - s^2) / (2 s), with x - s^2
// formed exactly by TwoProd.
//
// Every operation uses the explicitly rounded intrinsics (__fadd_rn,
// __fmul_rn, __fmaf_rn), which the compiler never contracts or reorders, so
// the error-free transformations stay exact.
#pragma once

#include <cuda_runtime.h>

namespace lbmhd {

struct ff {
    float hi, lo;
    ff() = default;
    __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr ff(int v) : hi((float)v), lo(0.0f) {}
    // Nearest double-word to a double (exact to 2^-48 relative); used for
    // constants and host-side parameters.
    __host__ __device__ constexpr ff(double v)
        : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ constexpr double to_double() const { return (double)hi + (double)lo; }
    // A hidden friend, found by argument-dependent lookup only, so that it
    // does not hide the float and double fabs inside this namespace.
    friend __device__ __forceinline__ ff fabs(ff x) {
        return x.hi < 0.0f ? ff(-x.hi, -x.lo) : x;
    }
};

// Division of constants only (folded at compile time in constexpr context);
// a runtime quotient goes through rcp(ff).
__host__ __device__ constexpr ff operator/(ff a, ff b) { return ff(a.to_double() / b.to_double()); }

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff(s, e);
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ ff operator-(ff x) { return ff(-x.hi, -x.lo); }

__device__ __forceinline__ ff operator+(ff x, ff y) {
    const ff s = two_sum(x.hi, y.hi);
    const float v = __fadd_rn(x.lo, y.lo);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, v));
}
__device__ __forceinline__ ff operator-(ff x, ff y) { return x + (-y); }

__device__ __forceinline__ ff operator*(ff x, ff y) {
    const float ch = __fmul_rn(x.hi, y.hi);
    const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);  // TwoProd: ch + cl1 = x.hi y.hi
    const float tl = __fmul_rn(x.hi, y.lo);
    const float cl2 = __fmaf_rn(x.lo, y.hi, tl);
    return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}

// x times an FP32 constant k: exact scaling when k is a power of two (the
// test folds at compile time for a literal k), else the FMA double-word by
// FP32 product of Joldes, Muller and Popescu (5 operations).
__device__ __forceinline__ ff kmul(float k, ff x) {
    if ((__float_as_uint(k) & 0x7fffffu) == 0u) return ff(__fmul_rn(x.hi, k), __fmul_rn(x.lo, k));
    const float ch = __fmul_rn(x.hi, k);
    const float cl = __fmaf_rn(x.lo, k, __fmaf_rn(x.hi, k, -ch));
    return fast_two_sum(ch, cl);
}

__device__ __forceinline__ ff& operator+=(ff& x, ff y) { return x = x + y; }
__device__ __forceinline__ ff& operator-=(ff& x, ff y) { return x = x - y; }
__device__ __forceinline__ ff& operator*=(ff& x, ff y) { return x = x * y; }

__device__ __forceinline__ bool operator>(ff a, ff b) {
    return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}
__device__ __forceinline__ bool operator<(ff a, ff b) { return b > a; }

// Sums of many FP32 terms without FP64 instructions: a += t in double-word
// (TwoSum of the high parts, the low parts added, FastTwoSum), 9 operations.
__device__ __forceinline__ void dw_accumulate(ff& a, float t) {
    const ff s = two_sum(a.hi, t);
    a = fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ ff rcp(ff x) {
    const float y = __frcp_rn(x.hi);
    float e = __fmaf_rn(-x.hi, y, 1.0f);  // exact residual of the rounded reciprocal
    e = __fmaf_rn(-x.lo, y, e);           // 1 - x y to double-word accuracy
    const float c = __fmul_rn(y, e);
    return fast_two_sum(y, __fmaf_rn(c, e, c));  // y (1 + e + e^2)
}

__device__ __forceinline__ ff sqrt_(ff x) {
    const float s = __fsqrt_rn(x.hi);
    const float p = __fmul_rn(s, s);
    const float pe = __fmaf_rn(s, s, -p);  // TwoProd: p + pe = s^2
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), pe), x.lo);
    const float h = s > 0.0f ? __fmul_rn(0.5f, __frcp_rn(s)) : 0.0f;
    return fast_two_sum(s, __fmul_rn(r, h));
}

}  // namespace lbmhd
