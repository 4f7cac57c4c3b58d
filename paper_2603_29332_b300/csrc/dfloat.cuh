// dfloat.cuh -- float-float ("double-word") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers (~44 significant bits).  Built
// from the classical error-free transformations: TwoSum (Knuth, TAOCP vol. 2), FastTwoSum
// (Dekker 1971), TwoProd via a fused multiply-add, and the double-word add / multiply / divide /
// square-root algorithms analysed by Joldes, Muller and Popescu (ACM TOMS 2017) and Karp and
// Markstein (1997).  Used where FP32 alone is too short: the mass matrix of a 90-DoF skeleton
// has a componentwise condition number ~1e5, so its entries and its factorisation need more
// than 24 bits, while FP64 on this part runs at a small fraction of the FP32 rate.
#pragma once
#include <cuda_runtime.h>

namespace msim {

// 8-byte aligned, so that a pair in shared memory moves as one 8-byte access (a half-warp per
// wavefront) rather than as two 4-byte accesses at an 8-byte stride (two-way bank conflicts)
struct __align__(8) df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float x) { return {x, 0.f}; }

// exact: a + b = s + e
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
// exact when |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = a + b;
    const float e = b - (s - a);
    return {s, e};
}
// exact: a * b = p + e
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}
// x + y; absolute error ~ 2^-44 (|x| + |y|)
__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    s.lo += x.lo + y.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_add_f(df x, float y) {
    df s = two_sum(x.hi, y);
    s.lo += x.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df df_mul(df x, df y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df x, float y) {
    const float p = x.hi * y;
    float e = fmaf(x.hi, y, -p);
    e = fmaf(x.lo, y, e);
    return fast_two_sum(p, e);
}
// acc + x * y (x float-float, y float)
__device__ __forceinline__ df df_fma_f(df acc, df x, float y) { return df_add(acc, df_mul_f(x, y)); }
// acc - x * y, all float-float; the product is kept unnormalised before the subtraction
__device__ __forceinline__ df df_fms(df acc, df x, df y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    df s = two_sum(acc.hi, -p);
    s.lo += acc.lo - e;
    return fast_two_sum(s.hi, s.lo);
}
// 1 / y: one Newton correction of the FP32 quotient
__device__ __forceinline__ df df_recip(df y) {
    const float q1 = 1.f / y.hi;
    const df p = df_mul_f(y, q1);          // ~1
    const df r = df_add_f(df_neg(p), 1.f);  // 1 - y q1
    const float q2 = r.hi / y.hi;
    return fast_two_sum(q1, q2);
}
// sqrt(x), x > 0 (Karp-Markstein: y + (x - y^2) / (2 y))
__device__ __forceinline__ df df_sqrt(df x) {
    const float y = sqrtf(x.hi);
    const df yy = two_prod(y, y);
    const float r = ((x.hi - yy.hi) - yy.lo + x.lo) * (0.5f / y);
    return fast_two_sum(y, r);
}
// 1 / sqrt(x), x > 0: FP32 reciprocal square root plus one Newton step y (1 + (1 - x y^2) / 2)
__device__ __forceinline__ df df_rsqrt(df x) {
    const float y = rsqrtf(x.hi);
    const df yy = two_prod(y, y);
    const df e = df_add_f(df_neg(df_mul(x, yy)), 1.f);   // 1 - x y^2, small
    return fast_two_sum(y, y * e.hi * 0.5f);
}
// renormalise an arbitrary pair (|lo| may exceed |hi|)
__device__ __forceinline__ df df_norm(float hi, float lo) { return two_sum(hi, lo); }

}  // namespace msim
