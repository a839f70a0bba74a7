// Double-float ("double-word") arithmetic on the float32 pipes.
//
// A value is hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits.  The
// building blocks are the classical error-free transforms: TwoSum (Knuth,
// TAOCP vol. 2, 4.2.2), FastTwoSum (Dekker 1971) and TwoProd through a fused
// multiply-add; the double-word add, multiply, divide and square root follow
// the algorithms analysed by Joldes, Muller and Popescu, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic", ACM TOMS
// 44(2), 2017 (relative errors of a few 2^-48).  Every float32 operation is
// written with a round-to-nearest intrinsic so the compiler cannot contract
// or reorder it.  Division and square root take their leading term from the
// hardware's approximate reciprocal and reciprocal square root (a few ulps);
// the correction computed from the exact remainder then gives about 2^-44
// relative, and every operation stays an odd function of its inputs.
#pragma once

#include <cuda_runtime.h>

namespace pc {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float h, float l) {
    df r;
    r.hi = h;
    r.lo = l;
    return r;
}

// s + e == a + b exactly
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df_make(s, e);
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return df_make(s, e);
}

__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    return df_make(p, e);
}

// accurate double-word + double-word
__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    const df t = two_sum(x.lo, y.lo);
    float c = __fadd_rn(s.lo, t.hi);
    df v = fast_two_sum(s.hi, c);
    c = __fadd_rn(t.lo, v.lo);
    return fast_two_sum(v.hi, c);
}

__device__ __forceinline__ df df_neg(df x) { return df_make(-x.hi, -x.lo); }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// double-word + float
__device__ __forceinline__ df df_add_f(df x, float y) {
    const df s = two_sum(x.hi, y);
    const float v = __fadd_rn(x.lo, s.lo);
    return fast_two_sum(s.hi, v);
}

// double-word * double-word
__device__ __forceinline__ df df_mul(df x, df y) {
    const df p = two_prod(x.hi, y.hi);
    float t = __fmul_rn(x.hi, y.lo);
    t = __fmaf_rn(x.lo, y.hi, t);
    const float c = __fadd_rn(p.lo, t);
    return fast_two_sum(p.hi, c);
}

// double-word * float
__device__ __forceinline__ df df_mul_f(df x, float y) {
    const df p = two_prod(x.hi, y);
    const float c = __fmaf_rn(x.lo, y, p.lo);
    return fast_two_sum(p.hi, c);
}

// double-word / double-word: approximate quotient of the leading terms, then one
// correction from the remainder x - q*y (formed with an exact product).
__device__ __forceinline__ df df_div(df x, df y) {
    const float ry = __fdividef(1.f, y.hi);
    const float q1 = __fmul_rn(x.hi, ry);
    const df r = df_sub(x, df_mul_f(y, q1));
    const float q2 = __fmul_rn(r.hi, ry);
    return fast_two_sum(q1, q2);
}

// square root of a non-negative double-word: s ~ sqrt(hi) from the approximate
// reciprocal square root, then the Newton correction (x - s^2) / (2 s) with x - s^2
// formed exactly.
__device__ __forceinline__ df df_sqrt(df x) {
    if (!(x.hi > 0.f)) return df_make(0.f, 0.f);
    const float rs = rsqrtf(x.hi);
    const float s = __fmul_rn(x.hi, rs);
    const df s2 = two_prod(s, s);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, s2.hi), s2.lo), x.lo);
    const float c = __fmul_rn(__fmul_rn(r, rs), 0.5f);
    return fast_two_sum(s, c);
}

__device__ __forceinline__ bool df_gt0(df x) { return x.hi > 0.f || (x.hi == 0.f && x.lo > 0.f); }
__device__ __forceinline__ bool df_lt(df x, df y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
__device__ __forceinline__ double df_to_d(df x) { return (double)x.hi + (double)x.lo; }

// Host split of a double into a double-word (hi = nearest float, lo = nearest float of the rest).
inline df df_split(double v) {
    df r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
}

}  // namespace pc
