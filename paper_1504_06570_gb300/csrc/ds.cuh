// Double-single arithmetic: a value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2,
// carrying about 48 significant bits on the FP32 pipes.
//
// GB300 issues FP32 fused multiply-adds about seventy times faster than FP64 ones, so the optics of the
// double-single photon path (positions, directions, surface transforms and intersections: the quantities
// that need more than single precision for micron accuracy over a metre-size focal plane) run on pairs of
// floats instead of doubles.  The building blocks are the error-free transformations of Knuth (TwoSum),
// Dekker (Fast2Sum, 1971) and the FMA-based exact product; the sums are the "sloppy" Dekker sums, whose
// error is bounded relative to the operands (about 2^-47 of the larger), which is the accuracy the optics
// needs (absolute errors against operand sizes of a few metres).  Every primitive is written with the
// IEEE round-to-nearest intrinsics so that the compiler neither contracts nor reorders the transformations.
#pragma once

#include <cuda_runtime.h>

// attributes of the larger primitives (quotient, roots): out of line keeps the photon kernel's code within
// the instruction cache
#ifndef PHOSIM_DS_HEAVY
#define PHOSIM_DS_HEAVY __noinline__
#endif

namespace phosim {

struct ds {
    float hi, lo;
};

// split a double into the nearest double-single pair (host set-up and rare device conversions)
__host__ __device__ __forceinline__ ds ds_of(double v) {
    ds r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
}
__host__ __device__ __forceinline__ double ds_value(ds a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ds ds_f(float v) { return {v, 0.f}; }

// exact: s + e == a + b (Knuth)
__device__ __forceinline__ ds two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// exact when |a| >= |b| (Dekker)
__device__ __forceinline__ ds fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// exact: p + e == a b
__device__ __forceinline__ ds two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ds operator-(ds a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ ds operator+(ds a, ds b) {
    const ds s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ds operator-(ds a, ds b) { return a + (-b); }
__device__ __forceinline__ ds operator+(ds a, float b) {
    const ds s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ds operator-(ds a, float b) { return a + (-b); }

__device__ __forceinline__ ds operator*(ds a, ds b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ds operator*(ds a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return fast_two_sum(p, e);
}

// a b + c with one normalisation
__device__ __forceinline__ ds dfma(ds a, ds b, ds c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    const ds s = two_sum(p, c.hi);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    e = __fadd_rn(e, __fadd_rn(s.lo, c.lo));
    return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ ds dfma(ds a, float b, ds c) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    const ds s = two_sum(p, c.hi);
    e = __fmaf_rn(a.lo, b, e);
    e = __fadd_rn(e, __fadd_rn(s.lo, c.lo));
    return fast_two_sum(s.hi, e);
}

// Two double-single numbers, the x and y components of a vector, carried as packed pairs for Blackwell's FP32x2
// instructions (one issue for both halves).  Every primitive below performs, in each half, exactly the
// operations of its scalar counterpart in the same order (a subtraction as the exact fused form b (-1) + a), so
// the results are bit for bit those of two scalar calls.
struct ds2 {
    float2 hi, lo;
};
__device__ __forceinline__ ds2 ds2_of(ds x, ds y) { return {make_float2(x.hi, y.hi), make_float2(x.lo, y.lo)}; }
__device__ __forceinline__ ds ds2_x(ds2 v) { return {v.hi.x, v.lo.x}; }
__device__ __forceinline__ ds ds2_y(ds2 v) { return {v.hi.y, v.lo.y}; }
__device__ __forceinline__ float2 f2_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ ds2 two_sum2(float2 a, float2 b) {
    const float2 s = __fadd2_rn(a, b);
    const float2 bb = f2_sub(s, a);
    return {s, __fadd2_rn(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb))};
}
__device__ __forceinline__ ds2 fast_two_sum2(float2 a, float2 b) {
    const float2 s = __fadd2_rn(a, b);
    return {s, f2_sub(b, f2_sub(s, a))};
}
// dfma(a, b, c) in each half, a shared
__device__ __forceinline__ ds2 dfma2(ds a, ds2 b, ds2 c) {
    const float2 ah = make_float2(a.hi, a.hi), al = make_float2(a.lo, a.lo);
    const float2 p = __fmul2_rn(ah, b.hi);
    float2 e = __ffma2_rn(ah, b.hi, f2_neg(p));
    const ds2 s = two_sum2(p, c.hi);
    e = __ffma2_rn(ah, b.lo, e);
    e = __ffma2_rn(al, b.hi, e);
    e = __fadd2_rn(e, __fadd2_rn(s.lo, c.lo));
    return fast_two_sum2(s.hi, e);
}
// a * b in each half with a shared (the scalar operator*(a, b))
__device__ __forceinline__ ds2 mul2(ds a, ds2 b) {
    const float2 ah = make_float2(a.hi, a.hi), al = make_float2(a.lo, a.lo);
    const float2 p = __fmul2_rn(ah, b.hi);
    float2 e = __ffma2_rn(ah, b.hi, f2_neg(p));
    e = __ffma2_rn(ah, b.lo, e);
    e = __ffma2_rn(al, b.hi, e);
    return fast_two_sum2(p, e);
}
// a * b in each half with b shared (the scalar operator*(a, b))
__device__ __forceinline__ ds2 mul2(ds2 a, ds b) {
    const float2 bh = make_float2(b.hi, b.hi), bl = make_float2(b.lo, b.lo);
    const float2 p = __fmul2_rn(a.hi, bh);
    float2 e = __ffma2_rn(a.hi, bh, f2_neg(p));
    e = __ffma2_rn(a.hi, bl, e);
    e = __ffma2_rn(a.lo, bh, e);
    return fast_two_sum2(p, e);
}

// a + b in each half (the scalar operator+(a, b))
__device__ __forceinline__ ds2 add2(ds2 a, ds2 b) {
    const ds2 s = two_sum2(a.hi, b.hi);
    return fast_two_sum2(s.hi, __fadd2_rn(s.lo, __fadd2_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ds2 neg2(ds2 a) { return {f2_neg(a.hi), f2_neg(a.lo)}; }
// a + b in each half for a single-precision b (the scalar operator+(a, float))
__device__ __forceinline__ ds2 add2(ds2 a, float2 b) {
    const ds2 s = two_sum2(a.hi, b);
    return fast_two_sum2(s.hi, __fadd2_rn(s.lo, a.lo));
}
// dfma(a, b, c) in each half for a shared single-precision b
__device__ __forceinline__ ds2 dfma2(ds2 a, float b, ds2 c) {
    const float2 bb = make_float2(b, b);
    const float2 p = __fmul2_rn(a.hi, bb);
    float2 e = __ffma2_rn(a.hi, bb, f2_neg(p));
    const ds2 s = two_sum2(p, c.hi);
    e = __ffma2_rn(a.lo, bb, e);
    e = __fadd2_rn(e, __fadd2_rn(s.lo, c.lo));
    return fast_two_sum2(s.hi, e);
}

// Quotient: a single-precision reciprocal estimate r, q1 = a r, then one correction from the remainder
// a - q1 b evaluated in double-single; relative error about 2^-45.
static __device__ PHOSIM_DS_HEAVY ds operator/(ds a, ds b) {
    const float r = __fdividef(1.f, b.hi);
    const float q1 = __fmul_rn(a.hi, r);
    const ds rem = a - b * q1;
    return fast_two_sum(q1, __fmul_rn(rem.hi, r));
}
static __device__ PHOSIM_DS_HEAVY ds ds_rcp(ds b) {
    const float r = __fdividef(1.f, b.hi);
    const ds rem = ds_f(1.f) - b * r;         // 1 - b r, small
    return fast_two_sum(r, __fmul_rn(rem.hi, r));
}

// Square root: y = a rsqrt(a) in single precision, then the Newton correction (a - y^2) / (2 y) with the
// residual exact (two_prod); relative error about 2^-44.  Non-positive arguments give 0.
static __device__ PHOSIM_DS_HEAVY ds ds_sqrt(ds a) {
    if (!(a.hi > 0.f)) return {0.f, 0.f};
    const float r = rsqrtf(a.hi);
    const float y = __fmul_rn(a.hi, r);
    const ds rem = a - two_prod(y, y);
    return fast_two_sum(y, __fmul_rn(rem.hi, __fmul_rn(0.5f, r)));
}

// Reciprocal square root: r0 = rsqrt(a.hi), e = 1 - a r0^2 evaluated in double-single, then the second-
// order Taylor correction r0 (1 + e / 2 + 3 e^2 / 8); relative error at the double-single rounding level.
static __device__ PHOSIM_DS_HEAVY ds ds_rsqrt(ds a) {
    const float r = rsqrtf(a.hi);
    const ds ar2 = a * two_prod(r, r);
    const float e = __fsub_rn(__fsub_rn(1.f, ar2.hi), ar2.lo);
    const float c = __fmul_rn(__fmul_rn(r, e), __fmaf_rn(0.375f, e, 0.5f));
    return fast_two_sum(r, c);
}

__device__ __forceinline__ bool ds_lt(ds a, ds b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool ds_le(ds a, ds b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
__device__ __forceinline__ ds ds_abs(ds a) { return a.hi < 0.f ? -a : a; }

// floor as a float holding an integer (|a| < 2^24); the low part decides when hi is itself an integer
__device__ __forceinline__ float ds_floor(ds a) {
    float f = floorf(a.hi);
    if (f == a.hi) f = __fadd_rn(f, floorf(a.lo));
    return f;
}
// a - f for the f above, rounded to single precision (a number in [0, 1))
__device__ __forceinline__ float ds_frac(ds a, float f) { return __fadd_rn(__fsub_rn(a.hi, f), a.lo); }

// the exact uniform ((w + 1/2) 2^-32) of a 32-bit word as a double-single pair
__device__ __forceinline__ ds ds_uniform(uint32_t w) {
    const float hi = __fmul_rn((float)(w >> 8), 5.9604644775390625e-8f);                  // 2^-24
    const float lo = __fmul_rn((float)(w & 0xffu) + 0.5f, 2.3283064365386963e-10f);       // 2^-32
    return fast_two_sum(hi, lo);
}

}  // namespace phosim
