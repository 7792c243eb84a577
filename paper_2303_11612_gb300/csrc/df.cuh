// Double-float arithmetic: a value is hi + lo with |lo| <= ulp(hi) / 2, about
// 48 significant bits (unit roundoff near 2^-47 for products and accurate
// sums). Built from the error-free transformations TwoSum (Knuth) and
// TwoProd by FMA (Dekker's splitting is unnecessary with a fused
// multiply-add); the operations follow Hida, Li and Bailey, "Library for
// double-double and quad-double arithmetic" (2007), restated for float pairs.
//
// On this GPU a dependent FP64 operation occupies the SM's narrow FP64 pipe
// for many cycles, so the small serial linear algebra of the extraction runs
// in pairs of FP32 words instead. Sc<T> selects the scalar: df for float
// data, plain double for double data.
#pragma once

#include <cuda_runtime.h>

namespace tk {

struct df {
    float hi, lo;
};

__host__ __device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float z = s - a;
    return {s, (a - (s - z)) + (b - z)};
}
__host__ __device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    const float s = a + b;
    return {s, b - (s - a)};
}
__host__ __device__ __forceinline__ df operator+(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
__host__ __device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }
__host__ __device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__host__ __device__ __forceinline__ df operator*(df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// Scalar traits: conversion, fused update and reciprocal square root.
template <typename S> struct Sc;
template <> struct Sc<df> {
    static __device__ __forceinline__ df zero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ df one() { return {1.f, 0.f}; }
    static __device__ __forceinline__ df from_float(float x) { return {x, 0.f}; }
    static __device__ __forceinline__ df from_double(double x) {
        const float h = (float)x;
        return {h, (float)(x - (double)h)};
    }
    // one rounding to double (relative 2^-53)
    static __device__ __forceinline__ double to_double(df x) { return (double)x.hi + (double)x.lo; }
    static __device__ __forceinline__ float to_float(df x) { return x.hi + x.lo; }
    static __device__ __forceinline__ df fma(df a, df b, df c) { return c + a * b; }
    static __device__ __forceinline__ bool gt(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
    static __device__ __forceinline__ bool finite(df a) { return isfinite(a.hi); }
    // 1/sqrt(a) for a > 0: FP32 estimate y0, one Newton step
    // y1 = y0 + y0 h / 2 with h = 1 - a y0^2 (doubles the ~22 correct bits).
    // y0^2 = p + pe exactly (FMA), and h is of the order of 2^-22, so forming
    // h = 1 - a_hi p - a_hi pe - a_lo p with FMAs in FP32 carries it to about
    // 2^-46 absolute (a_lo pe, below 2^-47, is dropped): a short dependent
    // chain, since this sits on the Cholesky's serial path.
    static __device__ __forceinline__ df rsqrt(df a) {
        const float y0 = rsqrtf(a.hi);
        const float p = y0 * y0;
        const float pe = fmaf(y0, y0, -p);
        float h = fmaf(-a.hi, p, 1.f);
        h = fmaf(-a.hi, pe, h);
        h = fmaf(-a.lo, p, h);
        return fast_two_sum(y0, y0 * (0.5f * h));
    }
};
template <> struct Sc<double> {
    static __device__ __forceinline__ double zero() { return 0.0; }
    static __device__ __forceinline__ double one() { return 1.0; }
    static __device__ __forceinline__ double from_float(float x) { return (double)x; }
    static __device__ __forceinline__ double from_double(double x) { return x; }
    static __device__ __forceinline__ double to_double(double x) { return x; }
    static __device__ __forceinline__ float to_float(double x) { return (float)x; }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
    static __device__ __forceinline__ bool gt(double a, double b) { return a > b; }
    static __device__ __forceinline__ bool finite(double a) { return isfinite(a); }
    // FP32 estimate refined by two Newton steps in FP64 (on the mantissa, so
    // the estimate never underflows or overflows)
    static __device__ __forceinline__ double rsqrt(double d) {
        int e;
        double m = frexp(d, &e);
        if (e & 1) { m *= 2.0; e -= 1; }
        double y = (double)rsqrtf((float)m);
        y = y * ::fma(-0.5 * m * y, y, 1.5);
        y = y * ::fma(-0.5 * m * y, y, 1.5);
        return ldexp(y, -e / 2);
    }
};

// Scalar used by the small linear algebra of data of type T.
template <typename T> struct SmallScalar;
template <> struct SmallScalar<float> { using type = df; };
template <> struct SmallScalar<double> { using type = double; };

}  // namespace tk
