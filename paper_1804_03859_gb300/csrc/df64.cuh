// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats (about 48 significant bits, unit roundoff ~ 2^-48 = 3.6e-15).
//
// Why: on GB300 the FP64 pipe issues 2 lane-operations per clock per SM
// while the FP32 pipe issues 128, so the stepper's FFTs and stencils run
// several times faster as double-float operations on the FP32 pipe than as
// native FP64, at an accuracy that still meets the FP64 parity bar of the
// method (relative L2 error 1e-12 per step).
//
// The operations are the classical error-free transformations: Knuth's
// two-sum, Dekker's fast two-sum (|a| >= |b|), and the product error from a
// fused multiply-add.  Addition is the "sloppy" variant (the low parts are
// added without their own error term): its error is bounded by ~2^-47 times
// |a| + |b|, the behaviour of an FP64 addition with a slightly shorter
// significand.  All intermediate operations use the _rn intrinsics so the
// compiler neither contracts nor reassociates them.
#pragma once

#include <cuda_runtime.h>

namespace nsstab {

struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ df64(int i) : df64((double)i) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

struct __align__(16) df64c {
    df64 x, y;
};

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df64(s, e);
}

__device__ __forceinline__ df64 df_quick_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
    const df64 s = df_two_sum(a.hi, b.hi);
    return df_quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_quick_two_sum(p, e);
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }

}  // namespace nsstab
