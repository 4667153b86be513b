// dfloat.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi) / 2, about 48 significant bits.  Built from the error-free transformations
// TwoSum (Knuth 1969), FastTwoSum (Dekker 1971) and the fused-multiply-add product error
// (a b - round(a b) = fma(a, b, -round(a b)) exactly).
//
// On a part whose FP32 rate is 64 times its FP64 rate, a double-float operation (5 to 11 FP32
// instructions) costs far less pipe time than the FP64 operation it replaces.  The mixed-precision
// stepper uses it for the steps close to the inner radius, where FP32 alone cannot resolve r - R1.
//
// Error bounds (relative, for operands and results away from underflow): add and subtract a few
// 2^-48 of the larger operand; multiply a few 2^-48; reciprocal and 1/sqrt a few 2^-46 (one
// Newton-Raphson correction of an FP32 seed, the residual formed in double-float).  The functions
// compile for the host as well (tests check them against exact rational arithmetic there).
#pragma once

#include <cmath>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace ck {

#define CK_HD __host__ __device__ __forceinline__

struct df {
    float hi, lo;
    CK_HD constexpr df() : hi(0.f), lo(0.f) {}
    CK_HD constexpr df(float h, float l) : hi(h), lo(l) {}
    // nearest double-float to a double (exact for the 48 leading bits); constant-folded for constants
    CK_HD constexpr explicit df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

// FP32 sum and product rounded on their own: on the device the _rn intrinsics are never merged into a
// fused multiply-add by the compiler, which would break the error-free transformations below (the host
// build of the tests compiles with -ffp-contract=off)
CK_HD float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
CK_HD float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
CK_HD float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}

// s + e = a + b exactly
CK_HD void df_two_sum(float a, float b, float &s, float &e) {
    s = f_add(a, b);
    const float bb = f_sub(s, a);
    e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (or a = 0); the result is normalised
CK_HD df df_quick(float a, float b) {
    const float s = f_add(a, b);
    return df(s, f_sub(b, f_sub(s, a)));
}

CK_HD df operator-(df a) { return df(-a.hi, -a.lo); }
CK_HD df operator+(df a, df b) {
    float s, e;
    df_two_sum(a.hi, b.hi, s, e);
    e = f_add(e, f_add(a.lo, b.lo));
    return df_quick(s, e);
}
CK_HD df operator-(df a, df b) { return a + (-b); }
CK_HD df operator*(df a, df b) {
    const float p = f_mul(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_quick(p, e);
}
CK_HD df operator*(df a, float b) {
    const float p = f_mul(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return df_quick(p, e);
}
CK_HD df operator*(float a, df b) { return b * a; }
// a b + c (one product, one sum)
CK_HD df df_fma(df a, df b, df c) { return a * b + c; }

// 1/a: y0 = FP32 reciprocal of a.hi, then y0 (1 + e) with e = 1 - a y0 formed to double-float accuracy
CK_HD df rcp_nr(df a) {
#ifdef __CUDA_ARCH__
    const float y0 = __fdividef(1.0f, a.hi);
#else
    const float y0 = 1.0f / a.hi;
#endif
    float e = fmaf(-a.hi, y0, 1.0f);
    e = fmaf(-a.lo, y0, e);
    return df_quick(y0, f_mul(y0, e));
}
// 1/sqrt(a), a > 0: y0 = FP32 estimate, e = 1 - a y0^2 (y0^2 split exactly), a^(-1/2) = y0 (1 - e)^(-1/2)
// ~ y0 (1 + e/2 + 3 e^2 / 8)
CK_HD df rsqrt_nr(df a) {
#ifdef __CUDA_ARCH__
    const float y0 = rsqrtf(a.hi);
#else
    const float y0 = 1.0f / sqrtf(a.hi);
#endif
    const float p = f_mul(y0, y0);
    const float pe = fmaf(y0, y0, -p);
    float e = fmaf(-a.hi, p, 1.0f);
    e = fmaf(-a.hi, pe, e);
    e = fmaf(-a.lo, p, e);
    return df_quick(y0, f_mul(f_mul(y0, e), fmaf(e, 0.375f, 0.5f)));
}

#undef CK_HD

}  // namespace ck
