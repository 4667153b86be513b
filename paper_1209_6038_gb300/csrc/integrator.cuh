// integrator.cuh -- the persistent integration kernel of the wavefront schedule, templated on a
// stepper that fixes the arithmetic:
//
//   Stepper64     FP64 throughout (the arithmetic of the plain path, step for step).
//   StepperMixed  right-hand sides of Eq. 2 / Eq. 8 and the stage combinations in FP32; the state
//                 (x, v) accumulated as float-float (TwoSum, Knuth 1969), so rounding does not build
//                 up over thousands of steps, and stage positions kept as float-float so r - R1 is
//                 formed without cancellation; whole steps in FP64 where r < R1 + 0.02 (where
//                 f -> 0); step control in FP32 on the part of the embedded error estimate that
//                 exceeds its own FP32 rounding bound (the estimate is a difference of nearly equal
//                 stage combinations, so without this the controller would chase rounding noise).
//
//   StepperMixed with the band in double-float (CLOAK_MIXED_FF): the steps within the band are taken
//                 in double-float (pairs of FP32 numbers, ~48 bits, dfloat.cuh) instead of FP64.
//
// Each lane owns one queued ray and refills from the queue when it finishes.  Every loop iteration
// runs ONE uniform step evaluation for all lanes; the surface-crossing search (bisection prefix,
// then Illinois regula falsi, see crossing() in physics.cuh) reuses that slot with a trial size.
#pragma once

#include "dfloat.cuh"
#include "physics.cuh"

namespace ck {

// ------------------------------------------------------------------ FP64 stepper
template <int VAR, int MODE, int INTEG>
struct Stepper64 {
    typedef double real;
    double y[6], k1[6], y1[6], e6[6], k7[6];
    bool need_k1;
    int vm;  // 2 * variant + mode when VAR = MODE = V_ANY

    // state of queue slot k; the first stage comes with it when the entry kernel computed it (Fermat form)
    template <typename Q>
    __device__ __forceinline__ void load(const Q &q, int k) {
        y[0] = q.x[k]; y[1] = q.y[k]; y[2] = q.z[k];
        y[3] = q.vx[k]; y[4] = q.vy[k]; y[5] = q.vz[k];
        const double a0 = q.ax[k];
        need_k1 = a0 != a0;
        if (!need_k1) {
            k1[0] = y[3]; k1[1] = y[4]; k1[2] = y[5];
            k1[3] = a0; k1[4] = q.ay[k]; k1[5] = q.az[k];
        }
    }
    __device__ __forceinline__ void eval(const Params &p, double s) {
        if (INTEG == I_RK4) {
            rk4_step<VAR, MODE>(p, y, s, y1, vm);
        } else {
            if (need_k1) rhs<VAR, MODE>(p, y, k1, vm);
            need_k1 = false;
            dp45_step<VAR, MODE>(p, y, k1, s, y1, e6, k7, vm);
        }
    }
    // DP5(4) step control (physics.cuh: dp_control); fac is the next-step factor
    __device__ __forceinline__ bool control(double tol, double &fac) const { return dp_control(y, y1, e6, tol, fac); }
    __device__ __forceinline__ double chord(const Params &p) const { return metal_chord(y[0], y[1], y1[0], y1[1], p.R1sq); }
    __device__ __forceinline__ double g_start(const Params &p, int ev) const { return event_g(p, ev, y); }
    __device__ __forceinline__ double g_end(const Params &p, int ev) const { return event_g(p, ev, y1); }
    // d/ds of the event function at the end of the last trial step of size s, with the end point's
    // derivative taken as the flow's, f(y1) = k7 (position part): the Newton slope of the crossing search
    __device__ __forceinline__ double g_rate(int ev) const { return event_dg(ev, y1, k7); }
    // the same at the start of the step, from k1 = f(y)
    __device__ __forceinline__ double g_rate_start(int ev) const { return event_dg(ev, y, k1); }
    __device__ __forceinline__ void take_step() {
#pragma unroll
        for (int i = 0; i < 6; ++i) y[i] = y1[i];
        if (INTEG == I_DP45) {
#pragma unroll
            for (int i = 0; i < 6; ++i) k1[i] = k7[i];  // first stage of the next step (FSAL)
        }
    }
    __device__ __forceinline__ void take_crossing() {
#pragma unroll
        for (int i = 0; i < 6; ++i) y[i] = y1[i];
        need_k1 = true;
    }
    __device__ __forceinline__ void mirror() {  // Sect. 4: single mirror ray at the metal cylinder
        double r = hypot(y[0], y[1]), nm0 = y[0] / r, nm1 = y[1] / r;
        double vn = y[3] * nm0 + y[4] * nm1;
        y[3] -= 2.0 * vn * nm0;
        y[4] -= 2.0 * vn * nm1;
        need_k1 = true;
    }
    __device__ __forceinline__ void state(double out[6]) const {
#pragma unroll
        for (int i = 0; i < 6; ++i) out[i] = y[i];
    }
    // final state into queue slot k (FP64 format)
    template <typename Q>
    __device__ __forceinline__ void store(const Q &q, int k) const {
        q.x[k] = y[0]; q.y[k] = y[1]; q.z[k] = y[2];
        q.vx[k] = y[3]; q.vy[k] = y[4]; q.vz[k] = y[5];
    }
};

// ------------------------------------------------------------------ mixed stepper
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// (hi, lo) + d  ->  renormalised (hi', lo')
__device__ __forceinline__ void ff_add(float hi, float lo, float d, float &oh, float &ol) {
    float s, e;
    two_sum(hi, d, s, e);
    e += lo;
    oh = s + e;
    ol = e - (oh - s);
}

// dv/dt of Eq. 8 / Eq. 2 in FP32 with the fast reciprocal square root and division.  The position
// comes as float-float (xh + xl, yh + yl) so that u = r - R1 keeps its relative precision close to
// the inner radius: r^2 is formed exactly (TwoProd / TwoSum) and u = (r^2 - R1^2) / (r + R1) with
// R1^2 as float-float (r^2 - R1^2 is then free of cancellation error).
template <int VAR, int MODE>
__device__ __forceinline__ void accel_f32_fixed(float R1, float R1sq_h, float R1sq_l, float K, float invK, float xh,
                                                float xl, float yh, float yl, float vx, float vy, float vz, float &ax,
                                                float &ay, float &az) {
    if (VAR == V_TEST || (VAR == V_RADIAL && MODE == M_ORD)) {
        ax = 0.f; ay = 0.f; az = 0.f;
        return;
    }
    float px = xh * xh, ex = fmaf(xh, xh, -px);
    float py = yh * yh, ey = fmaf(yh, yh, -py);
    float r2h, r2l;
    two_sum(px, py, r2h, r2l);
    r2l += ex + ey + 2.f * (xh * xl + yh * yl);
    float r2 = r2h + r2l;
    float ir = rsqrtf(r2);
    float r = r2 * ir;
    float x = xh + xl, y = yh + yl;
    float cx = x * ir, cy = y * ir;
    float vr = vx * cx + vy * cy;
    float vt = vy * cx - vx * cy;
    float u = __fdividef((r2h - R1sq_h) + (r2l - R1sq_l), r + R1);
    float g = __fdividef(2.f * R1 * ir, u);  // f'/f
    float ar, at, azz;
    if (MODE == M_EXT) {  // the simplified radial terms of accel_fixed
        const float gvr = -g * vr;
        at = gvr * vt;
        const float R1ir2 = R1 * ir * ir;
        if (VAR == V_RADIAL) {
            ar = R1ir2 * ir * (u * vz * vz - r * vt * vt);
            azz = gvr * vz;
        } else {
            ar = -R1ir2 * vt * vt;
            azz = 0.f;
        }
        (void)K; (void)invK;
    } else {
        float hg = 0.5f * g;
        ar = hg * (vt * vt + vz * vz - vr * vr);
        at = -g * vr * vt;
        azz = -g * vr * vz;
    }
    ax = ar * cx - at * cy;
    ay = ar * cy + at * cx;
    az = azz;
}

// dy/dt of the mixed stepper for one medium, inlined.  t: stage point (float), tl: low parts of its x and
// y.  The batch's medium is chosen once per step (StepperMixed::eval), not per right-hand side: each
// medium's step is one contiguous block of code with its seven right-hand sides inline.  (Inlining all
// four media at every one of the seven call sites overflowed the instruction caches -- "no instruction"
// was three quarters of the warps' stall cycles; one out-of-line right-hand side with the switch inside
// paid a call per stage; the switch per step is 2.5 % faster than that, with identical results.)
template <int VAR, int MODE>
__device__ __forceinline__ void rhs_f32(const Params &p, const float t[6], const float tl[2], float d[6]) {
    d[0] = t[3]; d[1] = t[4]; d[2] = t[5];
    accel_f32_fixed<VAR, MODE>(p.R1f, p.R1sq_hf, p.R1sq_lf, p.Kf, p.invKf, t[0], tl[0], t[1], tl[1], t[3], t[4], t[5],
                               d[3], d[4], d[5]);
}

// ------------------------------------------------------------------ double-float steps (the band near R1)
// The same right-hand side and the same Dormand-Prince / RK4 updates as the FP64 path, in double-float.
struct df3 {
    df x, y, z;
};
template <int VAR, int MODE>
__device__ __noinline__ df3 accel_df_call(df R1, df x, df y, df vx, df vy, df vz, int vm) {
    const df unused;  // K and 1/K: the simplified accelerations of accel_fixed do not read them
    df3 a;
    accel<VAR, MODE, df>(R1, unused, unused, x, y, vx, vy, vz, a.x, a.y, a.z, vm);
    return a;
}
// one medium: inline; the batch's any-medium form: one out-of-line copy with the switch inside
template <int VAR, int MODE>
__device__ __forceinline__ void rhs_df(df R1, const df y[6], df d[6], int vm) {
    d[0] = y[3]; d[1] = y[4]; d[2] = y[5];
    if (VAR != V_ANY) {
        const df unused;  // K and 1/K: the simplified accelerations of accel_fixed do not read them
        accel_fixed<VAR, MODE, df>(R1, unused, unused, y[0], y[1], y[3], y[4], y[5], d[3], d[4], d[5]);
    } else {
        const df3 a = accel_df_call<VAR, MODE>(R1, y[0], y[1], y[3], y[4], y[5], vm);
        d[3] = a.x; d[4] = a.y; d[5] = a.z;
    }
}
template <int VAR, int MODE>
__device__ __forceinline__ void dp45_step_df(df R1, const df y[6], const df k1[6], df h, df out[6], df err[6],
                                             df k7[6], int vm) {
    df k2[6], k3[6], k4[6], k5[6], k6[6], t[6];
    {
        const df c1 = h * df(DP::a21);
#pragma unroll
        for (int i = 0; i < 6; ++i) t[i] = df_fma(c1, k1[i], y[i]);
    }
    rhs_df<VAR, MODE>(R1, t, k2, vm);
    {
        const df c1 = h * df(DP::a31), c2 = h * df(DP::a32);
#pragma unroll
        for (int i = 0; i < 6; ++i) t[i] = df_fma(c2, k2[i], df_fma(c1, k1[i], y[i]));
    }
    rhs_df<VAR, MODE>(R1, t, k3, vm);
    {
        const df c1 = h * df(DP::a41), c2 = h * df(DP::a42), c3 = h * df(DP::a43);
#pragma unroll
        for (int i = 0; i < 6; ++i) t[i] = df_fma(c3, k3[i], df_fma(c2, k2[i], df_fma(c1, k1[i], y[i])));
    }
    rhs_df<VAR, MODE>(R1, t, k4, vm);
    {
        const df c1 = h * df(DP::a51), c2 = h * df(DP::a52), c3 = h * df(DP::a53), c4 = h * df(DP::a54);
#pragma unroll
        for (int i = 0; i < 6; ++i) t[i] = df_fma(c4, k4[i], df_fma(c3, k3[i], df_fma(c2, k2[i], df_fma(c1, k1[i], y[i]))));
    }
    rhs_df<VAR, MODE>(R1, t, k5, vm);
    {
        const df c1 = h * df(DP::a61), c2 = h * df(DP::a62), c3 = h * df(DP::a63), c4 = h * df(DP::a64),
                 c5 = h * df(DP::a65);
#pragma unroll
        for (int i = 0; i < 6; ++i)
            t[i] = df_fma(c5, k5[i], df_fma(c4, k4[i], df_fma(c3, k3[i], df_fma(c2, k2[i], df_fma(c1, k1[i], y[i])))));
    }
    rhs_df<VAR, MODE>(R1, t, k6, vm);
    {
        const df c1 = h * df(DP::b1), c3 = h * df(DP::b3), c4 = h * df(DP::b4), c5 = h * df(DP::b5),
                 c6 = h * df(DP::b6);
#pragma unroll
        for (int i = 0; i < 6; ++i)
            out[i] = df_fma(c6, k6[i], df_fma(c5, k5[i], df_fma(c4, k4[i], df_fma(c3, k3[i], df_fma(c1, k1[i], y[i])))));
    }
    rhs_df<VAR, MODE>(R1, out, k7, vm);
    {
        const df c1 = h * df(DP::e1), c3 = h * df(DP::e3), c4 = h * df(DP::e4), c5 = h * df(DP::e5),
                 c6 = h * df(DP::e6), c7 = h * df(DP::e7);
#pragma unroll
        for (int i = 0; i < 6; ++i)
            err[i] = df_fma(c7, k7[i], df_fma(c6, k6[i], df_fma(c5, k5[i], df_fma(c4, k4[i], df_fma(c3, k3[i], c1 * k1[i])))));
    }
}
template <int VAR, int MODE>
__device__ __forceinline__ void rk4_step_df(df R1, const df y[6], df h, df out[6], int vm) {
    df k[6], acc[6], t[6];
    const df hh = h * 0.5f, h6 = h * df(1.0 / 6.0);
    rhs_df<VAR, MODE>(R1, y, k, vm);
#pragma unroll
    for (int i = 0; i < 6; ++i) { acc[i] = k[i]; t[i] = df_fma(hh, k[i], y[i]); }
    rhs_df<VAR, MODE>(R1, t, k, vm);
#pragma unroll
    for (int i = 0; i < 6; ++i) { acc[i] = acc[i] + k[i] * 2.0f; t[i] = df_fma(hh, k[i], y[i]); }
    rhs_df<VAR, MODE>(R1, t, k, vm);
#pragma unroll
    for (int i = 0; i < 6; ++i) { acc[i] = acc[i] + k[i] * 2.0f; t[i] = df_fma(h, k[i], y[i]); }
    rhs_df<VAR, MODE>(R1, t, k, vm);
#pragma unroll
    for (int i = 0; i < 6; ++i) out[i] = df_fma(h6, acc[i] + k[i], y[i]);
}

// The band's steps near R1 (FP64 or double-float), out of line: rare, large, and kept out of the
// instruction stream of the FP32 steps.  Inputs and outputs pass through the caller's local memory.
template <int VAR, int MODE, int INTEG>
__device__ __noinline__ void band_step_f64(const Params &p, const double *y, double s, double *yo, double *e,
                                           double *k7, int vm) {
    if (INTEG == I_RK4) {
        rk4_step<VAR, MODE>(p, y, s, yo, vm);
    } else {
        double k1[6];
        rhs<VAR, MODE>(p, y, k1, vm);
        dp45_step<VAR, MODE>(p, y, k1, s, yo, e, k7, vm);
    }
}
template <int VAR, int MODE>
__device__ __forceinline__ void dp45_band_df(df R1, const df *y, df hs, df *yo, df *e, df *k7, int vm) {
    df k1[6];
    rhs_df<VAR, MODE>(R1, y, k1, vm);
    dp45_step_df<VAR, MODE>(R1, y, k1, hs, yo, e, k7, vm);
}
template <int VAR, int MODE, int INTEG>
__device__ __noinline__ void band_step_df(float R1h, float R1l, const df *y, float s, df *yo, df *e, df *k7, int vm) {
    const df R1(R1h, R1l), hs(s, 0.f);
    if (VAR == V_ANY && INTEG == I_DP45) {
        // the batch's medium chosen once per step: each medium's step with its right-hand sides inline
        // (a call per stage cost the double-float step 5 % of its integration)
        switch (vm) {
        case 0: dp45_band_df<V_RADIAL, M_ORD>(R1, y, hs, yo, e, k7, vm); break;
        case 1: dp45_band_df<V_RADIAL, M_EXT>(R1, y, hs, yo, e, k7, vm); break;
        case 2: dp45_band_df<V_AZIMUTHAL, M_ORD>(R1, y, hs, yo, e, k7, vm); break;
        default: dp45_band_df<V_AZIMUTHAL, M_EXT>(R1, y, hs, yo, e, k7, vm); break;
        }
        return;
    }
    if (INTEG == I_RK4) {
        rk4_step_df<VAR, MODE>(R1, y, hs, yo, vm);
    } else {
        df k1[6];
        rhs_df<VAR, MODE>(R1, y, k1, vm);
        dp45_step_df<VAR, MODE>(R1, y, k1, hs, yo, e, k7, vm);
    }
}

template <int VAR, int MODE, int INTEG>
struct StepperMixed {
    typedef float real;
    float yh[6], yl[6], k1[6];  // state (float-float) and first stage
    float y1h[6], y1l[6], e6[6], k7[6];
    float n6[6];  // rounding bound of the FP32 error estimate (noise floor)
    bool need_k1;
    int vm;  // 2 * variant + mode when VAR = MODE = V_ANY

    // the queue holds the mixed path's states as float-float pairs: no conversion
    template <typename Q>
    __device__ __forceinline__ void load(const Q &q, int k) {
        const double *a[6] = {q.x, q.y, q.z, q.vx, q.vy, q.vz};
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const float2 v = reinterpret_cast<const float2 *>(a[i])[k];
            yh[i] = v.x;
            yl[i] = v.y;
        }
        need_k1 = true;
    }
    template <typename Q>
    __device__ __forceinline__ void store(const Q &q, int k) const {
        double *a[6] = {q.x, q.y, q.z, q.vx, q.vy, q.vz};
#pragma unroll
        for (int i = 0; i < 6; ++i) reinterpret_cast<float2 *>(a[i])[k] = make_float2(yh[i], yl[i]);
    }
    __device__ __forceinline__ bool island(const Params &p) const {
        if (VAR == V_TEST || (VAR == V_RADIAL && MODE == M_ORD) || (VAR == V_ANY && vm == 0)) return false;
        float x = yh[0] + yl[0], y = yh[1] + yl[1];
        const float lim = p.band_limf;  // 0 without a band
        if (!(lim > 0.f)) return false;
        return x * x + y * y < lim * lim;
    }
    // stage point y + d: x, y as float-float (t, tl), the rest in FP32
    __device__ __forceinline__ void stage(const float d[6], float t[6], float tl[2]) const {
        ff_add(yh[0], yl[0], d[0], t[0], tl[0]);
        ff_add(yh[1], yl[1], d[1], t[1], tl[1]);
#pragma unroll
        for (int i = 2; i < 6; ++i) t[i] = yh[i] + (yl[i] + d[i]);
    }
    __device__ __forceinline__ void eval(const Params &p, float s) {
        if (p.band_df && island(p)) {  // double-float step from the float-float state
            df y[6], yo[6], e[6], kk7[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) y[i] = df(yh[i], yl[i]);
            const df R1(p.R1);
            band_step_df<VAR, MODE, INTEG>(R1.hi, R1.lo, y, s, yo, e, kk7, vm);
            if (INTEG == I_DP45) {
#pragma unroll
                for (int i = 0; i < 6; ++i) { e6[i] = e[i].hi + e[i].lo; k7[i] = kk7[i].hi; n6[i] = 0.f; }
            }
#pragma unroll
            for (int i = 0; i < 6; ++i) { y1h[i] = yo[i].hi; y1l[i] = yo[i].lo; }
            need_k1 = true;
            return;
        }
        if (island(p)) {  // FP64 step from the float-float state
            double y[6], yo[6], e[6], kk7[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) y[i] = (double)yh[i] + (double)yl[i];
            band_step_f64<VAR, MODE, INTEG>(p, y, (double)s, yo, e, kk7, vm);
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                y1h[i] = (float)yo[i];
                y1l[i] = (float)(yo[i] - (double)y1h[i]);
                if (INTEG == I_DP45) { e6[i] = (float)e[i]; k7[i] = (float)kk7[i]; n6[i] = 0.f; }
            }
            need_k1 = true;
            return;
        }
        if (VAR == V_ANY) {
            switch (vm) {
            case 0: eval_f32<V_RADIAL, M_ORD>(p, s); break;
            case 1: eval_f32<V_RADIAL, M_EXT>(p, s); break;
            case 2: eval_f32<V_AZIMUTHAL, M_ORD>(p, s); break;
            default: eval_f32<V_AZIMUTHAL, M_EXT>(p, s); break;
            }
        } else {
            eval_f32<VAR, MODE>(p, s);
        }
    }
    // the FP32 step (RK4, or DP5(4) with its error estimate) of medium V2 / M2 from the float-float state
    template <int V2, int M2>
    __device__ __forceinline__ void eval_f32(const Params &p, float s) {
        float t[6], tl[2], d[6], k2[6], k3[6], k4[6], k5[6], k6[6];
        if (INTEG == I_RK4) {
            float acc[6], kk[6];
            const float z6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            stage(z6, t, tl);
            rhs_f32<V2, M2>(p, t, tl, kk);
#pragma unroll
            for (int i = 0; i < 6; ++i) { acc[i] = kk[i]; d[i] = 0.5f * s * kk[i]; }
            stage(d, t, tl);
            rhs_f32<V2, M2>(p, t, tl, kk);
#pragma unroll
            for (int i = 0; i < 6; ++i) { acc[i] = fmaf(2.f, kk[i], acc[i]); d[i] = 0.5f * s * kk[i]; }
            stage(d, t, tl);
            rhs_f32<V2, M2>(p, t, tl, kk);
#pragma unroll
            for (int i = 0; i < 6; ++i) { acc[i] = fmaf(2.f, kk[i], acc[i]); d[i] = s * kk[i]; }
            stage(d, t, tl);
            rhs_f32<V2, M2>(p, t, tl, kk);
#pragma unroll
            for (int i = 0; i < 6; ++i) ff_add(yh[i], yl[i], s * (1.f / 6.f) * (acc[i] + kk[i]), y1h[i], y1l[i]);
            return;
        }
        if (need_k1) {
            const float z6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            stage(z6, t, tl);
            rhs_f32<V2, M2>(p, t, tl, k1);
            need_k1 = false;
        }
        const float a21 = (float)DP::a21, a31 = (float)DP::a31, a32 = (float)DP::a32, a41 = (float)DP::a41,
                    a42 = (float)DP::a42, a43 = (float)DP::a43, a51 = (float)DP::a51, a52 = (float)DP::a52,
                    a53 = (float)DP::a53, a54 = (float)DP::a54, a61 = (float)DP::a61, a62 = (float)DP::a62,
                    a63 = (float)DP::a63, a64 = (float)DP::a64, a65 = (float)DP::a65, b1 = (float)DP::b1,
                    b3 = (float)DP::b3, b4 = (float)DP::b4, b5 = (float)DP::b5, b6 = (float)DP::b6,
                    c1 = (float)DP::e1, c3 = (float)DP::e3, c4 = (float)DP::e4, c5 = (float)DP::e5,
                    c6 = (float)DP::e6, c7 = (float)DP::e7;
#pragma unroll
        for (int i = 0; i < 6; ++i) d[i] = s * (a21 * k1[i]);
        stage(d, t, tl);
        rhs_f32<V2, M2>(p, t, tl, k2);
#pragma unroll
        for (int i = 0; i < 6; ++i) d[i] = s * (a31 * k1[i] + a32 * k2[i]);
        stage(d, t, tl);
        rhs_f32<V2, M2>(p, t, tl, k3);
#pragma unroll
        for (int i = 0; i < 6; ++i) d[i] = s * (a41 * k1[i] + a42 * k2[i] + a43 * k3[i]);
        stage(d, t, tl);
        rhs_f32<V2, M2>(p, t, tl, k4);
#pragma unroll
        for (int i = 0; i < 6; ++i) d[i] = s * (a51 * k1[i] + a52 * k2[i] + a53 * k3[i] + a54 * k4[i]);
        stage(d, t, tl);
        rhs_f32<V2, M2>(p, t, tl, k5);
#pragma unroll
        for (int i = 0; i < 6; ++i) d[i] = s * (a61 * k1[i] + a62 * k2[i] + a63 * k3[i] + a64 * k4[i] + a65 * k5[i]);
        stage(d, t, tl);
        rhs_f32<V2, M2>(p, t, tl, k6);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            float dd = s * (b1 * k1[i] + b3 * k3[i] + b4 * k4[i] + b5 * k5[i] + b6 * k6[i]);
            ff_add(yh[i], yl[i], dd, y1h[i], y1l[i]);
            t[i] = y1h[i];
        }
        tl[0] = y1l[0];
        tl[1] = y1l[1];
#pragma unroll
        for (int i = 2; i < 6; ++i) t[i] = y1h[i] + y1l[i];
        rhs_f32<V2, M2>(p, t, tl, k7);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            e6[i] = s * (c1 * k1[i] + c3 * k3[i] + c4 * k4[i] + c5 * k5[i] + c6 * k6[i] + c7 * k7[i]);
            // each k_j carries a relative rounding error of a few FP32 ulps; so does their combination
            n6[i] = 8.f * 5.96e-8f * fabsf(s) *
                    (fabsf(c1 * k1[i]) + fabsf(c3 * k3[i]) + fabsf(c4 * k4[i]) + fabsf(c5 * k5[i]) +
                     fabsf(c6 * k6[i]) + fabsf(c7 * k7[i]));
        }
    }
    __device__ __forceinline__ bool control(float tol, float &fac) const {
        bool acc = true, bad = false;
        float fe = 0.f;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            float sc = tol + tol * fmaxf(fabsf(yh[i]), fabsf(y1h[i]));
            float ae = fmaxf(0.f, fabsf(e6[i]) - n6[i]);  // truncation error above the rounding noise
            if (e6[i] != e6[i]) bad = true;
            if (!(ae <= sc)) acc = false;
            fe = fmaxf(fe, __fdividef(ae, sc));
        }
        if (bad) { fac = 0.2f; return false; }
        fac = fe == 0.f ? 5.f : fminf(5.f, fmaxf(0.2f, 0.9f * __powf(fe, -0.2f)));
        if (!(fe < 3.0e38f)) fac = 0.2f;
        return acc;
    }
    // Event functions with the roots and signs of event_g (r^2 - R2^2, z - H/2, -z - H/2, R1^2 - r^2) from
    // the float-float position: r^2 is formed exactly (products by FMA, sums by TwoSum) and the surface
    // constants are float-float, so g keeps its precision where it is small -- next to the root, where the
    // crossing search reads it.  (In plain FP32, g carries an absolute error ~1e-7; on the short chords of
    // grazing rays, where g changes by little more than that, the crossing moved by up to 1e-4.)
    static __device__ __forceinline__ float gval(const Params &p, int ev, const float h[6], const float l[6]) {
        if (ev == EV_TOP) return (h[2] - p.halfH_hf) + (l[2] - p.halfH_lf);
        if (ev == EV_BOT) return (-h[2] - p.halfH_hf) + (-l[2] - p.halfH_lf);
        const float px = h[0] * h[0], ex = fmaf(h[0], h[0], -px);
        const float py = h[1] * h[1], ey = fmaf(h[1], h[1], -py);
        float r2h, r2l;
        two_sum(px, py, r2h, r2l);
        r2l += ex + ey + 2.f * (h[0] * l[0] + h[1] * l[1]);
        if (ev == EV_LAT) return (r2h - p.R2sq_hf) + (r2l - p.R2sq_lf);
        return (p.R1sq_hf - r2h) + (p.R1sq_lf - r2l);
    }
    __device__ __forceinline__ float chord(const Params &p) const {
        return metal_chord(yh[0] + yl[0], yh[1] + yl[1], y1h[0] + y1l[0], y1h[1] + y1l[1], p.R1sq_hf);
    }
    __device__ __forceinline__ float g_start(const Params &p, int ev) const { return gval(p, ev, yh, yl); }
    __device__ __forceinline__ float g_end(const Params &p, int ev) const { return gval(p, ev, y1h, y1l); }
    __device__ __forceinline__ void take_step() {
#pragma unroll
        for (int i = 0; i < 6; ++i) { yh[i] = y1h[i]; yl[i] = y1l[i]; }
        if (INTEG == I_DP45 && !need_k1) {
#pragma unroll
            for (int i = 0; i < 6; ++i) k1[i] = k7[i];
        }
    }
    __device__ __forceinline__ void take_crossing() {
#pragma unroll
        for (int i = 0; i < 6; ++i) { yh[i] = y1h[i]; yl[i] = y1l[i]; }
        need_k1 = true;
    }
    __device__ __forceinline__ void mirror() {
        double y[6];
        state(y);
        double r = hypot(y[0], y[1]), nm0 = y[0] / r, nm1 = y[1] / r;
        double vn = y[3] * nm0 + y[4] * nm1;
        y[3] -= 2.0 * vn * nm0;
        y[4] -= 2.0 * vn * nm1;
#pragma unroll
        for (int i = 3; i < 6; ++i) {
            yh[i] = (float)y[i];
            yl[i] = (float)(y[i] - (double)yh[i]);
        }
        need_k1 = true;
    }
    __device__ __forceinline__ void state(double out[6]) const {
#pragma unroll
        for (int i = 0; i < 6; ++i) out[i] = (double)yh[i] + (double)yl[i];
    }
};

// ------------------------------------------------------------------ lane phases of the persistent loop
// (k_wf_integrate in wavefront.cuh)
enum { PH_STEP = 0, PH_CROSS = 1, PH_FINAL = 2, PH_IDLE = 3 };

}  // namespace ck
