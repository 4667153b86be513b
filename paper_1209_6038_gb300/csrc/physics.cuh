// physics.cuh -- device-side physics of the uniaxial cylindrical cloaks
// (Halimeh & Wegener, arXiv:1209.6038), written for sm_103a.
//
// Formulation used on the GPU (equivalent to the paper's equations, chosen for
// few FP64 operations per evaluation):
//   * Eq. 7 with Eq. 14 / 15: in the cylindrical frame (r, theta, z) the
//     auxiliary matrix is diagonal, M = diag(K, f, g) with f = K((r-R1)/r)^2,
//     K = (R2/(R2-R1))^2 and g = f (radial, Eq. 14) or g = K (azimuthal,
//     Eq. 15).  The ordinary ray sees M_o = eps_o I with eps_o = K (radial) or
//     f (azimuthal).
//   * Eq. 8 (and Eq. 2 as its special case M = n^2 I) for a diagonal
//     M = diag(A(r), B(r), G(r)) with A = K constant reduces to
//       a_r = [ B' v_t^2/2 + G' v_z^2/2 - (A - B) v_t^2 / r ] / A  (+ -A' v_r^2/2A)
//       a_t = -(B'/B) v_r v_t,   a_z = -(G'/G) v_r v_z
//     with B'/B = f'/f = 2 R1 / (r (r - R1)).
//   * Sect. 3 entry refraction: tangential k is conserved and the normal
//     component q solves (n^T M^-1 n) q^2 + 2 (n^T M^-1 k_t) q + k_t^T M^-1 k_t - 1 = 0
//     (the extraordinary index surface of Eq. 9), root with inward ray velocity.
//   * Eq. 12 transmission from the 4x4 continuity system of tangential E, H.
#pragma once

#include <cstdint>

#include "cloak.h"

namespace ck {

// ------------------------------------------------------------------ FP64 reciprocal and 1/sqrt
// The equations of motion need one 1/sqrt and one reciprocal per evaluation.  On a part with few FP64
// units per SM these are formed from the coarse hardware approximations (PTX rcp.approx.ftz.f64 and
// rsqrt.approx.ftz.f64, relative error near 2^-20 or better) and one third-order Newton-Raphson step each,
// which leaves a relative error of a few 2^-53 (checked against the IEEE operations in the tests).
//   1/a:         e = 1 - a y0,    1/a = y0 / (1 - e) ~ y0 (1 + e + e^2)
//   1/sqrt(a):   e = 1 - a y0^2,  a^(-1/2) = y0 (1 - e)^(-1/2) ~ y0 (1 + e/2 + 3 e^2 / 8)
// Inputs are positive normal numbers here (r^2 and r - R1 inside the shell); a zero or negative input
// gives inf or NaN, which the step control rejects like the IEEE forms would.
__device__ __forceinline__ double rcp_nr(double a) {
    double y0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(a));
    const double e = fma(-a, y0, 1.0);
    return fma(y0, fma(e, e, e), y0);
}
__device__ __forceinline__ double rsqrt_nr(double a) {
    double y0;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(a));
    const double e = fma(-a * y0, y0, 1.0);
    return fma(y0 * e, fma(e, 0.375, 0.5), y0);
}
__device__ __forceinline__ float rcp_nr(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ float rsqrt_nr(float a) { return rsqrtf(a); }

enum { V_RADIAL = 0, V_AZIMUTHAL = 1, V_TEST = 2 };
enum { M_ORD = 0, M_EXT = 1 };
enum { I_RK4 = 0, I_DP45 = 1 };

struct Params {
    int variant;  // V_*
    double R1, R2, H, halfH, K, invK, R1x2, R1sq, R2sq;
    double eo_t, ee_t, c_t[3];  // homogeneous test medium
    unsigned long long scene_seed;
    int integ;
    int precision;  // 0 FP64, 1 mixed, 2 mixed without the FP64 band (wavefront schedule only)
    double mixed_band;  // FP64 steps where r < R1 + mixed_band (mixed precision)
    int band_df;        // ... taken in double-float instead of FP64
    // FP32 copies for the mixed-precision stepper, rounded once on the host (not converted per step):
    // R1, R2, H/2, K, 1/K, R1^2 as float-float (hi, lo), and the band's outer radius R1 + mixed_band
    // (0 without a band); R2^2 and H/2 as float-float for the event functions of the crossing search
    float R1f, R2f, halfHf, Kf, invKf, R1sq_hf, R1sq_lf, band_limf;
    float R2sq_hf, R2sq_lf, halfH_hf, halfH_lf;
    int dedicated_blocks;  // batched integration: blocks whose warps take the reserved long rays
    // schedule knobs (results do not depend on them): blocks for the slowest rays, rays reserved for them
    // per thread, resolution of the cost buckets (bucket = cost_scale x -log2 |L_z|)
    int long_ray_blocks, reserve_per_thread;
    float cost_scale;
    double h_or_tol;
    long long max_steps;
    // camera
    double eye[3], fw[3], rt[3], up[3], tx, ty;
    int W, Hp;
    // linear polariser in front of the camera: 0 none, 1 along the camera's right vector, 2 along its up vector
    int analyzer;
    // ray equations: 0 Fermat form (Eq. 2 / Eq. 8, state (x, v)); 1 Hamiltonian form (state (x, k), k = M v)
    int formulation;
    // per-sample output of the batched render: 0 colour (w r, w g, w b, w); 1 time-of-flight difference
    // (w dt, w, 0, 0) for the TOF difference images
    int tof;
};

// ------------------------------------------------------------------ helpers
template <typename T>
__device__ __forceinline__ T dot3(const T a[3], const T b[3]) {
    return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
}

// splitmix64 mixing step (Steele, Lea & Flood 2014)
__device__ __forceinline__ uint64_t sm64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double jitter(uint64_t seed, uint64_t pix, uint32_t s, uint32_t dim) {
    uint64_t h = sm64(sm64(sm64(seed) ^ pix) ^ ((uint64_t(s) << 8) | dim));
    return double(h >> 11) * 0x1.0p-53;
}

// ------------------------------------------------------------------ material
// Local uniaxial material (eps_o, eps_e, optic axis c) at x (Eqs. 1, 14, 15).
__device__ __forceinline__ void local_material(const Params &p, const double x[3], double &eo, double &ee,
                                               double c[3]) {
    if (p.variant == V_TEST) {
        eo = p.eo_t;
        ee = p.ee_t;
        c[0] = p.c_t[0]; c[1] = p.c_t[1]; c[2] = p.c_t[2];
        return;
    }
    double r = hypot(x[0], x[1]);
    double q = (r - p.R1) / r;
    double f = p.K * q * q;
    double cx = x[0] / r, cy = x[1] / r;
    if (p.variant == V_RADIAL) {
        eo = p.K; ee = f;
        c[0] = cx; c[1] = cy; c[2] = 0.0;
    } else {
        eo = f; ee = p.K;
        c[0] = -cy; c[1] = cx; c[2] = 0.0;
    }
}

// ------------------------------------------------------------------ equation of motion
// dv/dt of Eq. 8 (extraordinary) or Eq. 2 (ordinary) at (x, v); cylindrical closed form.
// VAR = MODE = -1 selects the medium at run time from vm = 2 * variant + mode (batched rendering).
enum { V_ANY = -1 };
template <int VAR, int MODE, typename T>
__device__ __forceinline__ void accel(T R1, T K, T invK, T x, T y, T vx, T vy, T vz, T &ax, T &ay, T &az, int vm = 0);
template <int VAR, int MODE, typename T>
__device__ __forceinline__ void accel_fixed(T R1, T K, T invK, T x, T y, T vx, T vy, T vz, T &ax, T &ay, T &az) {
    if (VAR == V_TEST || (VAR == V_RADIAL && MODE == M_ORD)) {  // homogeneous: straight lines (Sect. 4)
        ax = T(0); ay = T(0); az = T(0);
        return;
    }
    T r2 = x * x + y * y;
    T ir = rsqrt_nr(r2);
    T r = r2 * ir;
    T cx = x * ir, cy = y * ir;
    T vr = vx * cx + vy * cy;
    T vt = vy * cx - vx * cy;
    T u = r - R1;
    T g = T(2) * R1 * ir * rcp_nr(u);  // f'/f
    T ar, at, azz;
    if (MODE == M_EXT) {
        // With f = K u^2 / r^2 and f' = f g the radial term [f'/2 (v_t^2 + G-part) - (K - f) v_t^2 / r] / K
        // simplifies through 1 - u^2/r^2 = R1 (r + u) / r^2 (u = r - R1):
        //   radial    (M = diag(K, f, f)):  a_r = R1 (u v_z^2 - r v_t^2) / r^3
        //   azimuthal (M = diag(K, f, K)):  a_r = -R1 v_t^2 / r^2
        const T gvr = -g * vr;
        at = gvr * vt;
        const T R1ir2 = R1 * ir * ir;
        if (VAR == V_RADIAL) {
            ar = R1ir2 * ir * (u * vz * vz - r * vt * vt);
            azz = gvr * vz;
        } else {
            ar = -R1ir2 * vt * vt;
            azz = T(0);
        }
        (void)K; (void)invK;
    } else {  // azimuthal ordinary: M = f I, Eq. 2 with n = sqrt(f)
        T hg = T(0.5) * g;
        ar = hg * (vt * vt + vz * vz - vr * vr);
        at = -g * vr * vt;
        azz = -g * vr * vz;
    }
    ax = ar * cx - at * cy;
    ay = ar * cy + at * cx;
    az = azz;
}
template <int VAR, int MODE, typename T>
__device__ __forceinline__ void accel(T R1, T K, T invK, T x, T y, T vx, T vy, T vz, T &ax, T &ay, T &az, int vm) {
    if (VAR != V_ANY) {
        accel_fixed<VAR, MODE, T>(R1, K, invK, x, y, vx, vy, vz, ax, ay, az);
        return;
    }
    switch (vm) {
    case 0: accel_fixed<V_RADIAL, M_ORD, T>(R1, K, invK, x, y, vx, vy, vz, ax, ay, az); break;
    case 1: accel_fixed<V_RADIAL, M_EXT, T>(R1, K, invK, x, y, vx, vy, vz, ax, ay, az); break;
    case 2: accel_fixed<V_AZIMUTHAL, M_ORD, T>(R1, K, invK, x, y, vx, vy, vz, ax, ay, az); break;
    default: accel_fixed<V_AZIMUTHAL, M_EXT, T>(R1, K, invK, x, y, vx, vy, vz, ax, ay, az); break;
    }
}

// d(x, k)/dt of the Hamiltonian form, H = (k^T M^-1 k - 1) / 2: dx/dt = M^-1 k, dk/dt = -dH/dx, in closed
// cylindrical form with k_r = k . r-hat, k_t = k . theta-hat, g = f'/f, u = r - R1:
//   radial e    M^-1 = diag(1/K, 1/f, 1/f): dk_r = g (k_t^2 + k_z^2) / (2 f), dk_t = k_r k_t (1/f - 1/K) / r
//   azimuthal e M^-1 = diag(1/K, 1/f, 1/K): dk_r = g k_t^2 / (2 f),           dk_t = k_r k_t (1/f - 1/K) / r
//   azimuthal o M^-1 = I / f:              dk_r = g |k|^2 / (2 f),           dk_t = 0
//   radial o    M^-1 = I / K:              dk = 0
// (the terms in dk_t come from the rotation of the local frame with x at fixed Cartesian k)
template <int VAR, int MODE>
__device__ __forceinline__ void ham_fixed(double R1, double K, double invK, const double y[6], double dy[6]) {
    const double kx = y[3], ky = y[4], kz = y[5];
    if (VAR == V_RADIAL && MODE == M_ORD) {
        dy[0] = kx * invK; dy[1] = ky * invK; dy[2] = kz * invK;
        dy[3] = 0.0; dy[4] = 0.0; dy[5] = 0.0;
        return;
    }
    const double r2 = y[0] * y[0] + y[1] * y[1];
    const double ir = rsqrt_nr(r2), r = r2 * ir;
    const double cx = y[0] * ir, cy = y[1] * ir;
    const double kr = kx * cx + ky * cy, kt = ky * cx - kx * cy;
    const double u = r - R1, iu = rcp_nr(u);
    const double g = 2.0 * R1 * ir * iu;        // f'/f
    const double invf = invK * r2 * iu * iu;    // 1/f = r^2 / (K u^2)
    double vr, vt, vz, dkr, dkt;
    if (MODE == M_EXT) {
        vr = kr * invK;
        vt = kt * invf;
        dkt = kr * kt * (invf - invK) * ir;
        if (VAR == V_RADIAL) {
            vz = kz * invf;
            dkr = 0.5 * g * invf * (kt * kt + kz * kz);
        } else {
            vz = kz * invK;
            dkr = 0.5 * g * invf * kt * kt;
        }
    } else {  // azimuthal ordinary
        vr = kr * invf;
        vt = kt * invf;
        vz = kz * invf;
        dkr = 0.5 * g * invf * (kr * kr + kt * kt + kz * kz);
        dkt = 0.0;
    }
    dy[0] = vr * cx - vt * cy;
    dy[1] = vr * cy + vt * cx;
    dy[2] = vz;
    dy[3] = dkr * cx - dkt * cy;
    dy[4] = dkr * cy + dkt * cx;
    dy[5] = 0.0;
}

template <int VAR, int MODE>
__device__ __forceinline__ void rhs(const Params &p, const double y[6], double dy[6], int vm = 0) {
    if (p.formulation) {  // Hamiltonian form (radial and azimuthal cloaks)
        if (VAR != V_ANY) {
            ham_fixed<VAR, MODE>(p.R1, p.K, p.invK, y, dy);
            return;
        }
        switch (vm) {
        case 0: ham_fixed<V_RADIAL, M_ORD>(p.R1, p.K, p.invK, y, dy); break;
        case 1: ham_fixed<V_RADIAL, M_EXT>(p.R1, p.K, p.invK, y, dy); break;
        case 2: ham_fixed<V_AZIMUTHAL, M_ORD>(p.R1, p.K, p.invK, y, dy); break;
        default: ham_fixed<V_AZIMUTHAL, M_EXT>(p.R1, p.K, p.invK, y, dy); break;
        }
        return;
    }
    dy[0] = y[3]; dy[1] = y[4]; dy[2] = y[5];
    accel<VAR, MODE, double>(p.R1, p.K, p.invK, y[0], y[1], y[3], y[4], y[5], dy[3], dy[4], dy[5], vm);
}

// ------------------------------------------------------------------ integrators
template <int VAR, int MODE>
__device__ __forceinline__ void rk4_step(const Params &p, const double y[6], double h, double out[6], int vm = 0) {
    double k[6], acc[6], t[6];
    rhs<VAR, MODE>(p, y, k, vm);
#pragma unroll
    for (int i = 0; i < 6; ++i) { acc[i] = k[i]; t[i] = fma(0.5 * h, k[i], y[i]); }
    rhs<VAR, MODE>(p, t, k, vm);
#pragma unroll
    for (int i = 0; i < 6; ++i) { acc[i] = fma(2.0, k[i], acc[i]); t[i] = fma(0.5 * h, k[i], y[i]); }
    rhs<VAR, MODE>(p, t, k, vm);
#pragma unroll
    for (int i = 0; i < 6; ++i) { acc[i] = fma(2.0, k[i], acc[i]); t[i] = fma(h, k[i], y[i]); }
    rhs<VAR, MODE>(p, t, k, vm);
#pragma unroll
    for (int i = 0; i < 6; ++i) out[i] = fma(h * (1.0 / 6.0), acc[i] + k[i], y[i]);
}

// Dormand-Prince 5(4) tableau (Dormand & Prince 1980)
struct DP {
    static constexpr double a21 = 1.0 / 5;
    static constexpr double a31 = 3.0 / 40, a32 = 9.0 / 40;
    static constexpr double a41 = 44.0 / 45, a42 = -56.0 / 15, a43 = 32.0 / 9;
    static constexpr double a51 = 19372.0 / 6561, a52 = -25360.0 / 2187, a53 = 64448.0 / 6561, a54 = -212.0 / 729;
    static constexpr double a61 = 9017.0 / 3168, a62 = -355.0 / 33, a63 = 46732.0 / 5247, a64 = 49.0 / 176,
                            a65 = -5103.0 / 18656;
    static constexpr double b1 = 35.0 / 384, b3 = 500.0 / 1113, b4 = 125.0 / 192, b5 = -2187.0 / 6784,
                            b6 = 11.0 / 84;
    // e = b5th - b4th
    static constexpr double e1 = 35.0 / 384 - 5179.0 / 57600, e3 = 500.0 / 1113 - 7571.0 / 16695,
                            e4 = 125.0 / 192 - 393.0 / 640, e5 = -2187.0 / 6784 + 92097.0 / 339200,
                            e6 = 11.0 / 84 - 187.0 / 2100, e7 = -1.0 / 40;
};

// Fifth-order solution of one DP step of size h from y with first stage k1 = f(y).
// If err != nullptr also returns k7 = f(out) and the embedded error estimate.
template <int VAR, int MODE>
__device__ __forceinline__ void dp45_step(const Params &p, const double y[6], const double k1[6], double h,
                                          double out[6], double *err, double *k7, int vm = 0) {
    // stage points y + sum_l (h a_jl) k_l as FMA chains on the scaled coefficients (one FMA per term)
    double k2[6], k3[6], k4[6], k5[6], k6[6], t[6];
    {
        const double c1 = h * DP::a21;
#pragma unroll
        for (int i = 0; i < 6; ++i) t[i] = fma(c1, k1[i], y[i]);
    }
    rhs<VAR, MODE>(p, t, k2, vm);
    {
        const double c1 = h * DP::a31, c2 = h * DP::a32;
#pragma unroll
        for (int i = 0; i < 6; ++i) t[i] = fma(c2, k2[i], fma(c1, k1[i], y[i]));
    }
    rhs<VAR, MODE>(p, t, k3, vm);
    {
        const double c1 = h * DP::a41, c2 = h * DP::a42, c3 = h * DP::a43;
#pragma unroll
        for (int i = 0; i < 6; ++i) t[i] = fma(c3, k3[i], fma(c2, k2[i], fma(c1, k1[i], y[i])));
    }
    rhs<VAR, MODE>(p, t, k4, vm);
    {
        const double c1 = h * DP::a51, c2 = h * DP::a52, c3 = h * DP::a53, c4 = h * DP::a54;
#pragma unroll
        for (int i = 0; i < 6; ++i) t[i] = fma(c4, k4[i], fma(c3, k3[i], fma(c2, k2[i], fma(c1, k1[i], y[i]))));
    }
    rhs<VAR, MODE>(p, t, k5, vm);
    {
        const double c1 = h * DP::a61, c2 = h * DP::a62, c3 = h * DP::a63, c4 = h * DP::a64, c5 = h * DP::a65;
#pragma unroll
        for (int i = 0; i < 6; ++i)
            t[i] = fma(c5, k5[i], fma(c4, k4[i], fma(c3, k3[i], fma(c2, k2[i], fma(c1, k1[i], y[i])))));
    }
    rhs<VAR, MODE>(p, t, k6, vm);
    {
        const double c1 = h * DP::b1, c3 = h * DP::b3, c4 = h * DP::b4, c5 = h * DP::b5, c6 = h * DP::b6;
#pragma unroll
        for (int i = 0; i < 6; ++i)
            out[i] = fma(c6, k6[i], fma(c5, k5[i], fma(c4, k4[i], fma(c3, k3[i], fma(c1, k1[i], y[i])))));
    }
    if (err) {
        rhs<VAR, MODE>(p, out, k7, vm);
        const double c1 = h * DP::e1, c3 = h * DP::e3, c4 = h * DP::e4, c5 = h * DP::e5, c6 = h * DP::e6,
                     c7 = h * DP::e7;
#pragma unroll
        for (int i = 0; i < 6; ++i)
            err[i] = fma(c7, k7[i], fma(c6, k6[i], fma(c5, k5[i], fma(c4, k4[i], fma(c3, k3[i], c1 * k1[i])))));
    }
}

// DP5(4) step control: accept iff |e_i| <= tol + tol max(|y_i|, |y1_i|) for every component
// (decided in FP64); the step factor 0.9 err^(-1/5), clamped to [0.2, 5], is evaluated in FP32
// (it only sets the next step size).  NaN -> reject with factor 0.2.
__device__ __forceinline__ bool dp_control(const double y[6], const double y1[6], const double e6[6], double tol,
                                           double &fac) {
    bool acc = true, bad = false;
    float fe = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double sc = tol + tol * fmax(fabs(y[i]), fabs(y1[i]));
        double ae = fabs(e6[i]);
        if (ae != ae) bad = true;
        if (!(ae <= sc)) acc = false;
        fe = fmaxf(fe, __fdividef((float)ae, (float)sc));
    }
    if (bad) { fac = 0.2; return false; }
    float f = fe == 0.f ? 5.f : fminf(5.f, fmaxf(0.2f, 0.9f * __powf(fe, -0.2f)));
    if (!(fe < 3.0e38f)) f = 0.2f;
    fac = (double)f;
    return acc;
}

// A DP5(4) step whose end points lie outside the metal cylinder while its chord passes inside r < R1
// is retried with the step shortened to the chord's closest approach (straight radial ordinary rays
// would otherwise step over the metal).  Returns that fraction of the step, or 0.
template <typename T>
__device__ __forceinline__ T metal_chord(T x0, T y0, T x1, T y1, T R1sq) {
    T dx = x1 - x0, dy = y1 - y0, dd = dx * dx + dy * dy;
    T b = -(x0 * dx + y0 * dy);  // (closest-approach fraction) * dd
    // closest approach inside the step (0 < b < dd) and inside the metal: |x0|^2 - b^2/dd < R1^2
    if (!(b > T(0) && b < dd)) return T(0);
    if (!((x0 * x0 + y0 * y0 - R1sq) * dd < b * b)) return T(0);
    return b / dd;
}

// ------------------------------------------------------------------ surfaces
enum { EV_LAT = 0, EV_TOP = 1, EV_BOT = 2, EV_METAL = 3 };
// Event functions: positive once the surface has been crossed.  The radial surfaces use r^2 - R^2,
// which has the same roots and signs as r - R and needs no square root.
// Rate of change of the event function along a motion dx of the position x: grad g(x) . dx.
__device__ __forceinline__ double event_dg(int ev, const double x[3], const double dx[3]) {
    switch (ev) {
    case EV_LAT: return 2.0 * fma(x[0], dx[0], x[1] * dx[1]);
    case EV_TOP: return dx[2];
    case EV_BOT: return -dx[2];
    default: return -2.0 * fma(x[0], dx[0], x[1] * dx[1]);
    }
}
__device__ __forceinline__ double event_g(const Params &p, int ev, const double y[6]) {
    switch (ev) {
    case EV_LAT: return fma(y[0], y[0], y[1] * y[1]) - p.R2sq;
    case EV_TOP: return y[2] - p.halfH;
    case EV_BOT: return -y[2] - p.halfH;
    default: return p.R1sq - fma(y[0], y[0], y[1] * y[1]);
    }
}

// One step of size s from y with the integrator's own update (RK4, or the DP
// fifth-order solution given k1 = f(y)).
template <int VAR, int MODE, int INTEG>
__device__ __forceinline__ void flow(const Params &p, const double y[6], const double k1[6], double s, double out[6],
                                     int vm = 0) {
    if (INTEG == I_RK4) rk4_step<VAR, MODE>(p, y, s, out, vm);
    else dp45_step<VAR, MODE>(p, y, k1, s, out, nullptr, nullptr, vm);
}

// Root s* in (0, h] of g(flow_s(y)) for a surface crossed by the step (g(0) <= 0 < g(h)).
// When a coarse step crosses the surface more than once, the root is the one that
// bisection of [0, h] converges to: the first halvings are plain bisection (same
// midpoints as a pure bisection, so the same root is selected), then Illinois-modified
// regula falsi finishes inside the remaining bracket.
// Returns the end of the final bracket beyond the surface (exits) or before it (metal).
// Halvings before regula falsi: 12 for fixed-step RK4 (coarse steps can cross a surface more than
// once), 4 for the error-controlled DP5(4) steps.  Bracket resolution: 1e-13 of the step (FP64), or a
// regula falsi point on the surface to rounding.
template <int INTEG>
__device__ __forceinline__ constexpr int bisect_prefix() { return INTEG == I_RK4 ? 12 : 4; }
constexpr double CROSS_REL_TOL = 1e-13;
// Regula falsi also stops at a trial point where |g| <= CROSS_G_TOL times the surface's scale (R2^2,
// R1^2 or H/2): the point lies on the surface to the rounding of g.
constexpr double CROSS_G_TOL = 4e-16;
__device__ __forceinline__ double cross_g_scale(const Params &p, int ev) {
    return ev == EV_LAT ? p.R2sq : ev == EV_METAL ? p.R1sq : p.halfH;
}
template <int VAR, int MODE, int INTEG>
__device__ double crossing(const Params &p, const double y[6], const double k1[6], double h, double ghi, int ev) {
    double lo = 0.0, hi = h, glo = event_g(p, ev, y), t[6];
    if (!(glo <= 0.0)) glo = 0.0;
    for (int it = 0; it < bisect_prefix<INTEG>(); ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        flow<VAR, MODE, INTEG>(p, y, k1, mid, t);
        double gm = event_g(p, ev, t);
        if (gm > 0.0) { hi = mid; ghi = gm; }
        else { lo = mid; glo = gm; }
    }
    int side = 0;
    for (int it = 0; it < 200; ++it) {
        if (hi - lo <= CROSS_REL_TOL * hi) break;
        double s;
        if (it < 60 && ghi > glo) s = (lo * ghi - hi * glo) / (ghi - glo);
        else s = 0.5 * (lo + hi);
        if (!(s > lo && s < hi)) s = 0.5 * (lo + hi);
        if (!(s > lo && s < hi)) break;
        flow<VAR, MODE, INTEG>(p, y, k1, s, t);
        double gs = event_g(p, ev, t);
        if (gs > 0.0) {
            hi = s; ghi = gs;
            if (side == 1) glo *= 0.5;
            side = 1;
        } else {
            lo = s; glo = gs;
            if (side == -1) ghi *= 0.5;
            side = -1;
        }
        // the trial point lies on the surface to rounding: it is the crossing
        if (fabs(gs) <= CROSS_G_TOL * cross_g_scale(p, ev)) return s;
    }
    return ev == EV_METAL ? lo : hi;
}

// First entry of o + s d into the finite cylinder r <= R2, |z| <= H/2.
// face: EV_LAT / EV_TOP / EV_BOT, or -1 for a miss.
__device__ __forceinline__ int cylinder_entry(const Params &p, const double o[3], const double d[3], double pt[3],
                                              double n[3]) {
    double best = 1e300;
    int face = -1;
    double a = d[0] * d[0] + d[1] * d[1];
    double b = o[0] * d[0] + o[1] * d[1];
    double c = o[0] * o[0] + o[1] * o[1] - p.R2 * p.R2;
    if (a > 0.0) {
        double disc = b * b - a * c;
        if (disc >= 0.0) {
            double sq = sqrt(disc);
            // nearer root of a s^2 + 2 b s + c = 0 in cancellation-free form
            double s = (b < 0.0) ? c / (-b + sq) : (-b - sq) / a;
            if (s > 0.0 && fabs(o[2] + s * d[2]) <= p.halfH) { best = s; face = EV_LAT; }
        }
    }
    if (d[2] < 0.0) {
        double s = (p.halfH - o[2]) / d[2];
        double px = o[0] + s * d[0], py = o[1] + s * d[1];
        if (s > 0.0 && px * px + py * py <= p.R2 * p.R2 && s < best) { best = s; face = EV_TOP; }
    } else if (d[2] > 0.0) {
        double s = (-p.halfH - o[2]) / d[2];
        double px = o[0] + s * d[0], py = o[1] + s * d[1];
        if (s > 0.0 && px * px + py * py <= p.R2 * p.R2 && s < best) { best = s; face = EV_BOT; }
    }
    if (face < 0) return -1;
    for (int i = 0; i < 3; ++i) pt[i] = o[i] + best * d[i];
    if (face == EV_LAT) {
        double r = hypot(pt[0], pt[1]);
        n[0] = pt[0] / r; n[1] = pt[1] / r; n[2] = 0.0;
    } else {
        n[0] = 0.0; n[1] = 0.0; n[2] = face == EV_TOP ? 1.0 : -1.0;
    }
    return face;
}

__device__ __forceinline__ void face_normal(int ev, const double x[3], double n[3]) {
    if (ev == EV_LAT) {
        double r = hypot(x[0], x[1]);
        n[0] = x[0] / r; n[1] = x[1] / r; n[2] = 0.0;
    } else {
        n[0] = 0.0; n[1] = 0.0; n[2] = ev == EV_TOP ? 1.0 : -1.0;
    }
}

// ------------------------------------------------------------------ interface (Sect. 3)
// Inward wave of the mode with tangential wave vector kt at a face with outward normal n.
// Returns false if the mode is evanescent; else wave vector k and ray velocity v = M^-1 k (Eq. 6).
template <typename T>
__device__ __forceinline__ bool refract_in(int mode, T eo, T ee, const T c[3], const T n[3],
                                           const T kt[3], T k[3], T v[3]) {
    T kt2 = dot3(kt, kt);
    if (mode == M_ORD) {
        T a = eo - kt2;
        if (a < T(0)) return false;
        T q = -sqrt(a);
        T ie = T(1) / eo;
        for (int i = 0; i < 3; ++i) { k[i] = fma(q, n[i], kt[i]); v[i] = k[i] * ie; }
        return true;
    }
    T iee = T(1) / ee, dl = T(1) / eo - iee;
    T cn = dot3(c, n), ckt = dot3(c, kt);
    T A = fma(dl * cn, cn, iee);
    T B = dl * cn * ckt;
    T C = fma(iee, kt2, fma(dl * ckt, ckt, -T(1)));
    T disc = B * B - A * C;
    if (disc < T(0)) return false;
    T sq = sqrt(disc);
    T q;
    if (B > T(0)) q = (-B - sq) / A;
    else q = (-B + sq) > T(0) ? C / (-B + sq) : T(0);
    for (int i = 0; i < 3; ++i) k[i] = fma(q, n[i], kt[i]);
    T ck_ = dot3(c, k);
    for (int i = 0; i < 3; ++i) v[i] = fma(iee, k[i], dl * ck_ * c[i]);
    return true;
}

// k = M v for the mode (Eq. 6 inverted)
template <typename T>
__device__ __forceinline__ void wave_from_velocity(int mode, T eo, T ee, const T c[3],
                                                   const T v[3], T k[3]) {
    if (mode == M_ORD) {
        for (int i = 0; i < 3; ++i) k[i] = eo * v[i];
    } else {
        T cv = dot3(c, v);
        for (int i = 0; i < 3; ++i) k[i] = fma(ee, v[i], (eo - ee) * cv * c[i]);
    }
}

// ---- complex helpers for Eq. 12
template <typename T>
struct cxt {
    T re, im;
};
typedef cxt<double> cx;
template <typename T>
__device__ __forceinline__ cxt<T> C(T a, T b = T(0)) { return cxt<T>{a, b}; }
template <typename T>
__device__ __forceinline__ cxt<T> operator+(cxt<T> a, cxt<T> b) { return cxt<T>{a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cxt<T> operator-(cxt<T> a, cxt<T> b) { return cxt<T>{a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ cxt<T> operator*(cxt<T> a, cxt<T> b) {
    return cxt<T>{fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
template <typename T>
__device__ __forceinline__ cxt<T> operator*(T s, cxt<T> a) { return cxt<T>{s * a.re, s * a.im}; }
template <typename T>
__device__ __forceinline__ cxt<T> cdiv(cxt<T> a, cxt<T> b) {  // a / b = a conj(b) / |b|^2, one reciprocal
    const T id = rcp_nr(b.re * b.re + b.im * b.im);
    return cxt<T>{(a.re * b.re + a.im * b.im) * id, (a.im * b.re - a.re * b.im) * id};
}
template <typename T>
__device__ __forceinline__ T cabs2(cxt<T> a) { return a.re * a.re + a.im * a.im; }
template <typename T>
__device__ __forceinline__ cxt<T> cdot(const cxt<T> a[3], const cxt<T> b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <typename T>
__device__ __forceinline__ void ccross(const cxt<T> a[3], const cxt<T> b[3], cxt<T> o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
template <typename T>
__device__ __forceinline__ T vnorm2(const cxt<T> a[3]) { return cabs2(a[0]) + cabs2(a[1]) + cabs2(a[2]); }
// n . Re(E x conj(H))
template <typename T>
__device__ __forceinline__ T flux_n(const T n[3], const cxt<T> E[3], const cxt<T> H[3]) {
    T s = T(0);
    const int i1[3] = {1, 2, 0}, i2[3] = {2, 0, 1};
    for (int i = 0; i < 3; ++i) {
        // Re(E_a conj(H_b) - E_b conj(H_a))
        int a = i1[i], b = i2[i];
        T re = (E[a].re * H[b].re + E[a].im * H[b].im) - (E[b].re * H[a].re + E[b].im * H[a].im);
        s += n[i] * re;
    }
    return s;
}

// The same operations on real field components: while every wave at a face propagates (its wave vector
// real), the Eq. 12 system is real and is solved in real arithmetic (a quarter of the multiplications);
// the complex form serves faces with an evanescent wave.  fld<F>(a) is a as a field component of type F.
template <typename T>
__device__ __forceinline__ T cdiv(T a, T b) { return a * rcp_nr(b); }
template <typename T>
__device__ __forceinline__ T cabs2(T a) { return a * a; }
template <typename T>
__device__ __forceinline__ T cdot(const T a[3], const T b[3]) { return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2])); }
template <typename T>
__device__ __forceinline__ void ccross(const T a[3], const T b[3], T o[3]) {
    o[0] = fma(a[1], b[2], -a[2] * b[1]);
    o[1] = fma(a[2], b[0], -a[0] * b[2]);
    o[2] = fma(a[0], b[1], -a[1] * b[0]);
}
template <typename T>
__device__ __forceinline__ T vnorm2(const T a[3]) { return cdot(a, a); }
// n . (E x H)
template <typename T>
__device__ __forceinline__ T flux_n(const T n[3], const T E[3], const T H[3]) {
    T x[3];
    ccross(E, H, x);
    return dot3(n, x);
}
template <typename T>
__device__ __forceinline__ T fld_(T a, T *) { return a; }
template <typename T>
__device__ __forceinline__ cxt<T> fld_(T a, cxt<T> *) { return cxt<T>{a, T(0)}; }
template <typename F, typename T>
__device__ __forceinline__ F fld(T a) { return fld_(a, (F *)nullptr); }
template <typename T>
__device__ __forceinline__ T re_(T a) { return a; }
template <typename T>
__device__ __forceinline__ T re_(cxt<T> a) { return a.re; }
template <typename T>
__device__ __forceinline__ T im_(T) { return T(0); }
template <typename T>
__device__ __forceinline__ T im_(cxt<T> a) { return a.im; }

// Inward wave (possibly evanescent: decaying into the medium) of the mode with tangential kt.
template <typename T>
__device__ __forceinline__ void inward_wave_c(int mode, T eo, T ee, const T c[3], const T n[3],
                                              const T kt[3], cxt<T> k[3]) {
    T kr[3], vr[3];
    if (refract_in(mode, eo, ee, c, n, kt, kr, vr)) {
        for (int i = 0; i < 3; ++i) k[i] = C(kr[i]);
        return;
    }
    cxt<T> q;
    if (mode == M_ORD) {
        q = C(T(0), -sqrt(dot3(kt, kt) - eo));
    } else {
        T iee = T(1) / ee, dl = T(1) / eo - iee;
        T cn = dot3(c, n), ckt = dot3(c, kt);
        T A = fma(dl * cn, cn, iee), B = dl * cn * ckt, Cc = iee * dot3(kt, kt) + dl * ckt * ckt - T(1);
        q = C(-B / A, -sqrt(A * Cc - B * B) / A);
    }
    for (int i = 0; i < 3; ++i) k[i] = C(kt[i]) + q * C(n[i]);
}

// Field directions of a plane wave of the mode (Sect. 3): D_o perpendicular to the ordinary
// main section, D_e in the extraordinary main section and perpendicular to k; E = eps^-1 D,
// H = k x E.  Degenerate k parallel to c: D_o along z x k (x x k if that vanishes too).
// ieo = 1/eo, dl = 1/ee - 1/eo; F: T (real k) or cxt<T>.
template <typename T, typename F>
__device__ __forceinline__ void wave_fields_f(int mode, T ieo, T dl, const T c[3], const F k[3], F E[3], F H[3]) {
    F cc[3] = {fld<F>(c[0]), fld<F>(c[1]), fld<F>(c[2])}, Do[3], D[3];
    ccross(cc, k, Do);
    T kk2 = vnorm2(k);
    if (vnorm2(Do) < T(1e-20) * kk2) {
        F z3[3] = {fld<F>(T(0)), fld<F>(T(0)), fld<F>(T(1))};
        ccross(z3, k, Do);
        if (vnorm2(Do) < T(1e-20) * kk2) {
            F x3[3] = {fld<F>(T(1)), fld<F>(T(0)), fld<F>(T(0))};
            ccross(x3, k, Do);
        }
        if (mode == M_EXT) ccross(k, Do, D);
        else for (int i = 0; i < 3; ++i) D[i] = Do[i];
    } else if (mode == M_ORD) {
        for (int i = 0; i < 3; ++i) D[i] = Do[i];
    } else {
        F kk = cdot(k, k), ckk = cdot(cc, k);
        for (int i = 0; i < 3; ++i) D[i] = kk * cc[i] - ckk * k[i];
    }
    // eps^-1 = I/eo + (1/ee - 1/eo) c c^T
    F cD = cdot(cc, D);
    for (int i = 0; i < 3; ++i) E[i] = ieo * D[i] + (dl * c[i]) * cD;
    ccross(k, E, H);
}
template <typename T>
__device__ __forceinline__ void wave_fields(int mode, T eo, T ee, const T c[3], const cxt<T> k[3],
                                            cxt<T> E[3], cxt<T> H[3]) {
    T ieo = T(1) / eo, dl = T(1) / ee - ieo;
    wave_fields_f(mode, ieo, dl, c, k, E, H);
}


template <typename T>
__device__ __forceinline__ void unit_perp(const T n[3], T t[3]) {
    // any unit vector perpendicular to n
    T a[3] = {T(0), T(0), T(0)};
    int m = fabs(n[0]) < fabs(n[1]) ? (fabs(n[0]) < fabs(n[2]) ? 0 : 2) : (fabs(n[1]) < fabs(n[2]) ? 1 : 2);
    a[m] = T(1);
    t[0] = n[1] * a[2] - n[2] * a[1];
    t[1] = n[2] * a[0] - n[0] * a[2];
    t[2] = n[0] * a[1] - n[1] * a[0];
    T l = sqrt(dot3(t, t));
    for (int i = 0; i < 3; ++i) t[i] /= l;
}

template <typename T>
__device__ __forceinline__ void s_basis(const T k[3], const T n[3], T s[3]) {
    s[0] = k[1] * n[2] - k[2] * n[1];
    s[1] = k[2] * n[0] - k[0] * n[2];
    s[2] = k[0] * n[1] - k[1] * n[0];
    T l = sqrt(dot3(s, s));
    if (l < T(1e-12)) unit_perp(n, s);
    else for (int i = 0; i < 3; ++i) s[i] /= l;
}

// Solve the 4x4 system A X = B for NR right-hand sides (Gaussian elimination, partial pivoting), in
// complex (F = cxt<T>) or real (F = T) arithmetic.
template <int NR, typename F>
__device__ bool csolve4(F A[4][4], F B[4][NR]) {
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        auto best = cabs2(A[col][col]);
        for (int r = col + 1; r < 4; ++r) {
            auto v = cabs2(A[r][col]);
            if (v > best) { best = v; piv = r; }
        }
        if (best == decltype(best)(0)) return false;
        if (piv != col) {
            for (int k = 0; k < 4; ++k) { F t = A[col][k]; A[col][k] = A[piv][k]; A[piv][k] = t; }
            for (int k = 0; k < NR; ++k) { F t = B[col][k]; B[col][k] = B[piv][k]; B[piv][k] = t; }
        }
        for (int r = col + 1; r < 4; ++r) {
            F f = cdiv(A[r][col], A[col][col]);
            for (int k = col; k < 4; ++k) A[r][k] = A[r][k] - f * A[col][k];
            for (int k = 0; k < NR; ++k) B[r][k] = B[r][k] - f * B[col][k];
        }
    }
    for (int r = 3; r >= 0; --r)
        for (int k = 0; k < NR; ++k) {
            F s = B[r][k];
            for (int j = r + 1; j < 4; ++j) s = s - A[r][j] * B[j][k];
            B[r][k] = cdiv(s, A[r][r]);
        }
    return true;
}


// Eq. 12, vacuum -> medium, unpolarised light (mean over s and p): transmission into `mode`.  ko, ke: the
// wave vectors of the two inward waves (F = T when both propagate, cxt<T> when one is evanescent).
template <typename T, typename F>
static __device__ __noinline__ T trans_in_f(int mode, T eo, T ee, const T c[3], const T n[3], const T d[3],
                                            const F ko[3], const F ke[3]) {
    const T ieo = T(1) / eo, dl = T(1) / ee - ieo;
    T dn = dot3(d, n), kr[3];
    for (int i = 0; i < 3; ++i) kr[i] = d[i] - T(2) * dn * n[i];
    F Eo[3], Ho[3], Ee[3], He[3];
    wave_fields_f(M_ORD, ieo, dl, c, ko, Eo, Ho);
    wave_fields_f(M_EXT, ieo, dl, c, ke, Ee, He);
    T s[3], pi[3], pr[3], t2[3];
    s_basis(d, n, s);
    pi[0] = s[1] * d[2] - s[2] * d[1]; pi[1] = s[2] * d[0] - s[0] * d[2]; pi[2] = s[0] * d[1] - s[1] * d[0];
    pr[0] = s[1] * kr[2] - s[2] * kr[1]; pr[1] = s[2] * kr[0] - s[0] * kr[2]; pr[2] = s[0] * kr[1] - s[1] * kr[0];
    t2[0] = n[1] * s[2] - n[2] * s[1]; t2[1] = n[2] * s[0] - n[0] * s[2]; t2[2] = n[0] * s[1] - n[1] * s[0];
    // columns: reflected s, reflected p, -o, -e ; rows: E.t1, E.t2, H.t1, H.t2 with t1 = s
    F Ers[3] = {fld<F>(s[0]), fld<F>(s[1]), fld<F>(s[2])}, Erp[3] = {fld<F>(pr[0]), fld<F>(pr[1]), fld<F>(pr[2])},
      Hrs[3], Hrp[3];
    F ckr[3] = {fld<F>(kr[0]), fld<F>(kr[1]), fld<F>(kr[2])};
    ccross(ckr, Ers, Hrs);
    ccross(ckr, Erp, Hrp);
    F ct1[3] = {fld<F>(s[0]), fld<F>(s[1]), fld<F>(s[2])}, ct2[3] = {fld<F>(t2[0]), fld<F>(t2[1]), fld<F>(t2[2])};
    const F *colE[4] = {Ers, Erp, Eo, Ee}, *colH[4] = {Hrs, Hrp, Ho, He};
    F A[4][4], B[4][2];
    for (int j = 0; j < 4; ++j) {
        T sg = j < 2 ? T(1) : -T(1);
        A[0][j] = sg * cdot(colE[j], ct1);
        A[1][j] = sg * cdot(colE[j], ct2);
        A[2][j] = sg * cdot(colH[j], ct1);
        A[3][j] = sg * cdot(colH[j], ct2);
    }
    F cd[3] = {fld<F>(d[0]), fld<F>(d[1]), fld<F>(d[2])};
    T fin[2];
    for (int pol = 0; pol < 2; ++pol) {
        const T *e = pol == 0 ? s : pi;
        F Ei[3] = {fld<F>(e[0]), fld<F>(e[1]), fld<F>(e[2])}, Hi[3];
        ccross(cd, Ei, Hi);
        B[0][pol] = -T(1) * cdot(Ei, ct1);
        B[1][pol] = -T(1) * cdot(Ei, ct2);
        B[2][pol] = -T(1) * cdot(Hi, ct1);
        B[3][pol] = -T(1) * cdot(Hi, ct2);
        fin[pol] = fabs(flux_n(n, Ei, Hi));
    }
    if (!csolve4<2>(A, B)) return T(0);
    const F *Em = mode == M_ORD ? Eo : Ee, *Hm = mode == M_ORD ? Ho : He;
    int row = mode == M_ORD ? 2 : 3;
    T fm = fabs(flux_n(n, Em, Hm));
    return T(0.5) * (cabs2(B[row][0]) * fm / fin[0] + cabs2(B[row][1]) * fm / fin[1]);
}
template <typename T>
__device__ __forceinline__ T transmission_in(int mode, T eo, T ee, const T c[3], const T n[3], const T d[3]) {
    T dn = dot3(d, n), kt[3], ko[3], ke[3], v[3];
    for (int i = 0; i < 3; ++i) kt[i] = d[i] - dn * n[i];
    if (refract_in(M_ORD, eo, ee, c, n, kt, ko, v) && refract_in(M_EXT, eo, ee, c, n, kt, ke, v))
        return trans_in_f<T, T>(mode, eo, ee, c, n, d, ko, ke);
    cxt<T> koc[3], kec[3];
    inward_wave_c(M_ORD, eo, ee, c, n, kt, koc);
    inward_wave_c(M_EXT, eo, ee, c, n, kt, kec);
    return trans_in_f<T, cxt<T>>(mode, eo, ee, c, n, d, koc, kec);
}

// Eq. 12, medium -> vacuum (Sect. 3, last paragraph): fraction of the incident mode's normal
// energy flux carried by the refracted vacuum wave.  0 for total internal reflection.
// axis: a linear polariser the transmitted vacuum wave then meets (nullable): the result is multiplied by
// the fraction of that wave's flux along the axis taken across the wave (Malus's law).  kro, kre: the wave
// vectors of the two reflected (inward) waves (F = T when both propagate, cxt<T> when one is evanescent).
template <typename T, typename F>
static __device__ __noinline__ T trans_out_f(int mode, T eo, T ee, const T c[3], const T n[3], const T k[3],
                                             const T kt[3], T kt2, const F kro[3], const F kre[3], const T *axis) {
    const T ieo = T(1) / eo, dl = T(1) / ee - ieo;
    T kv[3], s[3], pv[3], t2[3];
    T qn = sqrt(T(1) - kt2);
    for (int i = 0; i < 3; ++i) kv[i] = fma(qn, n[i], kt[i]);
    s_basis(kv, n, s);
    pv[0] = s[1] * kv[2] - s[2] * kv[1]; pv[1] = s[2] * kv[0] - s[0] * kv[2]; pv[2] = s[0] * kv[1] - s[1] * kv[0];
    t2[0] = n[1] * s[2] - n[2] * s[1]; t2[1] = n[2] * s[0] - n[0] * s[2]; t2[2] = n[0] * s[1] - n[1] * s[0];
    F ckv[3] = {fld<F>(kv[0]), fld<F>(kv[1]), fld<F>(kv[2])};
    F Es[3] = {fld<F>(s[0]), fld<F>(s[1]), fld<F>(s[2])}, Ep[3] = {fld<F>(pv[0]), fld<F>(pv[1]), fld<F>(pv[2])},
      Hs[3], Hp[3];
    ccross(ckv, Es, Hs);
    ccross(ckv, Ep, Hp);
    F Ero[3], Hro[3], Ere[3], Hre[3], Em[3], Hm[3];
    wave_fields_f(M_ORD, ieo, dl, c, kro, Ero, Hro);
    wave_fields_f(M_EXT, ieo, dl, c, kre, Ere, Hre);
    F ck3[3] = {fld<F>(k[0]), fld<F>(k[1]), fld<F>(k[2])};
    wave_fields_f(mode, ieo, dl, c, ck3, Em, Hm);
    F ct1[3] = {fld<F>(s[0]), fld<F>(s[1]), fld<F>(s[2])}, ct2[3] = {fld<F>(t2[0]), fld<F>(t2[1]), fld<F>(t2[2])};
    const F *colE[4] = {Es, Ep, Ero, Ere}, *colH[4] = {Hs, Hp, Hro, Hre};
    F A[4][4], B[4][1];
    for (int j = 0; j < 4; ++j) {
        T sg = j < 2 ? T(1) : -T(1);
        A[0][j] = sg * cdot(colE[j], ct1);
        A[1][j] = sg * cdot(colE[j], ct2);
        A[2][j] = sg * cdot(colH[j], ct1);
        A[3][j] = sg * cdot(colH[j], ct2);
    }
    B[0][0] = cdot(Em, ct1);
    B[1][0] = cdot(Em, ct2);
    B[2][0] = cdot(Hm, ct1);
    B[3][0] = cdot(Hm, ct2);
    T fm = fabs(flux_n(n, Em, Hm));
    if (!csolve4<1>(A, B)) return T(0);
    F Et[3], Ht[3];
    for (int i = 0; i < 3; ++i) { Et[i] = B[0][0] * Es[i] + B[1][0] * Ep[i]; Ht[i] = B[0][0] * Hs[i] + B[1][0] * Hp[i]; }
    const T Tr = fabs(flux_n(n, Et, Ht)) / fm;
    if (!axis) return Tr;
    // the polariser's axis across the transmitted wave kv
    const T ak = dot3(axis, kv);
    T a[3];
    for (int i = 0; i < 3; ++i) a[i] = axis[i] - ak * kv[i];
    const T al2 = dot3(a, a);
    T er = T(0), ei = T(0), e2 = T(0);
    for (int i = 0; i < 3; ++i) {
        er += re_(Et[i]) * a[i];
        ei += im_(Et[i]) * a[i];
        e2 += re_(Et[i]) * re_(Et[i]) + im_(Et[i]) * im_(Et[i]);
    }
    return al2 > T(0) && e2 > T(0) ? Tr * (er * er + ei * ei) / (al2 * e2) : T(0);
}
template <typename T>
__device__ __forceinline__ T transmission_out(int mode, T eo, T ee, const T c[3], const T n[3], const T k[3],
                                              const T *axis = nullptr) {
    T kn = dot3(k, n), kt[3];
    for (int i = 0; i < 3; ++i) kt[i] = k[i] - kn * n[i];
    T kt2 = dot3(kt, kt);
    if (kt2 > T(1)) return T(0);
    T kro[3], kre[3], v[3];
    if (refract_in(M_ORD, eo, ee, c, n, kt, kro, v) && refract_in(M_EXT, eo, ee, c, n, kt, kre, v))
        return trans_out_f<T, T>(mode, eo, ee, c, n, k, kt, kt2, kro, kre, axis);
    cxt<T> kroc[3], krec[3];
    inward_wave_c(M_ORD, eo, ee, c, n, kt, kroc);
    inward_wave_c(M_EXT, eo, ee, c, n, kt, krec);
    return trans_out_f<T, cxt<T>>(mode, eo, ee, c, n, k, kt, kt2, kroc, krec, axis);
}


// First-order reflections (Sect. 3 last paragraphs, Sect. 4).
// Reflection coefficients of a wave of `mode` (real wave vector k, travelling towards the face with outward
// normal n) into the ordinary and extraordinary waves it reflects into: R[0], R[1].  Under total internal
// reflection (|k_t| > 1) the vacuum side carries the evanescent wave that decays away from the face and
// R[0] + R[1] = 1.  Returns false if the 4x4 field-continuity system is singular.
static __device__ __noinline__ bool internal_reflection(int mode, double eo, double ee, const double c[3],
                                                        const double n[3], const double k[3], double R[2]) {
    double kn = dot3(k, n), kt[3];
    for (int i = 0; i < 3; ++i) kt[i] = k[i] - kn * n[i];
    const double kt2 = dot3(kt, kt);
    const bool tir = kt2 > 1.0;
    const double qn = sqrt(fabs(1.0 - kt2));
    cx kv[3];
    for (int i = 0; i < 3; ++i) kv[i] = tir ? cx{kt[i], qn * n[i]} : cx{fma(qn, n[i], kt[i]), 0.0};
    double s[3];
    s_basis(kt, n, s);  // perpendicular to the plane of incidence (kt x n); p = s x k
    cx Es[3] = {C(s[0]), C(s[1]), C(s[2])}, Ep[3], Hs[3], Hp[3];
    ccross(Es, kv, Ep);
    ccross(kv, Es, Hs);
    ccross(kv, Ep, Hp);
    cx t2c[3] = {C(n[1] * s[2] - n[2] * s[1]), C(n[2] * s[0] - n[0] * s[2]), C(n[0] * s[1] - n[1] * s[0])};
    cx ct1[3] = {C(s[0]), C(s[1]), C(s[2])};
    cx kro[3], kre[3], Ero[3], Hro[3], Ere[3], Hre[3], Em[3], Hm[3];
    inward_wave_c(M_ORD, eo, ee, c, n, kt, kro);
    inward_wave_c(M_EXT, eo, ee, c, n, kt, kre);
    wave_fields(M_ORD, eo, ee, c, kro, Ero, Hro);
    wave_fields(M_EXT, eo, ee, c, kre, Ere, Hre);
    cx ck3[3] = {C(k[0]), C(k[1]), C(k[2])};
    wave_fields(mode, eo, ee, c, ck3, Em, Hm);
    const cx *colE[4] = {Es, Ep, Ero, Ere}, *colH[4] = {Hs, Hp, Hro, Hre};
    cx A[4][4], B[4][1];
    for (int j = 0; j < 4; ++j) {
        double sg = j < 2 ? 1.0 : -1.0;
        A[0][j] = sg * cdot(colE[j], ct1);
        A[1][j] = sg * cdot(colE[j], t2c);
        A[2][j] = sg * cdot(colH[j], ct1);
        A[3][j] = sg * cdot(colH[j], t2c);
    }
    B[0][0] = cdot(Em, ct1);
    B[1][0] = cdot(Em, t2c);
    B[2][0] = cdot(Hm, ct1);
    B[3][0] = cdot(Hm, t2c);
    const double fm = fabs(flux_n(n, Em, Hm));
    R[0] = R[1] = 0.0;
    if (!csolve4<1>(A, B) || !(fm > 0.0)) return false;
    R[0] = cabs2(B[2][0]) * fabs(flux_n(n, Ero, Hro)) / fm;
    R[1] = cabs2(B[3][0]) * fabs(flux_n(n, Ere, Hre)) / fm;
    return true;
}

// Fraction of unpolarised room light that the outer surface at a face point (normal n, local material)
// reflects into the camera ray d, through the camera's polariser `axis` (nullable).  By reciprocity of the
// lossless interface this is the mean over the camera-side polarisations of the reflectance of a vacuum
// wave incident along d: (R_s + R_p) / 2, or behind a polariser R(e) / 2 for the incident polarisation e
// along the polariser's axis taken across d.
static __device__ __noinline__ double vacuum_reflection(double eo, double ee, const double c[3], const double n[3],
                                                        const double d[3], const double *axis) {
    double dn = dot3(d, n), kt[3], kr[3];
    for (int i = 0; i < 3; ++i) { kt[i] = d[i] - dn * n[i]; kr[i] = d[i] - 2.0 * dn * n[i]; }
    cx ko[3], ke[3], Eo[3], Ho[3], Ee[3], He[3];
    inward_wave_c(M_ORD, eo, ee, c, n, kt, ko);
    inward_wave_c(M_EXT, eo, ee, c, n, kt, ke);
    wave_fields(M_ORD, eo, ee, c, ko, Eo, Ho);
    wave_fields(M_EXT, eo, ee, c, ke, Ee, He);
    double s[3], pi[3], pr[3], t2[3];
    s_basis(d, n, s);
    pi[0] = s[1] * d[2] - s[2] * d[1]; pi[1] = s[2] * d[0] - s[0] * d[2]; pi[2] = s[0] * d[1] - s[1] * d[0];
    pr[0] = s[1] * kr[2] - s[2] * kr[1]; pr[1] = s[2] * kr[0] - s[0] * kr[2]; pr[2] = s[0] * kr[1] - s[1] * kr[0];
    t2[0] = n[1] * s[2] - n[2] * s[1]; t2[1] = n[2] * s[0] - n[0] * s[2]; t2[2] = n[0] * s[1] - n[1] * s[0];
    cx Ers[3] = {C(s[0]), C(s[1]), C(s[2])}, Erp[3] = {C(pr[0]), C(pr[1]), C(pr[2])}, Hrs[3], Hrp[3];
    cx ckr[3] = {C(kr[0]), C(kr[1]), C(kr[2])};
    ccross(ckr, Ers, Hrs);
    ccross(ckr, Erp, Hrp);
    cx ct1[3] = {C(s[0]), C(s[1]), C(s[2])}, ct2[3] = {C(t2[0]), C(t2[1]), C(t2[2])};
    const cx *colE[4] = {Ers, Erp, Eo, Ee}, *colH[4] = {Hrs, Hrp, Ho, He};
    cx A[4][4], B[4][2];
    for (int j = 0; j < 4; ++j) {
        double sg = j < 2 ? 1.0 : -1.0;
        A[0][j] = sg * cdot(colE[j], ct1);
        A[1][j] = sg * cdot(colE[j], ct2);
        A[2][j] = sg * cdot(colH[j], ct1);
        A[3][j] = sg * cdot(colH[j], ct2);
    }
    // incident polarisations: s and p, or the polariser's axis across d (second column unused)
    double e[2][3];
    for (int i = 0; i < 3; ++i) { e[0][i] = s[i]; e[1][i] = pi[i]; }
    if (axis) {
        const double ad = dot3(axis, d);
        double a[3];
        for (int i = 0; i < 3; ++i) a[i] = axis[i] - ad * d[i];
        const double al = sqrt(dot3(a, a));
        if (!(al > 0.0)) return 0.0;
        for (int i = 0; i < 3; ++i) e[0][i] = a[i] / al;
    }
    cx cd[3] = {C(d[0]), C(d[1]), C(d[2])};
    double fin[2];
    for (int pol = 0; pol < 2; ++pol) {
        cx Ei[3] = {C(e[pol][0]), C(e[pol][1]), C(e[pol][2])}, Hi[3];
        ccross(cd, Ei, Hi);
        B[0][pol] = -1.0 * cdot(Ei, ct1);
        B[1][pol] = -1.0 * cdot(Ei, ct2);
        B[2][pol] = -1.0 * cdot(Hi, ct1);
        B[3][pol] = -1.0 * cdot(Hi, ct2);
        fin[pol] = fabs(flux_n(n, Ei, Hi));
    }
    if (!csolve4<2>(A, B)) return 0.0;
    double Rv[2];
    for (int pol = 0; pol < 2; ++pol) {
        cx Er[3], Hr[3];
        for (int i = 0; i < 3; ++i) {
            Er[i] = B[0][pol] * Ers[i] + B[1][pol] * Erp[i];
            Hr[i] = B[0][pol] * Hrs[i] + B[1][pol] * Hrp[i];
        }
        Rv[pol] = fabs(flux_n(n, Er, Hr)) / fin[pol];
    }
    return axis ? 0.5 * Rv[0] : 0.5 * (Rv[0] + Rv[1]);
}

// axis of the camera's polariser, or null
__device__ __forceinline__ const double *analyzer_axis(const Params &p) {
    return p.analyzer == 1 ? p.rt : p.analyzer == 2 ? p.up : nullptr;
}

// ------------------------------------------------------------------ room and camera
// Distance along the unit direction d from o to the room's box (below) and the face reached (-1: none).
__device__ __forceinline__ double room_distance(const Params &p, const double o[3], const double d[3], int &face) {
    const double Lb = 10.0, z0 = -p.halfH, z1 = z0 + 10.0;
    double best = 1e300, s;
    face = -1;
    if (d[0] > 0.0) { s = (Lb - o[0]) / d[0]; if (s < best) { best = s; face = 0; } }
    else if (d[0] < 0.0) { s = (-Lb - o[0]) / d[0]; if (s < best) { best = s; face = 1; } }
    if (d[1] > 0.0) { s = (Lb - o[1]) / d[1]; if (s < best) { best = s; face = 2; } }
    else if (d[1] < 0.0) { s = (-Lb - o[1]) / d[1]; if (s < best) { best = s; face = 3; } }
    if (d[2] < 0.0) { s = (z0 - o[2]) / d[2]; if (s < best) { best = s; face = 4; } }
    else if (d[2] > 0.0) { s = (z1 - o[2]) / d[2]; if (s < best) { best = s; face = 5; } }
    return best;
}
// Procedural room: box x, y in [-10, 10], z in [-H/2, -H/2 + 10]; checkered walls and floor with
// 8 tiles per unit and splitmix64-hashed tints; constant ceiling.  Returns the tile id.
__device__ __forceinline__ int room_hit(const Params &p, const double o[3], const double d[3], float rgb[3]) {
    const double Lb = 10.0, z0 = -p.halfH;
    int face;
    const double best = room_distance(p, o, d, face);
    if (face < 0) { rgb[0] = rgb[1] = rgb[2] = 0.f; return -1; }
    if (face == 5) { rgb[0] = 0.55f; rgb[1] = 0.55f; rgb[2] = 0.6f; return 5 << 20; }
    double qx = o[0] + best * d[0], qy = o[1] + best * d[1], qz = o[2] + best * d[2];
    double u, v;
    int nv;
    if (face <= 1) { u = qy + Lb; v = qz - z0; nv = 80; }
    else if (face <= 3) { u = qx + Lb; v = qz - z0; nv = 80; }
    else { u = qx + Lb; v = qy + Lb; nv = 160; }
    int i = (int)floor(u * 8.0), j = (int)floor(v * 8.0);
    i = min(max(i, 0), 159);
    j = min(max(j, 0), nv - 1);
    uint64_t h = sm64(sm64(sm64(sm64(p.scene_seed) ^ uint64_t(face)) ^ uint64_t(i)) ^ uint64_t(j));
    float base = ((i + j) & 1) ? 0.25f : 0.85f;
    for (int c = 0; c < 3; ++c) rgb[c] = base * (0.6f + 0.4f * float((h >> (8 * c)) & 255u) / 255.0f);
    return (face << 20) | (i << 10) | j;
}

__device__ __forceinline__ void camera_ray(const Params &p, int i, int j, int s, int spp, uint64_t seed, double o[3],
                                           double d[3]) {
    double xi1 = 0.5, xi2 = 0.5;
    if (spp > 1) {
        uint64_t pix = uint64_t(j) * uint64_t(p.W) + uint64_t(i);
        xi1 = jitter(seed, pix, s, 0);
        xi2 = jitter(seed, pix, s, 1);
    }
    double px = (2.0 * (i + xi1) / p.W - 1.0) * p.tx;
    double py = (1.0 - 2.0 * (j + xi2) / p.Hp) * p.ty;
    double l2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        d[k] = p.fw[k] + px * p.rt[k] + py * p.up[k];
        l2 += d[k] * d[k];
    }
    double il = 1.0 / sqrt(l2);
    for (int k = 0; k < 3; ++k) { d[k] *= il; o[k] = p.eye[k]; }
}

}  // namespace ck
