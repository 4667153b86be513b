// sur_physics.cuh -- ray geometry of the learned surrogate (device): training-ray sampling, network
// inputs, regression targets and the exit rebuilt from a prediction.
//
// Both media are invariant under rotation about the axis and translation along it (Eqs. 14, 15), so
// a ray keeps k_z and L_z = (x cross k)_z from the entry face to the exit face.  For a ray that enters
// and leaves through r = R2 the vacuum exit direction is therefore fixed by the exit azimuth: in the
// local (r, theta, z) frame it is the entry direction with its radial component reversed.
#pragma once

#include "physics.cuh"
#include "surrogate.h"

namespace ck {

// x as an unevaluated pair hi + lo of BF16 (f16 = 0) or FP16 (f16 = 1) numbers (bit patterns), the network's
// input representation: the first layer weighs both parts alike
__device__ __forceinline__ void sur_split_pair(float x, int f16, uint16_t *hi, uint16_t *lo) {
    if (f16) {
        const __half h = __float2half_rn(x), l = __float2half_rn(x - __half2float(h));
        *hi = __half_as_ushort(h);
        *lo = __half_as_ushort(l);
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x), l = __float2bfloat16_rn(x - __bfloat162float(h));
        *hi = __bfloat16_as_ushort(h);
        *lo = __bfloat16_as_ushort(l);
    }
}

// local frame at azimuth phi
__device__ __forceinline__ void sur_frame(double phi, double rh[3], double th[3]) {
    double s, c;
    sincos(phi, &s, &c);
    rh[0] = c; rh[1] = s; rh[2] = 0.0;
    th[0] = -s; th[1] = c; th[2] = 0.0;
}

// entry azimuth in [0, 2 pi) and the local components of the vacuum direction
__device__ __forceinline__ double sur_local(const double P[3], const double d[3], double &dr, double &dt,
                                            double &dz) {
    double phi = atan2(P[1], P[0]);
    if (phi < 0.0) phi += 2.0 * M_PI;
    double rh[3], th[3];
    sur_frame(phi, rh, th);
    dr = d[0] * rh[0] + d[1] * rh[1];
    dt = d[0] * th[0] + d[1] * th[1];
    dz = d[2];
    return phi;
}

// The same local components with the frame taken from the position itself (r-hat = (x, y) / r), without
// the azimuth: no FP64 transcendental, which the render-side kernels avoid (the GPU's FP64 unit is scarce).
__device__ __forceinline__ void sur_local_frame(const double P[3], const double d[3], double rh[2], double &dr,
                                                double &dt, double &dz) {
    const double ir = rsqrt_nr(fma(P[0], P[0], P[1] * P[1]));
    rh[0] = P[0] * ir;
    rh[1] = P[1] * ir;
    dr = fma(d[0], rh[0], d[1] * rh[1]);
    dt = fma(d[1], rh[0], -d[0] * rh[1]);
    dz = d[2];
}

// training ray i: entry point uniform on the lateral surface, direction cosine-weighted about the
// inward normal (a uniform point of the unit disc lifted onto the hemisphere), mode and variant uniform
__device__ __forceinline__ void sur_sample(unsigned long long seed, unsigned long long i, double R2, double H,
                                           double P[3], double d[3], int &mode, int &variant) {
    const double u0 = jitter(seed, i, SUR_STREAM, 0), u1 = jitter(seed, i, SUR_STREAM, 1);
    const double u2 = jitter(seed, i, SUR_STREAM, 2), u3 = jitter(seed, i, SUR_STREAM, 3);
    const double u4 = jitter(seed, i, SUR_STREAM, 4);
    double rh[3], th[3];
    sur_frame(2.0 * M_PI * u1, rh, th);
    P[0] = R2 * rh[0]; P[1] = R2 * rh[1]; P[2] = (u0 - 0.5) * H;
    double s, c;
    sincos(2.0 * M_PI * u3, &s, &c);
    const double rho = sqrt(u2), dr = -sqrt(1.0 - u2), dt = rho * c, dz = rho * s;
    d[0] = dr * rh[0] + dt * th[0];
    d[1] = dr * rh[1] + dt * th[1];
    d[2] = dz;
    const int bits = (int)(u4 * 4.0);
    mode = bits & 1;
    variant = bits >> 1;
}

// network inputs: z / (H/2), phi / pi - 1, asin(d_z) / (pi/2), atan2(d_theta, -d_r) / (pi/2),
// 2 mode - 1, 2 variant - 1, R1 / R2.  The angles in FP32: an input enters the network as a pair of
// BF16 or FP16 numbers (16 or 22 significant bits), below FP32's 24.
__device__ __forceinline__ void sur_features(double R1, double R2, double H, int variant, int mode, const double P[3],
                                             const double d[3], float x[SUR_IN]) {
    double rh[2], dr, dt, dz;
    sur_local_frame(P, d, rh, dr, dt, dz);
    float phi = atan2f((float)P[1], (float)P[0]);
    if (phi < 0.f) phi += 2.f * (float)M_PI;
    x[0] = (float)(P[2] / (0.5 * H));
    x[1] = phi * (float)M_1_PI - 1.f;
    x[2] = asinf(fminf(fmaxf((float)dz, -1.f), 1.f)) * (float)M_2_PI;
    x[3] = atan2f((float)dt, (float)-dr) * (float)M_2_PI;
    x[4] = (float)(2 * mode - 1);
    x[5] = (float)(2 * variant - 1);
    x[6] = (float)(R1 / R2);
}

// regression targets of a traced ray: (exit z - entry z) / (2 R2), cos psi, sin psi, tof / 4 with psi the
// exit azimuth's departure from the straight line's -- functions of the direction angles, mode and variant
// alone (both media are invariant under rotation about the axis and translation along it); false unless
// the ray left through the lateral surface
__device__ __forceinline__ bool sur_targets(double R2, double H, const double P[3], const double d[3],
                                            const cloak_record &rec, float t[4]) {
    if (rec.status != CLOAK_RAY_EXITED && rec.status != CLOAK_RAY_HIT_METAL_EXITED) return false;
    const double re = hypot(rec.exit_pos[0], rec.exit_pos[1]);
    if (fabs(re - R2) > 1e-9 * R2 || !(fabs(rec.exit_pos[2]) < 0.5 * H)) return false;
    double dr, dt, dz;
    const double phi = sur_local(P, d, dr, dt, dz);
    const double psi = atan2(rec.exit_pos[1], rec.exit_pos[0]) - (phi + M_PI - 2.0 * atan2(dt, -dr));
    double s, c;
    sincos(psi, &s, &c);
    t[0] = (float)((rec.exit_pos[2] - P[2]) / (2.0 * R2));  // translation along the axis: a height change
    t[1] = (float)c;
    t[2] = (float)s;
    t[3] = (float)(rec.tof * 0.25);
    return true;
}

// exit point on r = R2, vacuum exit direction (k_z, L_z conserved) and time of flight from y[0..3]: the exit
// azimuth is phi + pi - 2 alpha + psi (alpha = atan2(d_theta, -d_r), psi = atan2(y2, y1)), composed as a
// product of unit complex numbers, e^{i phe} = -e^{i phi} conj(e^{i alpha})^2 e^{i psi}, in FP64 algebra
__device__ __forceinline__ void sur_reconstruct(double R2, double H, const double P[3], const double d[3],
                                                const float y[4], double pos[3], double dir[3], double &tof) {
    double e[2], dr, dt, dz;
    sur_local_frame(P, d, e, dr, dt, dz);
    const double ia = rsqrt_nr(fma(dr, dr, dt * dt)), ac = -dr * ia, as = dt * ia;  // e^{i alpha}
    const double bc = fma(ac, ac, -as * as), bs = -2.0 * ac * as;                  // conj(e^{i alpha})^2
    const double y1 = (double)y[1], y2 = (double)y[2], yy = fma(y1, y1, y2 * y2);
    const double ip = yy > 0.0 ? rsqrt_nr(yy) : 0.0;
    const double pc = yy > 0.0 ? y1 * ip : 1.0, ps = y2 * ip;                      // e^{i psi} (psi = 0 at y = 0)
    const double qc = fma(bc, pc, -bs * ps), qs = fma(bc, ps, bs * pc);
    double rh[3], th[3];
    rh[0] = -fma(e[0], qc, -e[1] * qs);
    rh[1] = -fma(e[0], qs, e[1] * qc);
    rh[2] = 0.0;
    th[0] = -rh[1]; th[1] = rh[0]; th[2] = 0.0;
    pos[0] = R2 * rh[0];
    pos[1] = R2 * rh[1];
    pos[2] = P[2] + (double)y[0] * 2.0 * R2;
    dir[0] = -dr * rh[0] + dt * th[0];
    dir[1] = -dr * rh[1] + dt * th[1];
    dir[2] = dz;
    tof = 4.0 * (double)y[3];
}

}  // namespace ck
