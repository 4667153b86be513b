// kernels_surrogate.cu -- the learned surrogate inside a render: network inputs of the queued rays, and
// the gate that finishes the rays whose prediction it trusts (exit rebuilt from k_z / L_z conservation,
// Eq. 12 factor of the exit face, room lookup) and takes them out of the integration.
#include "batch.h"
#include "sur_physics.cuh"
#include "surrogate.h"
#include "wavefront.cuh"

namespace ck {

// one queued ray's network inputs (each as a pair hi, lo in columns j and SUR_IN + j, BF16 or FP16 as f16
// says: the first layer weighs both alike) and whether it entered through the lateral surface (the
// surrogate's support)
__device__ __forceinline__ void sur_feature_row(const Params &p, int mode, const Queue &q, unsigned int k,
                                                const double d[3], uint16_t *X, int f16, unsigned char *elig) {
    const double P[3] = {q.x[k], q.y[k], q.z[k]};
    const bool lateral = fabs(hypot(P[0], P[1]) - p.R2) <= 1e-9 * p.R2 && fabs(P[2]) < p.halfH;
    float x[SUR_IN];
    sur_features(p.R1, p.R2, p.H, p.variant == V_AZIMUTHAL ? 1 : 0, mode, P, d, x);
    uint16_t *row = X + (size_t)k * 64;
#pragma unroll
    for (int j = 0; j < SUR_IN; ++j) sur_split_pair(x[j], f16, row + j, row + SUR_IN + j);
    elig[k] = lateral ? 1 : 0;
}

__global__ void __launch_bounds__(256) k_sur_features(Params p, int mode, int spp, unsigned long long seed, Queue q,
                                                      uint16_t *X, int f16, unsigned char *elig) {
    const unsigned int n = q.count[0];
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const long long idx = q.id[k], pix = idx / spp;
        double o[3], d[3];
        camera_ray(p, (int)(pix % p.W), (int)(pix / p.W), (int)(idx - pix * spp), spp, seed, o, d);
        sur_feature_row(p, mode, q, k, d, X, f16, elig);
    }
}

__global__ void __launch_bounds__(256) k_sur_features_batch(Params p, const ViewDev *views, int nviews, int spp,
                                                            unsigned long long seed, Queue q, uint16_t *X, int f16,
                                                            unsigned char *elig) {
    const unsigned int n = q.count[0];
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double o[3], d[3];
        batch_camera_ray(views, nviews, spp, seed, q.id[k], o, d);
        const int vm = key_vm(q.key[k]);
        Params pv = p;
        pv.variant = vm >> 1;
        sur_feature_row(pv, vm & 1, q, k, d, X, f16, elig);
    }
}

// The gate for one queued ray: if the network is confident (predicted log10 exit error <= gate) and the
// predicted exit lies on the lateral surface, the ray is finished here (exit rebuilt from k_z / L_z
// conservation, Eq. 12 factor of the exit face, room lookup) and leaves the integration.
__device__ __forceinline__ void sur_gate_one(const Params &p, int mode, const Queue &q, unsigned int k,
                                             const double d[3], const float *Y, const unsigned char *elig, float gate,
                                             float4 *samples, cloak_record *recs) {
    if (!elig[k]) return;
    const float *y = Y + (size_t)k * 16;
    if (!(y[4] <= gate) || !(y[1] * y[1] + y[2] * y[2] > 0.f)) return;
    const double P[3] = {q.x[k], q.y[k], q.z[k]};
    // the height moves monotonically along the ray: a predicted exit inside the lateral surface means
    // no cap was crossed -- with a margin of twice the exit-point error the confidence allows
    // (predicted log10 error c bounds the exit-point error by 10 R2 10^c)
    const double margin = 20.0 * p.R2 * (double)exp10f(y[4]);
    if (!(fabs(P[2] + 2.0 * p.R2 * (double)y[0]) < p.halfH - margin)) return;
    double pos[3], dout[3], tof;
    sur_reconstruct(p.R2, p.H, P, d, y, pos, dout, tof);
    double nrm[3], eo, ee, c[3], mdout[3] = {-dout[0], -dout[1], -dout[2]};
    face_normal(EV_LAT, pos, nrm);
    local_material(p, pos, eo, ee, c);
    cloak_record rec;
    float rgb[3] = {0.f, 0.f, 0.f};
    rec.mode = mode;
    rec.steps = 0;
    rec.tof = tof;
    rec.status = CLOAK_RAY_EXITED;
    if (p.variant == V_RADIAL && mode == 0) {
        // radial o-rays run straight inside (eps_o = K constant, Sect. 4): they met the metal
        // cylinder iff the entry line passes within R1 of the axis ahead of the entry point
        const double ux = q.vx[k], uy = q.vy[k], uu = ux * ux + uy * uy;
        const double tc = -(P[0] * ux + P[1] * uy), cr = P[0] * uy - P[1] * ux;
        if (tc > 0.0 && cr * cr < p.R1sq * uu) rec.status = CLOAK_RAY_HIT_METAL_EXITED;
    }
    set_vec(rec.exit_pos, pos);
    set_vec(rec.exit_dir, dout);
    // light from the room enters here and leaves towards the camera at the entry face
    rec.weight = transmission_in(mode, eo, ee, c, nrm, mdout) * q.w_out[k];
    rec.tile_id = room_hit(p, pos, dout, rgb);
    store_sample(samples, recs, q.id[k], rec, rgb);
    // out of the integration: one ray fewer in its cost bucket, slot marked as finished
    atomicSub(q.bins + q.key[k], 1u);
    q.key[k] = -1;
}

__global__ void __launch_bounds__(128) k_sur_gate(Params p, int mode, int spp, unsigned long long seed, Queue q,
                                                  const float *Y, const unsigned char *elig, float gate,
                                                  float4 *samples, cloak_record *recs, const unsigned int *err) {
    if (*err) return;  // the network's forward pass timed out: every ray stays with the integrator
    const unsigned int n = q.count[0];
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const long long idx = q.id[k], pix = idx / spp;
        double o[3], d[3];
        camera_ray(p, (int)(pix % p.W), (int)(pix / p.W), (int)(idx - pix * spp), spp, seed, o, d);
        sur_gate_one(p, mode, q, k, d, Y, elig, gate, samples, recs);
    }
}

__global__ void __launch_bounds__(128) k_sur_gate_batch(Params p, const ViewDev *views, int nviews, int spp,
                                                        unsigned long long seed, Queue q, const float *Y,
                                                        const unsigned char *elig, float gate, float4 *samples,
                                                        const unsigned int *err) {
    if (*err) return;  // the network's forward pass timed out: every ray stays with the integrator
    const unsigned int n = q.count[0];
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double o[3], d[3];
        batch_camera_ray(views, nviews, spp, seed, q.id[k], o, d);
        const int vm = key_vm(q.key[k]);
        Params pv = p;
        pv.variant = vm >> 1;
        sur_gate_one(pv, vm & 1, q, k, d, Y, elig, gate, samples, nullptr);
    }
}

__global__ void k_sur_conf(double R2, double H, unsigned long long seed, long long i0, long long n, const float *Y,
                           float *T_all) {
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const long long i = i0 + b;
    float *T = T_all + i * SUR_TSTRIDE;
    if (T[5] == 0.f) {  // not a lateral exit: outside the surrogate's support
        T[4] = 0.f;
        return;
    }
    double P[3], d[3];
    int mode, variant;
    sur_sample(seed, (unsigned long long)i, R2, H, P, d, mode, variant);
    double p1[3], d1[3], p0[3], d0[3], t1, t0;
    sur_reconstruct(R2, H, P, d, Y + b * 16, p1, d1, t1);
    sur_reconstruct(R2, H, P, d, T, p0, d0, t0);
    double cx = d1[1] * d0[2] - d1[2] * d0[1], cy = d1[2] * d0[0] - d1[0] * d0[2], cz = d1[0] * d0[1] - d1[1] * d0[0];
    double ang = atan2(sqrt(cx * cx + cy * cy + cz * cz), d1[0] * d0[0] + d1[1] * d0[1] + d1[2] * d0[2]);
    // exit error as seen in the image: the room's walls are about ten cylinder radii away, so moving the
    // exit point by dp moves the room point as much as turning the exit ray by dp / (10 R2)
    double dp = sqrt((p1[0] - p0[0]) * (p1[0] - p0[0]) + (p1[1] - p0[1]) * (p1[1] - p0[1]) +
                     (p1[2] - p0[2]) * (p1[2] - p0[2])) / (10.0 * R2);
    T[4] = (float)log10(fmax(ang + dp, 1e-7));
}

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

cudaError_t launch_sur_features(const Params &p, int mode, int spp, unsigned long long seed, const Queue &q, SurNet *s,
                                cudaStream_t st) {
    k_sur_features<<<sm_count() * 8, 256, 0, st>>>(p, mode, spp, seed, q, s->X, s->inf_f16, s->elig);
    return cudaGetLastError();
}

cudaError_t launch_sur_features_batch(const Params &p, const ViewDev *views, int nviews, int spp,
                                      unsigned long long seed, const Queue &q, SurNet *s, cudaStream_t st) {
    k_sur_features_batch<<<sm_count() * 8, 256, 0, st>>>(p, views, nviews, spp, seed, q, s->X, s->inf_f16, s->elig);
    return cudaGetLastError();
}

cudaError_t launch_sur_gate_batch(const Params &p, const ViewDev *views, int nviews, int spp, unsigned long long seed,
                                  const Queue &q, SurNet *s, float4 *samples, cudaStream_t st) {
    k_sur_gate_batch<<<sm_count() * 16, 128, 0, st>>>(p, views, nviews, spp, seed, q, s->Y, s->elig, s->gate, samples,
                                                              s->err);
    return cudaGetLastError();
}

cudaError_t launch_sur_gate(const Params &p, int mode, int spp, unsigned long long seed, const Queue &q, SurNet *s,
                            float4 *samples, cloak_record *recs, cudaStream_t st) {
    k_sur_gate<<<sm_count() * 16, 128, 0, st>>>(p, mode, spp, seed, q, s->Y, s->elig, s->gate, samples, recs,
                                                        s->err);
    return cudaGetLastError();
}

cudaError_t launch_sur_conf_targets(double R2, double H, unsigned long long seed, long long i0, long long n,
                                    const float *Y, float *T_all, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_sur_conf<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(R2, H, seed, i0, n, Y, T_all);
    return cudaGetLastError();
}

}  // namespace ck
