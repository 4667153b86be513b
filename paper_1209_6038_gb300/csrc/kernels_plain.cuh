// kernels_plain.cuh -- the plain FP64 path: one thread per pixel (render), per sample
// (records) or per ray (trace_rays); the whole Sect. 4 pipeline in one kernel.
// This is the comparator the optimised paths are measured against.
#pragma once
#include <cuda_runtime.h>

#include "internal.h"
#include "trace.cuh"

namespace ck {

template <int VAR, int MODE, int INTEG>
__global__ void __launch_bounds__(128) k_render_plain(Params p, int spp, unsigned long long seed, float4 *out) {
    long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= (long long)p.W * p.Hp) return;
    int i = (int)(pix % p.W), j = (int)(pix / p.W);
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
    for (int s = 0; s < spp; ++s) {
        double o[3], d[3];
        camera_ray(p, i, j, s, spp, seed, o, d);
        cloak_record rec;
        float rgb[3];
        trace_ray<VAR, MODE, INTEG>(p, o, d, rec, rgb);
        float w = (float)rec.weight;
        acc0 += w * rgb[0];
        acc1 += w * rgb[1];
        acc2 += w * rgb[2];
        acc3 += w;
    }
    float inv = 1.0f / spp;
    out[pix] = make_float4(acc0 * inv, acc1 * inv, acc2 * inv, acc3 * inv);
}

template <int VAR, int MODE, int INTEG>
__global__ void __launch_bounds__(128) k_records_plain(Params p, int spp, unsigned long long seed,
                                                        cloak_record *out) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long npix = (long long)p.W * p.Hp;
    if (idx >= npix * spp) return;
    long long pix = idx / spp;
    int s = (int)(idx - pix * spp);
    int i = (int)(pix % p.W), j = (int)(pix / p.W);
    double o[3], d[3];
    camera_ray(p, i, j, s, spp, seed, o, d);
    cloak_record rec;
    float rgb[3];
    trace_ray<VAR, MODE, INTEG>(p, o, d, rec, rgb);
    out[idx] = rec;
}

template <int VAR, int MODE, int INTEG>
__global__ void __launch_bounds__(128) k_trace_rays(Params p, const double *rays, long long n, cloak_record *out) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const double *r = rays + 6 * idx;
    double o[3] = {r[0], r[1], r[2]}, d[3] = {r[3], r[4], r[5]};
    cloak_record rec;
    float rgb[3];
    trace_ray<VAR, MODE, INTEG>(p, o, d, rec, rgb);
    out[idx] = rec;
}

// ---------------------------------------------------------------- launchers (one variant per translation unit)
template <int V, int M, int I>
static cudaError_t render_plain_vmi(const Params &p, int spp, unsigned long long seed, float4 *out, cudaStream_t st) {
    long long n = (long long)p.W * p.Hp;
    const int bs = 128;
    k_render_plain<V, M, I><<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(p, spp, seed, out);
    return cudaGetLastError();
}
template <int V, int M, int I>
static cudaError_t records_plain_vmi(const Params &p, int spp, unsigned long long seed, cloak_record *out,
                                     cudaStream_t st) {
    long long n = (long long)p.W * p.Hp * spp;
    const int bs = 128;
    k_records_plain<V, M, I><<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(p, spp, seed, out);
    return cudaGetLastError();
}
template <int V, int M, int I>
static cudaError_t trace_rays_vmi(const Params &p, const double *rays, long long n, cloak_record *out,
                                  cudaStream_t st) {
    const int bs = 128;
    k_trace_rays<V, M, I><<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(p, rays, n, out);
    return cudaGetLastError();
}

#define CK_MI_SWITCH(FN, ...)                                             \
    if (mode == M_ORD && p.integ == I_RK4) return FN<V, M_ORD, I_RK4>(__VA_ARGS__);   \
    if (mode == M_ORD && p.integ == I_DP45) return FN<V, M_ORD, I_DP45>(__VA_ARGS__); \
    if (mode == M_EXT && p.integ == I_RK4) return FN<V, M_EXT, I_RK4>(__VA_ARGS__);   \
    if (mode == M_EXT && p.integ == I_DP45) return FN<V, M_EXT, I_DP45>(__VA_ARGS__); \
    return cudaErrorInvalidValue;

template <int V>
cudaError_t launch_render_plain_v(const Params &p, int mode, int spp, unsigned long long seed, float4 *out,
                                  cudaStream_t st) {
    CK_MI_SWITCH(render_plain_vmi, p, spp, seed, out, st)
}
template <int V>
cudaError_t launch_records_plain_v(const Params &p, int mode, int spp, unsigned long long seed, cloak_record *out,
                                   cudaStream_t st) {
    CK_MI_SWITCH(records_plain_vmi, p, spp, seed, out, st)
}
template <int V>
cudaError_t launch_trace_rays_v(const Params &p, int mode, const double *rays, long long n, cloak_record *out,
                                cudaStream_t st) {
    CK_MI_SWITCH(trace_rays_vmi, p, rays, n, out, st)
}

#define CK_INSTANTIATE_PLAIN(V)                                                                                   \
    template cudaError_t launch_render_plain_v<V>(const Params &, int, int, unsigned long long, float4 *,         \
                                                  cudaStream_t);                                                  \
    template cudaError_t launch_records_plain_v<V>(const Params &, int, int, unsigned long long, cloak_record *,   \
                                                   cudaStream_t);                                                 \
    template cudaError_t launch_trace_rays_v<V>(const Params &, int, const double *, long long, cloak_record *,    \
                                                cudaStream_t);

}  // namespace ck
