// internal.h -- declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include "cloak.h"
#include "physics.cuh"

namespace ck {

template <int V>
cudaError_t launch_render_plain_v(const Params &p, int mode, int spp, unsigned long long seed, float4 *out,
                                  cudaStream_t st);
template <int V>
cudaError_t launch_records_plain_v(const Params &p, int mode, int spp, unsigned long long seed, cloak_record *out,
                                   cudaStream_t st);
template <int V>
cudaError_t launch_trace_rays_v(const Params &p, int mode, const double *rays, long long n, cloak_record *out,
                                cudaStream_t st);
extern template cudaError_t launch_render_plain_v<0>(const Params &, int, int, unsigned long long, float4 *, cudaStream_t);
extern template cudaError_t launch_render_plain_v<1>(const Params &, int, int, unsigned long long, float4 *, cudaStream_t);
extern template cudaError_t launch_render_plain_v<2>(const Params &, int, int, unsigned long long, float4 *, cudaStream_t);
extern template cudaError_t launch_records_plain_v<0>(const Params &, int, int, unsigned long long, cloak_record *, cudaStream_t);
extern template cudaError_t launch_records_plain_v<1>(const Params &, int, int, unsigned long long, cloak_record *, cudaStream_t);
extern template cudaError_t launch_records_plain_v<2>(const Params &, int, int, unsigned long long, cloak_record *, cudaStream_t);
extern template cudaError_t launch_trace_rays_v<0>(const Params &, int, const double *, long long, cloak_record *, cudaStream_t);
extern template cudaError_t launch_trace_rays_v<1>(const Params &, int, const double *, long long, cloak_record *, cudaStream_t);
extern template cudaError_t launch_trace_rays_v<2>(const Params &, int, const double *, long long, cloak_record *, cudaStream_t);

inline cudaError_t launch_render_plain(const Params &p, int mode, int spp, unsigned long long seed, float4 *out,
                                cudaStream_t st) {
    if (p.variant == V_RADIAL) return launch_render_plain_v<0>(p, mode, spp, seed, out, st);
    if (p.variant == V_AZIMUTHAL) return launch_render_plain_v<1>(p, mode, spp, seed, out, st);
    return launch_render_plain_v<2>(p, mode, spp, seed, out, st);
}
inline cudaError_t launch_records_plain(const Params &p, int mode, int spp, unsigned long long seed, cloak_record *out,
                                 cudaStream_t st) {
    if (p.variant == V_RADIAL) return launch_records_plain_v<0>(p, mode, spp, seed, out, st);
    if (p.variant == V_AZIMUTHAL) return launch_records_plain_v<1>(p, mode, spp, seed, out, st);
    return launch_records_plain_v<2>(p, mode, spp, seed, out, st);
}
inline cudaError_t launch_trace_rays(const Params &p, int mode, const double *rays, long long n, cloak_record *out,
                              cudaStream_t st) {
    if (p.variant == V_RADIAL) return launch_trace_rays_v<0>(p, mode, rays, n, out, st);
    if (p.variant == V_AZIMUTHAL) return launch_trace_rays_v<1>(p, mode, rays, n, out, st);
    return launch_trace_rays_v<2>(p, mode, rays, n, out, st);
}

struct Queue;
// A step run between the entry kernel and the sort of the wavefront schedule (the learned surrogate
// finishes the rays it is confident about there).
struct WfHook {
    cudaError_t (*fn)(void *ctx, const Queue &q, cudaStream_t st);
    void *ctx;
};
template <int V>
cudaError_t launch_wavefront_v(const Params &p, int mode, int spp, unsigned long long seed, const Queue &q,
                               float4 *samples, cloak_record *recs, int packet, cudaStream_t st, cudaEvent_t *ev,
                               const WfHook *hook);
extern template cudaError_t launch_wavefront_v<0>(const Params &, int, int, unsigned long long, const Queue &, float4 *, cloak_record *, int, cudaStream_t, cudaEvent_t *, const WfHook *);
extern template cudaError_t launch_wavefront_v<1>(const Params &, int, int, unsigned long long, const Queue &, float4 *, cloak_record *, int, cudaStream_t, cudaEvent_t *, const WfHook *);
extern template cudaError_t launch_wavefront_v<2>(const Params &, int, int, unsigned long long, const Queue &, float4 *, cloak_record *, int, cudaStream_t, cudaEvent_t *, const WfHook *);
// ev (nullable): ev[1] after entry, ev[2] after integration, ev[3] after exit (ev[0] is recorded by the caller)
// hook (nullable): run after the entry kernel, before the sort
inline cudaError_t launch_wavefront(const Params &p, int mode, int spp, unsigned long long seed, const Queue &q,
                                    float4 *samples, cloak_record *recs, int packet, cudaStream_t st,
                                    cudaEvent_t *ev, const WfHook *hook = nullptr) {
    if (p.variant == V_RADIAL) return launch_wavefront_v<0>(p, mode, spp, seed, q, samples, recs, packet, st, ev, hook);
    if (p.variant == V_AZIMUTHAL)
        return launch_wavefront_v<1>(p, mode, spp, seed, q, samples, recs, packet, st, ev, hook);
    return launch_wavefront_v<2>(p, mode, spp, seed, q, samples, recs, packet, st, ev, hook);
}
cudaError_t launch_resolve(int npix, int spp, const float4 *samples, float4 *out, cudaStream_t st);
cudaError_t launch_eval_rhs(const Params &p, int mode, const double *y, long long n, double *dy, cudaStream_t st);
// FMA throughput microbenchmark (alu_peak.cu): fp64 != 0 selects FP64 chains, else FP32
cudaError_t launch_fma_peak(int fp64, int blocks, int threads, long long iters, void *sink, double *flops,
                            cudaStream_t st);

}  // namespace ck
