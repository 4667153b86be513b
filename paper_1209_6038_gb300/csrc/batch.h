// batch.h -- device view table of a batched render (internal).
#pragma once

#include <cuda_runtime.h>

#include "physics.cuh"

namespace ck {

struct Queue;

struct ViewDev {
    double eye[3], fw[3], rt[3], up[3], tx, ty;  // pinhole camera frame
    long long ray_begin;                         // first global sample index of the view
    long long pix_begin;                         // first global pixel index of the view
    float4 *out;                                 // the view's image
    int W, Hp, vm;                               // size; vm = 2 * variant + polarization
    int pad;
};
// one entry per view is copied host to device at every batched render (bench.py counts these bytes)
static_assert(sizeof(ViewDev) == 152, "view table entry size changed: update bench.py's VIEW_TABLE_BYTES");

// view of global sample (by_pixel false) or pixel (by_pixel true) g: binary search on the prefix sums
__device__ __forceinline__ int find_view(const ViewDev *v, int n, long long g, bool by_pixel) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        long long b = by_pixel ? v[mid].pix_begin : v[mid].ray_begin;
        if (b <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// camera ray of sample s of pixel (i, j) of a view (the pinhole camera of camera_ray with the view's frame)
__device__ __forceinline__ void view_camera_ray(const ViewDev &v, int i, int j, int s, int spp, uint64_t seed,
                                                double o[3], double d[3]) {
    double xi1 = 0.5, xi2 = 0.5;
    if (spp > 1) {
        uint64_t pix = uint64_t(j) * uint64_t(v.W) + uint64_t(i);
        xi1 = jitter(seed, pix, s, 0);
        xi2 = jitter(seed, pix, s, 1);
    }
    double px = (2.0 * (i + xi1) / v.W - 1.0) * v.tx;
    double py = (1.0 - 2.0 * (j + xi2) / v.Hp) * v.ty;
    double l2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        d[k] = v.fw[k] + px * v.rt[k] + py * v.up[k];
        l2 += d[k] * d[k];
    }
    double il = 1.0 / sqrt(l2);
    for (int k = 0; k < 3; ++k) { d[k] *= il; o[k] = v.eye[k]; }
}

// camera ray of the queued sample with global index g
__device__ __forceinline__ void batch_camera_ray(const ViewDev *views, int nviews, int spp, uint64_t seed, long long g,
                                                 double o[3], double d[3]) {
    const ViewDev &vw = views[find_view(views, nviews, g, false)];
    const long long local = g - vw.ray_begin, pix = local / spp;
    view_camera_ray(vw, (int)(pix % vw.W), (int)(pix / vw.W), (int)(local - pix * spp), spp, seed, o, d);
}

struct WfHook;

// queue scratch and per-sample buffer as for the wavefront schedule; views: device copy of the table
// ev (nullable, used while capturing): ev[0] before, ev[1] after entry + sort, ev[2] after integration,
// ev[3] after exit, ev[4] after resolve -- recorded as external event nodes of the graph
// hook (nullable): called after the entry kernel, before the sort (the learned surrogate)
cudaError_t launch_batch(const Params &p, const ViewDev *views, int nviews, int spp, unsigned long long seed,
                         long long total, long long total_pix, const Queue &q, float4 *samples, int packet,
                         cudaStream_t st, cudaEvent_t *ev, const WfHook *hook = nullptr);

// unpolarised image of views 0 (ordinary) and 1 (extraordinary) of the last batch: samples as carved
// for that batch, views: its device table
cudaError_t launch_tof_resolve(const Params &p, const ViewDev *views, int spp, unsigned long long seed, long long npix,
                               const float4 *samples, float4 *out, cudaStream_t st);
cudaError_t launch_unpol_resolve(const Params &p, const ViewDev *views, int spp, unsigned long long seed, long long npix,
                                 const float4 *samples, const float4 *refl, float4 *out, cudaStream_t st);
// first-order reflections of the main rays of the last batch (queue q): reflected rays through queue q2
// (capacity >= 2 x q's), refl[2 g + m'] (nrefl = 2 x samples of the batch) written on st
cudaError_t launch_reflections(const Params &p, const Queue &q, const Queue &q2, float4 *refl, long long nrefl,
                               int packet, cudaStream_t st);
// reference panels without the cloak: 0 the room alone, 1 the bare metal cylinder (radius R1, height H)
cudaError_t launch_panel(const Params &p, int panel, int spp, unsigned long long seed, float4 *out, cudaStream_t st);

}  // namespace ck
