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

// queue scratch and per-sample buffer as for the wavefront schedule; views: device copy of the table
// ev (nullable, used while capturing): ev[0] before, ev[1] after entry + sort, ev[2] after integration,
// ev[3] after exit, ev[4] after resolve -- recorded as external event nodes of the graph
cudaError_t launch_batch(const Params &p, const ViewDev *views, int nviews, int spp, unsigned long long seed,
                         long long total, long long total_pix, const Queue &q, float4 *samples, int packet,
                         cudaStream_t st, cudaEvent_t *ev);

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
