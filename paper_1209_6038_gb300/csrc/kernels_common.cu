// Kernels shared by all variants.
#include "wavefront.cuh"

namespace ck {

// mean over the samples of each pixel, in sample order (the plain path accumulates the same way)
__global__ void k_wf_resolve(int npix, int spp, const float4 *samples, float4 *out) {
    int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= npix) return;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    const float4 *s = samples + (long long)pix * spp;
    for (int k = 0; k < spp; ++k) {
        float4 v = s[k];
        a0 += v.x; a1 += v.y; a2 += v.z; a3 += v.w;
    }
    float inv = 1.0f / spp;
    out[pix] = make_float4(a0 * inv, a1 * inv, a2 * inv, a3 * inv);
}

// reserve > 0: set aside the first min(reserve, segment size) rays of the medium segment whose highest
// nonempty cost bucket is highest (its slowest rays are the slowest of the batch) for the long-ray
// blocks of the integration kernel: count[8] = that segment, count[9] = the number reserved.
__global__ void k_wf_sort_scan(Queue q, int nbins, unsigned int reserve) {
    if (threadIdx.x != 0) return;
    unsigned int off = 0;
    for (int v = 3; v >= 0; --v) {  // empty segments for the media a single image does not use
        q.bins[SEG_OFFSET + 2 * v] = 0;
        q.bins[SEG_OFFSET + 2 * v + 1] = 0;
    }
    int top_v = -1, top_cost = -1;
    for (int b = nbins - 1; b >= 0; --b) {  // descending key: slowest rays first
        unsigned int c = q.bins[b];
        q.bins[NBINS_BATCH + b] = off;
        if (b % NBINS == NBINS - 1) q.bins[SEG_OFFSET + 2 * key_vm(b)] = off;
        q.bins[SEG_OFFSET + 2 * key_vm(b) + 1] += c;
        off += c;
        if (c && b % NBINS > top_cost) {
            top_cost = b % NBINS;
            top_v = key_vm(b);
        }
    }
    q.count[2] = off;
    if (reserve && top_v >= 0) {
        const unsigned int len = q.bins[SEG_OFFSET + 2 * top_v + 1];
        q.count[8] = (unsigned int)top_v;
        q.count[9] = len < reserve ? len : reserve;
    }
}

__global__ void k_wf_sort_scatter(Queue q) {
    const unsigned int n = q.count[0];
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int key = q.key[k];
        if (key < 0) continue;  // finished before the integration (learned surrogate)
        unsigned int pos = atomicAdd(q.bins + NBINS_BATCH + key, 1u);
        q.perm[pos] = (int)k;
    }
}

// right-hand side of the ray equations (the handle's formulation) at n states; vm = 2 * variant + mode
__global__ void k_eval_rhs(Params p, int vm, const double *y, long long n, double *dy) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s[6], d[6];
    for (int a = 0; a < 6; ++a) s[a] = y[6 * i + a];
    rhs<V_ANY, V_ANY>(p, s, d, vm);
    for (int a = 0; a < 6; ++a) dy[6 * i + a] = d[a];
}

cudaError_t launch_eval_rhs(const Params &p, int mode, const double *y, long long n, double *dy, cudaStream_t st) {
    k_eval_rhs<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(p, 2 * p.variant + mode, y, n, dy);
    return cudaGetLastError();
}

cudaError_t launch_resolve(int npix, int spp, const float4 *samples, float4 *out, cudaStream_t st) {
    k_wf_resolve<<<(npix + 255) / 256, 256, 0, st>>>(npix, spp, samples, out);
    return cudaGetLastError();
}

}  // namespace ck
