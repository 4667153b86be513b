// kernels_panels.cu -- the reference panels of the paper's figures (Fig. 1(a), (b)): the room seen without
// the cylinder, and with the bare metal cylinder of radius R1 and height H (a mirror, reflectance 1).
#include "batch.h"
#include "physics.cuh"

namespace ck {

__global__ void __launch_bounds__(128) k_panel(Params p, int panel, int spp, unsigned long long seed, float4 *out) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)p.W * p.Hp) return;
    const int i = (int)(g % p.W), j = (int)(g / p.W);
    // the metal cylinder alone: the cloak's outer surface moved onto the metal (no shell, no end discs
    // beyond it)
    Params pm = p;
    pm.R2 = p.R1;
    pm.R2sq = p.R1sq;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    for (int s = 0; s < spp; ++s) {
        double o[3], d[3], pt[3], n[3];
        float rgb[3] = {0.f, 0.f, 0.f};
        camera_ray(p, i, j, s, spp, seed, o, d);
        if (panel == 1 && cylinder_entry(pm, o, d, pt, n) >= 0) {
            const double dn = dot3(d, n);
            double dr[3];
            for (int k = 0; k < 3; ++k) dr[k] = d[k] - 2.0 * dn * n[k];
            room_hit(p, pt, dr, rgb);
        } else {
            room_hit(p, o, d, rgb);
        }
        a0 += rgb[0]; a1 += rgb[1]; a2 += rgb[2];
    }
    const float inv = 1.0f / spp;
    out[g] = make_float4(a0 * inv, a1 * inv, a2 * inv, 1.0f);
}

cudaError_t launch_panel(const Params &p, int panel, int spp, unsigned long long seed, float4 *out, cudaStream_t st) {
    const long long n = (long long)p.W * p.Hp;
    k_panel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(p, panel, spp, seed, out);
    return cudaGetLastError();
}

}  // namespace ck
