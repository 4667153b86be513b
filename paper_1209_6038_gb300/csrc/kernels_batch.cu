// kernels_batch.cu -- batched rendering: many views (poses x media x polarizations x resolutions)
// through one camera/entry kernel, one cost-ordered device queue, ONE persistent integration kernel
// with the medium selected per ray at run time, one exit kernel and one resolve kernel.
#include "batch.h"
#include "sur_physics.cuh"
#include "surrogate.h"
#include "wavefront.cuh"

namespace ck {

__global__ void __launch_bounds__(128) k_batch_entry(Params p, const ViewDev *views, int nviews, int spp,
                                                     unsigned long long seed, long long total, Queue q,
                                                     float4 *samples) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const ViewDev &vw = views[find_view(views, nviews, g, false)];
    long long local = g - vw.ray_begin, pix = local / spp;
    int s = (int)(local - pix * spp);
    int i = (int)(pix % vw.W), j = (int)(pix / vw.W);
    double o[3], d[3], y[6], k0[3], n_in[3], mat[5];
    view_camera_ray(vw, i, j, s, spp, seed, o, d);
    Params pv = p;
    pv.variant = vw.vm >> 1;
    const int mode = vw.vm & 1;
    cloak_record rec;
    float rgb[3];
    bool inside = mode ? enter<M_EXT>(pv, o, d, rec, rgb, y, k0, n_in, mat)
                       : enter<M_ORD>(pv, o, d, rec, rgb, y, k0, n_in, mat);
    if (!inside) {
        if (p.tof) store_tof_sample(pv, samples, g, o, d, rec);
        else store_sample(samples, nullptr, g, rec, rgb);
        return;
    }
    double mk0[3] = {-k0[0], -k0[1], -k0[2]}, c[3] = {mat[2], mat[3], mat[4]};
    // the camera's polariser along this view's own right or up vector
    const double *axis = p.analyzer == 1 ? vw.rt : p.analyzer == 2 ? vw.up : nullptr;
    double w_out = entry_factor(p, mode, mat[0], mat[1], c, n_in, mk0, axis);
    // queue key: medium/mode (major: one segment of the sorted queue per medium) and cost bucket (minor,
    // slowest first within a segment after the descending sort)
    double dy[6];
    const bool first = p.precision == 0 && p.formulation == 0;  // the FP64 Fermat stepper's first stage
    if (first) rhs<V_ANY, V_ANY>(pv, y, dy, vw.vm);
    queue_append(q, y, w_out, (int)g, batch_key(vw.vm, cost_bucket(p, y, k0)), first ? dy + 3 : nullptr,
                 p.precision != 0);
}

__global__ void __launch_bounds__(128) k_batch_exit(Params p, const ViewDev *views, int nviews, int spp,
                                                    unsigned long long seed, Queue q, float4 *samples) {
    const unsigned int n = q.count[0];
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if (q.key[k] < 0) continue;  // finished before the integration (learned surrogate)
        long long g = q.id[k];
        const ViewDev &vw = views[find_view(views, nviews, g, false)];
        long long local = g - vw.ray_begin, pix = local / spp;
        int s = (int)(local - pix * spp);
        double o[3], d[3];
        view_camera_ray(vw, (int)(pix % vw.W), (int)(pix / vw.W), s, spp, seed, o, d);
        Params pv = p;
        int vm = key_vm(q.key[k]);
        pv.variant = vm >> 1;
        cloak_record rec;
        float rgb[3];
        exit_slot(pv, vm & 1, q, k, d, rec, rgb);
        if (p.tof) store_tof_sample(pv, samples, g, o, d, rec);
        else store_sample(samples, nullptr, g, rec, rgb);
    }
}

// per pixel of every view: mean over its samples in sample order, into the view's own image
__global__ void k_batch_resolve(const ViewDev *views, int nviews, int spp, long long total_pix,
                                const float4 *samples) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total_pix) return;
    const ViewDev &vw = views[find_view(views, nviews, g, true)];
    long long pix = g - vw.pix_begin;
    const float4 *sp = samples + vw.ray_begin + pix * spp;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int k = 0; k < spp; ++k) {
        float4 v = sp[k];
        a0 += v.x; a1 += v.y; a2 += v.z; a3 += v.w;
    }
    float inv = 1.0f / spp;
    vw.out[pix] = make_float4(a0 * inv, a1 * inv, a2 * inv, a3 * inv);
}

// Unpolarised light (the paper's Fig. 1(c) / 2(c)): per pixel, the mean over its samples of the ordinary
// plus the extraordinary sample of views 0 and 1 (the same camera); a ray that never enters the shell
// (it misses the cylinder or mirrors off a metal end disc) is the same for both modes and counts once.
// With first-order reflections (refl non-null: per sample index g, refl[2 g + m'] is the light that
// reflected at the far face from mode m' into the sample's mode) a sample that enters also receives the
// room light the outer surface reflects into the camera, once.
__global__ void k_unpol_resolve(Params p, const ViewDev *views, int spp, unsigned long long seed, long long npix,
                                const float4 *samples, const float4 *refl, float4 *out) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npix) return;
    const ViewDev &v0 = views[0];
    const int i = (int)(g % v0.W), j = (int)(g / v0.W);
    const long long go = views[0].ray_begin + g * spp, ge = views[1].ray_begin + g * spp;
    const float4 *so = samples + go, *se = samples + ge;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int s = 0; s < spp; ++s) {
        double o[3], d[3], pt[3], n[3];
        view_camera_ray(v0, i, j, s, spp, seed, o, d);
        const int face = cylinder_entry(p, o, d, pt, n);
        const bool enters = face >= 0 && !(face != EV_LAT && p.R1 > 0.0 && hypot(pt[0], pt[1]) <= p.R1);
        float4 v = so[s];
        if (enters) {
            const float4 e = se[s];
            v.x += e.x; v.y += e.y; v.z += e.z; v.w += e.w;
            if (refl) {
                const float4 r[4] = {refl[2 * (go + s)], refl[2 * (go + s) + 1], refl[2 * (ge + s)], refl[2 * (ge + s) + 1]};
                for (int q = 0; q < 4; ++q) { v.x += r[q].x; v.y += r[q].y; v.z += r[q].z; v.w += r[q].w; }
                double eo, ee, c[3], dr[3];
                local_material(p, pt, eo, ee, c);
                const double dn = dot3(d, n);
                for (int q = 0; q < 3; ++q) dr[q] = d[q] - 2.0 * dn * n[q];
                const double axis[3] = {p.analyzer == 1 ? v0.rt[0] : v0.up[0], p.analyzer == 1 ? v0.rt[1] : v0.up[1],
                                        p.analyzer == 1 ? v0.rt[2] : v0.up[2]};
                const float w = (float)vacuum_reflection(eo, ee, c, n, d, p.analyzer ? axis : nullptr);
                float rgb[3];
                room_hit(p, pt, dr, rgb);
                v.x += w * rgb[0]; v.y += w * rgb[1]; v.z += w * rgb[2]; v.w += w;
            }
        }
        a0 += v.x; a1 += v.y; a2 += v.z; a3 += v.w;
    }
    const float inv = 1.0f / spp;
    out[g] = make_float4(a0 * inv, a1 * inv, a2 * inv, a3 * inv);
}

// Time-of-flight difference image (Sect. 4 after Ref. [10]) from the TOF samples (w dt, w) of views 0
// (ordinary) and 1 (extraordinary) of one camera, per pixel: (0) intensity-weighted mean TOF difference
// of both polarizations, a ray that never enters the shell counting once; (1) of the ordinary and (2) of
// the extraordinary light alone; (3) the summed weight, mean over samples.  0 where no light arrives.
__global__ void k_tof_resolve(Params p, const ViewDev *views, int spp, unsigned long long seed, long long npix,
                              const float4 *samples, float4 *out) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npix) return;
    const ViewDev &v0 = views[0];
    const int i = (int)(g % v0.W), j = (int)(g / v0.W);
    const float4 *so = samples + views[0].ray_begin + g * spp, *se = samples + views[1].ray_begin + g * spp;
    double A = 0, W = 0, Ao = 0, Wo = 0, Ae = 0, We = 0;
    for (int s = 0; s < spp; ++s) {
        double o[3], d[3], pt[3], n[3];
        view_camera_ray(v0, i, j, s, spp, seed, o, d);
        const int face = cylinder_entry(p, o, d, pt, n);
        const bool enters = face >= 0 && !(face != EV_LAT && p.R1 > 0.0 && hypot(pt[0], pt[1]) <= p.R1);
        const float4 a = so[s], b = se[s];
        Ao += a.x; Wo += a.y; Ae += b.x; We += b.y;
        A += a.x + (enters ? b.x : 0.f);
        W += a.y + (enters ? b.y : 0.f);
    }
    out[g] = make_float4(W > 0 ? (float)(A / W) : 0.f, Wo > 0 ? (float)(Ao / Wo) : 0.f, We > 0 ? (float)(Ae / We) : 0.f,
                         (float)(W / spp));
}

cudaError_t launch_tof_resolve(const Params &p, const ViewDev *views, int spp, unsigned long long seed, long long npix,
                               const float4 *samples, float4 *out, cudaStream_t st) {
    k_tof_resolve<<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(p, views, spp, seed, npix, samples, out);
    return cudaGetLastError();
}

cudaError_t launch_unpol_resolve(const Params &p, const ViewDev *views, int spp, unsigned long long seed, long long npix,
                                 const float4 *samples, const float4 *refl, float4 *out, cudaStream_t st) {
    k_unpol_resolve<<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(p, views, spp, seed, npix, samples, refl, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ first-order reflections
// Each main ray that reached a face (status EXITED or HIT_METAL_EXITED in the queue; total internal
// reflection is decided at exit) reflects there, run backwards, into the ordinary and extraordinary
// waves: they are appended to the second queue q2 with their camera-side weight (the main ray's
// camera-side Eq. 12 factor x the reflection coefficient) and the slot id 2 g + m'.
__global__ void __launch_bounds__(128) k_refl_spawn(Params p, Queue q, Queue q2) {
    const unsigned int n = q.count[0];
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int key = q.key[k], status = q.status[k];
        if (key < 0 || (status != CLOAK_RAY_EXITED && status != CLOAK_RAY_HIT_METAL_EXITED)) continue;
        const int vm = key_vm(key), mode = vm & 1;
        Params pv = p;
        pv.variant = vm >> 1;
        double ys[6];
        get_state(p.precision != 0, q, k, ys);
        const double x[3] = {ys[0], ys[1], ys[2]}, w[3] = {ys[3], ys[4], ys[5]};
        double nrm[3], eo, ee, c[3], kk[3];
        face_normal(q.face[k], x, nrm);
        local_material(pv, x, eo, ee, c);
        if (p.formulation) set_vec(kk, w);
        else wave_from_velocity(mode, eo, ee, c, w, kk);
        double R[2];
        if (!internal_reflection(mode, eo, ee, c, nrm, kk, R)) continue;
        const double kn = dot3(kk, nrm);
        double kt[3];
        for (int i = 0; i < 3; ++i) kt[i] = kk[i] - kn * nrm[i];
        for (int m2 = 0; m2 < 2; ++m2) {
            double k2[3], v2[3];
            if (!(R[m2] > 0.0) || !refract_in(m2, eo, ee, c, nrm, kt, k2, v2)) continue;
            const double y[6] = {x[0], x[1], x[2], p.formulation ? k2[0] : v2[0], p.formulation ? k2[1] : v2[1],
                                 p.formulation ? k2[2] : v2[2]};
            queue_append(q2, y, q.w_out[k] * R[m2], 2 * q.id[k] + m2,
                         batch_key(2 * pv.variant + m2, cost_bucket(p, y, k2)), nullptr, p.precision != 0);
        }
    }
}

// Exit of the reflected rays: refraction into the room at their own exit (no further reflection), the
// Eq. 12 factor of room light entering there, the room colour: refl[id] = (w rgb, w).
__global__ void __launch_bounds__(128) k_refl_exit(Params p, Queue q2, float4 *refl) {
    const unsigned int n = q2.count[0];
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int vm = key_vm(q2.key[k]);
        Params pv = p;
        pv.variant = vm >> 1;
        const double dz[3] = {0.0, 0.0, 1.0};
        cloak_record rec;
        float rgb[3];
        exit_slot(pv, vm & 1, q2, k, dz, rec, rgb);
        const float w = (float)rec.weight;
        refl[q2.id[k]] = make_float4(w * rgb[0], w * rgb[1], w * rgb[2], w);
    }
}

template <int I, int PREC>
static cudaError_t refl_ip(const Params &p, const Queue &q, const Queue &q2, float4 *refl, long long nrefl, int packet,
                           cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMemsetAsync(q2.count, 0, QUEUE_HEADER_BYTES, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(refl, 0, (size_t)nrefl * sizeof(float4), st);
    if (e != cudaSuccess) return e;
    k_refl_spawn<<<sms * 16, 128, 0, st>>>(p, q, q2);
    k_wf_sort_scan<<<1, 32, 0, st>>>(q2, NBINS_BATCH, 0u);
    k_wf_sort_scatter<<<sms * 8, 256, 0, st>>>(q2);
    const int pk = packet > 0 ? packet : 128;
    int nb = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wf_integrate_kernel<V_ANY, V_ANY, I, PREC>(), pk, 0)) !=
        cudaSuccess)
        return e;
    wf_integrate_kernel<V_ANY, V_ANY, I, PREC>()<<<(nb > 0 ? nb : 1) * sms, pk, 0, st>>>(p, q2);
    k_refl_exit<<<sms * 16, 128, 0, st>>>(p, q2, refl);
    return cudaGetLastError();
}

cudaError_t launch_reflections(const Params &p, const Queue &q, const Queue &q2, float4 *refl, long long nrefl,
                               int packet, cudaStream_t st) {
    if (p.integ == I_RK4)
        return p.precision ? refl_ip<I_RK4, 1>(p, q, q2, refl, nrefl, packet, st)
                           : refl_ip<I_RK4, 0>(p, q, q2, refl, nrefl, packet, st);
    return p.precision ? refl_ip<I_DP45, 1>(p, q, q2, refl, nrefl, packet, st)
                       : refl_ip<I_DP45, 0>(p, q, q2, refl, nrefl, packet, st);
}

static inline void mark(cudaEvent_t *ev, int i, cudaStream_t st) {
    if (ev) cudaEventRecordWithFlags(ev[i], st, cudaEventRecordExternal);
}

template <int I, int PREC>
static cudaError_t batch_ip(const Params &p, const ViewDev *views, int nviews, int spp, unsigned long long seed,
                            long long total, long long total_pix, const Queue &q, float4 *samples, int packet,
                            cudaStream_t st, cudaEvent_t *ev, const WfHook *hook) {
    const int bs = 128;
    mark(ev, 0, st);
    cudaError_t e = cudaMemsetAsync(q.count, 0, QUEUE_HEADER_BYTES, st);
    if (e != cudaSuccess) return e;
    k_batch_entry<<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>(p, views, nviews, spp, seed, total, q, samples);
    if (hook && (e = hook->fn(hook->ctx, q, st)) != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int pk = packet > 0 ? packet : 128;
    // the slowest rays of the batch go to the warps of LONG_RAY_BLOCKS blocks that have their SMs to
    // themselves (k_wf_integrate)
    k_wf_sort_scan<<<1, 32, 0, st>>>(q, NBINS_BATCH, (unsigned int)(p.long_ray_blocks * pk * p.reserve_per_thread));
    k_wf_sort_scatter<<<sms * 8, 256, 0, st>>>(q);
    mark(ev, 1, st);
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wf_integrate_kernel<V_ANY, V_ANY, I, PREC>(), pk, 0);
    if (e != cudaSuccess) return e;
    Params pl = p;
    pl.dedicated_blocks = p.long_ray_blocks;
    wf_integrate_kernel<V_ANY, V_ANY, I, PREC>()<<<(nb > 0 ? nb : 1) * sms, pk, 0, st>>>(pl, q);
    mark(ev, 2, st);
    k_batch_exit<<<sms * 16, 128, 0, st>>>(p, views, nviews, spp, seed, q, samples);
    mark(ev, 3, st);
    k_batch_resolve<<<(unsigned)((total_pix + 255) / 256), 256, 0, st>>>(views, nviews, spp, total_pix, samples);
    mark(ev, 4, st);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ surrogate training rays
// Ray i of the seeded training set, started half a unit outside its entry point so that the
// entry search finds that point; its network inputs go to X_all, its targets (after the exit
// kernel) to T_all.
__global__ void __launch_bounds__(128) k_sur_gen_entry(Params p, long long n, unsigned long long seed, Queue q,
                                                       float *X_all, float *T_all) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double P[3], d[3];
    int mode, variant;
    sur_sample(seed, (unsigned long long)i, p.R2, p.H, P, d, mode, variant);
    float x[SUR_IN];
    sur_features(p.R1, p.R2, p.H, variant, mode, P, d, x);
    float *X = X_all + i * SUR_XSTRIDE, *T = T_all + i * SUR_TSTRIDE;
#pragma unroll
    for (int j = 0; j < SUR_IN; ++j) X[j] = x[j];
    X[SUR_IN] = 0.f;
#pragma unroll
    for (int j = 0; j < SUR_TSTRIDE; ++j) T[j] = 0.f;
    double o[3] = {P[0] - 0.5 * d[0], P[1] - 0.5 * d[1], P[2] - 0.5 * d[2]}, y[6], k0[3], n_in[3], mat[5];
    Params pv = p;
    pv.variant = variant ? V_AZIMUTHAL : V_RADIAL;
    cloak_record rec;
    float rgb[3];
    const bool inside = mode ? enter<M_EXT>(pv, o, d, rec, rgb, y, k0, n_in, mat)
                             : enter<M_ORD>(pv, o, d, rec, rgb, y, k0, n_in, mat);
    if (!inside) return;
    queue_append(q, y, 1.0, (int)i, batch_key(2 * variant + mode, cost_bucket(p, y, k0)), nullptr, p.precision != 0);
}

__global__ void __launch_bounds__(128) k_sur_gen_exit(Params p, unsigned long long seed, Queue q, float *T_all) {
    const unsigned int n = q.count[0];
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const long long i = q.id[k];
        double P[3], d[3];
        int mode, variant;
        sur_sample(seed, (unsigned long long)i, p.R2, p.H, P, d, mode, variant);
        Params pv = p;
        pv.variant = variant ? V_AZIMUTHAL : V_RADIAL;
        cloak_record rec;
        float rgb[3], t[4];
        exit_slot(pv, mode, q, k, d, rec, rgb);
        float *T = T_all + i * SUR_TSTRIDE;
        const bool lateral = sur_targets(p.R2, p.H, P, d, rec, t);
#pragma unroll
        for (int j = 0; j < 4; ++j) T[j] = lateral ? t[j] : 0.f;
        T[4] = 0.f;
        T[5] = lateral ? 1.f : 0.f;
        T[6] = (float)rec.status;
        T[7] = (float)rec.steps;
    }
}

template <int I, int PREC>
static cudaError_t sur_data_ip(const Params &p, long long n, unsigned long long seed, const Queue &q, float *X_all,
                               float *T_all, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(q.count, 0, QUEUE_HEADER_BYTES, st);
    if (e != cudaSuccess) return e;
    k_sur_gen_entry<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(p, n, seed, q, X_all, T_all);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_wf_sort_scan<<<1, 32, 0, st>>>(q, NBINS_BATCH, 0u);
    k_wf_sort_scatter<<<sms * 8, 256, 0, st>>>(q);
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wf_integrate_kernel<V_ANY, V_ANY, I, PREC>(), 128, 0);
    if (e != cudaSuccess) return e;
    wf_integrate_kernel<V_ANY, V_ANY, I, PREC>()<<<(nb > 0 ? nb : 1) * sms, 128, 0, st>>>(p, q);
    k_sur_gen_exit<<<sms * 16, 128, 0, st>>>(p, seed, q, T_all);
    return cudaGetLastError();
}

cudaError_t launch_sur_data(const Params &p, long long n, unsigned long long seed, const Queue &q, float *X_all,
                            float *T_all, cudaStream_t st) {
    if (p.integ == I_RK4)
        return p.precision ? sur_data_ip<I_RK4, 1>(p, n, seed, q, X_all, T_all, st)
                           : sur_data_ip<I_RK4, 0>(p, n, seed, q, X_all, T_all, st);
    return p.precision ? sur_data_ip<I_DP45, 1>(p, n, seed, q, X_all, T_all, st)
                       : sur_data_ip<I_DP45, 0>(p, n, seed, q, X_all, T_all, st);
}

cudaError_t launch_batch(const Params &p, const ViewDev *views, int nviews, int spp, unsigned long long seed,
                         long long total, long long total_pix, const Queue &q, float4 *samples, int packet,
                         cudaStream_t st, cudaEvent_t *ev, const WfHook *hook) {
    if (p.integ == I_RK4)
        return p.precision
                   ? batch_ip<I_RK4, 1>(p, views, nviews, spp, seed, total, total_pix, q, samples, packet, st, ev, hook)
                   : batch_ip<I_RK4, 0>(p, views, nviews, spp, seed, total, total_pix, q, samples, packet, st, ev, hook);
    return p.precision
               ? batch_ip<I_DP45, 1>(p, views, nviews, spp, seed, total, total_pix, q, samples, packet, st, ev, hook)
               : batch_ip<I_DP45, 0>(p, views, nviews, spp, seed, total, total_pix, q, samples, packet, st, ev, hook);
}

}  // namespace ck
