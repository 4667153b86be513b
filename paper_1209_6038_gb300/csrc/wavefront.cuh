// wavefront.cuh -- the optimised FP64 schedule.
//
//   A  k_wf_entry      one thread per (pixel, sample): camera ray, cylinder entry, Sect. 3 entry
//                      refraction and the Eq. 12 factor of the entry face; rays that miss or hit a
//                      metal disc are shaded at once, rays that enter are appended to a compacted
//                      device queue (SoA, FP64 state).
//   B  k_wf_integrate  persistent kernel, one resident grid: every lane owns one queued ray and
//                      refills itself from the queue when its ray leaves.  Each loop iteration runs
//                      ONE uniform step evaluation (DP5(4): six right-hand sides; RK4: four) for every
//                      lane; the surface-crossing search is a lane state that reuses that same step
//                      slot with a trial step size, so root finding never serialises a warp.
//                      FP64 or mixed arithmetic (integrator.cuh).
//   C  k_wf_exit       one thread per queued ray: exit refraction, Eq. 12 factor of the exit face,
//                      room lookup.
//   D  k_wf_resolve    per pixel: mean over its samples in sample order.
//
// The arithmetic of every ray is that of the plain path (trace.cuh) step for step.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "integrator.cuh"
#include "internal.h"
#include "trace.cuh"

namespace ck {

// queue slot layout (structure of arrays; capacity = rays per image)
struct Queue {
    double *x, *y, *z, *vx, *vy, *vz;  // state on entry; final state after B
    double *ax, *ay, *az;              // dv/dt at the entry state (Fermat form, FP64), NaN where not computed
    double *w_out;                     // Eq. 12 factor of the entry face (physical exit towards the camera)
    double *t;                         // time of flight after B
    int *id;                           // sample index (pixel * spp + sample)
    int *status;                       // CLOAK_RAY_* after B (EXITED / HIT_METAL_EXITED means: crossed a face)
    int *steps;
    int *face;                         // surface crossed at exit (EV_LAT / EV_TOP / EV_BOT)
    int *key;                          // cost bucket of the ray (larger = more steps expected)
    int *perm;                         // integration order: slots sorted by descending cost bucket
    unsigned int *count;               // [0] queued rays, [1] next ray of the integration kernel,
                                       // [2] rays to integrate, [4 + v] next ray of medium segment v
    unsigned int *bins;                // [nbins] bucket sizes, [nbins] scatter cursors (nbins <= 256), then
                                       // per medium segment v: [SEG_OFFSET + 2v] first index into perm, [+1] size
    long long cap;
};

constexpr int NBINS = 64;         // cost buckets of a single image
constexpr int NBINS_BATCH = 256;  // medium/mode x cost bucket of a batch: key = vm * NBINS + cost
constexpr int SEG_OFFSET = 2 * NBINS_BATCH;
__host__ __device__ constexpr int batch_key(int vm, int cost) { return vm * NBINS + cost; }
__host__ __device__ constexpr int key_vm(int key) { return key / NBINS; }
constexpr size_t QUEUE_HEADER_BYTES = 4096;
// count[8]: medium segment of the reserved long rays, count[9]: their number, count[10]: their cursor;
// from count[DEDICATED_FLAGS]: one flag per SM id (mod 256) that hosts a long-ray block
constexpr int DEDICATED_FLAGS = 576;
constexpr int LONG_RAY_BLOCKS = 4;  // default number of blocks (SMs) for the long rays
static_assert((DEDICATED_FLAGS + 256) * 4 <= (int)QUEUE_HEADER_BYTES, "queue header too small");
static_assert(DEDICATED_FLAGS * 4 >= 64 + 4 * (SEG_OFFSET + 8), "long-ray flags overlap the bins");
// every array of the queue starts on a 256-byte boundary (the float4 per-sample buffer needs 16 bytes)
constexpr size_t queue_array_bytes(long long cap, size_t elem) { return ((size_t)cap * elem + 255) & ~(size_t)255; }
constexpr size_t queue_bytes(long long cap) {
    return QUEUE_HEADER_BYTES + 11 * queue_array_bytes(cap, sizeof(double)) + queue_array_bytes(cap, sizeof(float4)) +
           6 * queue_array_bytes(cap, sizeof(int));
}

// Lay the queue, its sort arrays and the per-sample buffer out in `base` (queue_bytes(cap) bytes,
// 256-byte aligned).  The header (counters and bins) must be zeroed before each render.
inline void carve_queue(char *base, long long cap, Queue &q, float4 **samples) {
    q.count = (unsigned int *)base;
    q.bins = (unsigned int *)(base + 64);
    char *b = base + QUEUE_HEADER_BYTES;
    double **dp[11] = {&q.x, &q.y, &q.z, &q.vx, &q.vy, &q.vz, &q.ax, &q.ay, &q.az, &q.w_out, &q.t};
    for (int i = 0; i < 11; ++i) { *dp[i] = (double *)b; b += queue_array_bytes(cap, sizeof(double)); }
    *samples = (float4 *)b;
    b += queue_array_bytes(cap, sizeof(float4));
    int **ip[6] = {&q.id, &q.status, &q.steps, &q.face, &q.key, &q.perm};
    for (int i = 0; i < 6; ++i) { *ip[i] = (int *)b; b += queue_array_bytes(cap, sizeof(int)); }
    q.cap = cap;
}

// Cost bucket of an entering ray from its axial angular momentum L = (x cross k)_z: rays that pass
// close to the inner radius (small |L|) are the slow ones (the ray speed grows like 1/L there).
__device__ __forceinline__ int cost_bucket(const Params &p, const double x[3], const double k[3]) {
    float L = fabsf((float)(x[0] * k[1] - x[1] * k[0]));
    int b = (int)(-p.cost_scale * __log2f(L + 1e-30f));
    return min(max(b, 0), NBINS - 1);
}

__device__ __forceinline__ void store_sample(float4 *samples, cloak_record *recs, long long id,
                                             const cloak_record &rec, const float rgb[3]) {
    if (samples) {
        float w = (float)rec.weight;
        samples[id] = make_float4(w * rgb[0], w * rgb[1], w * rgb[2], w);
    }
    if (recs) recs[id] = rec;
}

// Per-sample output of a TOF difference render (Params::tof): (w dt, w, 0, 0).
__device__ __forceinline__ void store_tof_sample(const Params &p, float4 *samples, long long id, const double o[3],
                                                 const double d[3], const cloak_record &rec) {
    const double w = rec.weight;
    samples[id] = make_float4((float)(w * tof_difference(p, o, d, rec)), (float)w, 0.f, 0.f);
}

// State format of the queue.  FP64 renders keep (x, v) as doubles; the mixed-precision path keeps each
// component as a float-float pair (hi, lo) in the same 8-byte slot, so that its FP32 stepper loads and
// stores rays with no FP64 arithmetic (a lone refilling lane converting doubles held the SM's FP64 unit
// 16 cycles per instruction for its whole warp).
__device__ __forceinline__ void put_state(bool ff, const Queue &q, unsigned int k, const double y[6]) {
    double *a[6] = {q.x, q.y, q.z, q.vx, q.vy, q.vz};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        if (ff) {
            const float hi = (float)y[i];
            reinterpret_cast<float2 *>(a[i])[k] = make_float2(hi, (float)(y[i] - (double)hi));
        } else {
            a[i][k] = y[i];
        }
    }
}
__device__ __forceinline__ void get_state(bool ff, const Queue &q, unsigned int k, double y[6]) {
    const double *a[6] = {q.x, q.y, q.z, q.vx, q.vy, q.vz};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        if (ff) {
            const float2 v = reinterpret_cast<const float2 *>(a[i])[k];
            y[i] = (double)v.x + (double)v.y;
        } else {
            y[i] = a[i][k];
        }
    }
}

// Eq. 12 factors of the mixed-precision path: the field-continuity solve in FP32 where the vacuum wave meets
// the face at more than ~11.5 degrees from grazing (cos > 0.2), in FP64 otherwise (the 4x4 system loses its
// conditioning towards grazing).  The face geometry, the double refraction and the exit refraction stay
// in FP64 on every path.
constexpr double F32_EQ12_MIN_COS = 0.2;
// axis: the camera's polariser (nullable)
__device__ __forceinline__ double entry_factor(const Params &p, int mode, double eo, double ee, const double c[3],
                                               const double n[3], const double k[3], const double *axis) {
    if (p.precision != 0) {
        const double kn = dot3(k, n), kt2 = dot3(k, k) - kn * kn;  // the vacuum wave's normal part: 1 - kt2
        if (1.0 - kt2 > F32_EQ12_MIN_COS * F32_EQ12_MIN_COS) {
            const float cf[3] = {(float)c[0], (float)c[1], (float)c[2]}, nf[3] = {(float)n[0], (float)n[1], (float)n[2]},
                        kf[3] = {(float)k[0], (float)k[1], (float)k[2]};
            float af[3];
            if (axis) { af[0] = (float)axis[0]; af[1] = (float)axis[1]; af[2] = (float)axis[2]; }
            return (double)transmission_out(mode, (float)eo, (float)ee, cf, nf, kf, axis ? af : (const float *)nullptr);
        }
    }
    return transmission_out(mode, eo, ee, c, n, k, axis);
}
// cos_vac: |d . n| of the vacuum wave d at the exit face
__device__ __forceinline__ double exit_factor(const Params &p, int mode, double eo, double ee, const double c[3],
                                              const double n[3], const double d[3], double cos_vac) {
    if (p.precision != 0 && cos_vac > F32_EQ12_MIN_COS) {
        const float cf[3] = {(float)c[0], (float)c[1], (float)c[2]}, nf[3] = {(float)n[0], (float)n[1], (float)n[2]},
                    df[3] = {(float)d[0], (float)d[1], (float)d[2]};
        return (double)transmission_in(mode, (float)eo, (float)ee, cf, nf, df);
    }
    return transmission_in(mode, eo, ee, c, n, d);
}

// Append an entering ray to the queue; one atomic per warp for the slot and one per distinct key.
// a: dv/dt at y (the integrator's first stage, computed here where every lane of the warp has one), or
// null.  ff: store the state as float-float pairs (mixed precision).
__device__ __forceinline__ void queue_append(const Queue &q, const double y[6], double w_out, int id, int key,
                                             const double *a = nullptr, bool ff = false) {
    const unsigned int act = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    unsigned int base = 0;
    if (lane == leader) base = atomicAdd(q.count, (unsigned int)__popc(act));
    base = __shfl_sync(act, base, leader);
    unsigned int slot = base + __popc(act & ((1u << lane) - 1u));
    put_state(ff, q, slot, y);
    q.ax[slot] = a ? a[0] : __longlong_as_double(0x7ff8000000000000ll);
    q.ay[slot] = a ? a[1] : 0.0;
    q.az[slot] = a ? a[2] : 0.0;
    q.w_out[slot] = w_out;
    q.id[slot] = id;
    q.key[slot] = key;
    unsigned int same = __match_any_sync(act, key);
    if (lane == __ffs(same) - 1) atomicAdd(q.bins + key, (unsigned int)__popc(same));
}

template <int VAR, int MODE>
__global__ void __launch_bounds__(128) k_wf_entry(Params p, int spp, unsigned long long seed, Queue q,
                                                  float4 *samples, cloak_record *recs) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long n = (long long)p.W * p.Hp * spp;
    if (idx >= n) return;
    long long pix = idx / spp;
    int s = (int)(idx - pix * spp);
    int i = (int)(pix % p.W), j = (int)(pix / p.W);
    double o[3], d[3], y[6], k0[3], n_in[3], mat[5];
    camera_ray(p, i, j, s, spp, seed, o, d);
    cloak_record rec;
    float rgb[3];
    if (!enter<MODE>(p, o, d, rec, rgb, y, k0, n_in, mat)) {
        store_sample(samples, recs, idx, rec, rgb);
        return;
    }
    // Eq. 12 at the entry face along the physical direction: light leaves the cloak towards the camera
    double mk0[3] = {-k0[0], -k0[1], -k0[2]}, c[3] = {mat[2], mat[3], mat[4]};
    double w_out = entry_factor(p, MODE, mat[0], mat[1], c, n_in, mk0, analyzer_axis(p));
    double dy[6];
    const bool first = p.precision == 0 && p.formulation == 0;  // the FP64 Fermat stepper's first stage
    if (first) rhs<VAR, MODE>(p, y, dy);
    queue_append(q, y, w_out, (int)idx, cost_bucket(p, y, k0), first ? dy + 3 : nullptr, p.precision != 0);
}

// Longest-first order: a counting sort of the queue by descending key.  k_wf_sort_scan turns the bucket
// sizes into scatter cursors and medium segments, k_wf_sort_scatter writes the permutation.  With the
// batch key (medium major, cost minor) every medium occupies one contiguous segment of the permutation,
// in descending cost order.
__global__ void k_wf_sort_scan(Queue q, int nbins, unsigned int reserve);
__global__ void k_wf_sort_scatter(Queue q);

template <int VAR, int MODE, int INTEG, int PREC>
__device__ __forceinline__ void wf_integrate_body(const Params &p, const Queue &q) {
    typedef typename std::conditional<PREC == 0, Stepper64<VAR, MODE, INTEG>, StepperMixed<VAR, MODE, INTEG>>::type S;
    typedef typename S::real R;
    S st;
    st.vm = 0;
    const unsigned int n = q.count[2];  // rays left to integrate after the sort
    const int nev = p.R1 > 0.0 ? 4 : 3;
    const R tol = (R)p.h_or_tol, h0 = INTEG == I_RK4 ? (R)p.h_or_tol : (R)1e-3;
    const R conv = sizeof(R) == 8 ? (R)CROSS_REL_TOL : (R)2.4e-7;  // bracket resolution of the crossing search
    constexpr int prefix = bisect_prefix<INTEG>();
    // FP64 DP5(4): when the ray moves towards the surface at both ends of the crossing step (one crossing
    // inside it), the search takes safeguarded Newton steps on the step function itself, the slope from
    // the end point's derivative f(y1), starting from a Newton step off the coarse step's end
    constexpr bool NEWTON = INTEG == I_DP45 && PREC == 0;
    constexpr double NEWTON_LAST = 1e-6;
    // medium segments of the permutation (batch: one per medium/mode; a lane draws rays from its
    // warp's current segment, so that the lanes of a warp evaluate one medium's equations)
    // the first segment is chosen per SM, so that the warps resident on one SM run one medium's code
    // (a quarter of the kernel's instructions for the instruction caches)
    unsigned int smid = 0;
    if (VAR == V_ANY) asm("mov.u32 %0, %%smid;" : "=r"(smid));
    int seg = VAR == V_ANY ? 3 - (int)(smid & 3u) : 0;
    // Long-ray blocks: the sort reserved the first rl rays of the order (of medium segment rv in a
    // batch) -- those that pass closest to the inner radius, up to ~3e4 steps each -- for the warps of
    // the first p.dedicated_blocks blocks.  The other blocks resident on those SMs leave at once, so
    // these warps share their SM's FP64 unit with no others and advance their long rays at close to
    // one warp's latency; on a full SM they would get a twelfth of it and finish last, after the rest
    // of the queue.  (A block that misses the flag only costs speed: every ray is still integrated once.)
    const unsigned int rl = q.count[9];
    const unsigned int rv = rl ? q.count[8] : 0u;
    bool reserve = false;
    if (rl) {
        if (VAR != V_ANY) asm("mov.u32 %0, %%smid;" : "=r"(smid));
        volatile unsigned int *sm_taken = q.count + DEDICATED_FLAGS;
        if ((int)blockIdx.x < p.dedicated_blocks) {
            reserve = true;
            seg = (int)rv;
            if (threadIdx.x == 0) sm_taken[smid & 255u] = 1u;
        } else {
            __nanosleep(2000);
            unsigned int f = 0;
            if ((threadIdx.x & 31u) == 0) f = sm_taken[smid & 255u];
            if (__shfl_sync(0xffffffffu, f, 0)) return;  // the whole warp leaves
        }
    }
    // lane state
    R h = h0, t = 0;
    int steps = 0, phase = PH_IDLE, slot = -1;
    bool metal = false;
    // crossing state
    R hs = 0, fac = 1, lo = 0, hi = 0, glo = 0, ghi = 0, sbest = 0, g1[4];
    int ev = 0, evbest = -1, side = 0, it = 0;
    bool newton = false, fin = false;
    R snext = 0;
    unsigned int pending = 0;
    bool drained = false;  // the queue had no ray left for this lane

    // Every lane of a warp stays in the loop until the whole warp is drained, and the warp reconverges
    // before the one step evaluation of each iteration, which all its live lanes then run together
    // (stepping and crossing search alike).
    for (;;) {
        // ---- refill: a lane without a ray takes the next queued one
        if (phase == PH_IDLE && !drained) {
            if (VAR == V_ANY) {
                if (reserve) {  // a long-ray lane: the reserved rays first
                    const unsigned int k = atomicAdd(q.count + 10, 1u);
                    if (k < rl) {
                        slot = q.perm[__ldg(q.bins + SEG_OFFSET + 2 * rv) + k];
                        seg = (int)rv;
                        st.vm = seg;
                        phase = PH_STEP;
                    } else {
                        reserve = false;
                    }
                }
                // the current segment first, then the others in descending medium order (segment rv
                // without its reserved head)
                for (int tries = 0; tries < 4 && phase != PH_STEP; ++tries) {
                    const unsigned int skip = (unsigned int)seg == rv ? rl : 0u;
                    const unsigned int len = __ldg(q.bins + SEG_OFFSET + 2 * seg + 1) - skip;
                    const unsigned int k = len ? atomicAdd(q.count + 4 + seg, 1u) : 0xffffffffu;
                    if (k < len) {
                        slot = q.perm[__ldg(q.bins + SEG_OFFSET + 2 * seg) + skip + k];
                        st.vm = seg;
                        phase = PH_STEP;
                        break;
                    }
                    seg = (seg + 3) & 3;
                }
            } else {
                if (reserve) {  // a long-ray lane: the reserved head of the order first
                    const unsigned int k = atomicAdd(q.count + 10, 1u);
                    if (k < rl) {
                        slot = q.perm[k];
                        phase = PH_STEP;
                    } else {
                        reserve = false;
                    }
                }
                if (phase != PH_STEP) {
                    const unsigned int k = atomicAdd(q.count + 1, 1u) + rl;
                    if (k < n) {
                        slot = q.perm[k];
                        phase = PH_STEP;
                    }
                }
            }
            if (phase == PH_STEP) {
                st.load(q, slot);
                h = h0; t = 0; steps = 0; metal = false;
            }
        }
        const bool live = phase != PH_IDLE;
        if (!live) drained = true;
        const unsigned int lm = __ballot_sync(0xffffffffu, live);
        if (!lm) break;     // the whole warp is drained
        if (!live) continue;
        int status = -1;
        if (phase == PH_STEP && (steps >= p.max_steps || (INTEG == I_DP45 && h < (R)1e-14))) status = CLOAK_RAY_STEP_LIMIT;
        R s = phase == PH_STEP ? h : sbest;
        if (phase == PH_CROSS) {
            // next trial point: Newton (see above), or a bisection prefix, then Illinois regula falsi
            // (see crossing())
            if (newton) s = snext;
            else if (it < prefix) s = (R)0.5 * (lo + hi);
            else if (it - prefix < 60 && ghi > glo) s = (lo * ghi - hi * glo) * rcp_nr(ghi - glo);
            else s = (R)0.5 * (lo + hi);
            if (!(s > lo && s < hi)) s = (R)0.5 * (lo + hi);
        }
        __syncwarp(lm);  // a convergence point: keeps the compiler from splitting the evaluation by phase
        bool land = false;
        if (status < 0) {
            st.eval(p, s);
            if (phase == PH_STEP) {
                ++steps;
                fac = 1;
                bool accept = true;
                if (INTEG == I_DP45) {
                    if (!st.control(tol, fac)) {
                        h *= fmin(fac, (R)1);
                        fac = 1;
                        accept = false;
                    }
                }
                if (accept) {
                    pending = 0;
                    for (int e = 0; e < nev; ++e) {
                        g1[e] = st.g_end(p, e);
                        if (g1[e] > (R)0) pending |= 1u << e;
                    }
                    R sc = 0;
                    if (INTEG == I_DP45 && nev == 4 && !(pending & (1u << EV_METAL))) sc = st.chord(p);
                    if (sc > (R)0) {
                        h *= sc;  // retried: the step's chord passes through the metal cylinder
                    } else if (!pending) {
                        st.take_step();
                        t += h;
                        h *= fac;
                    } else {
                        hs = h;
                        sbest = (R)1e30;
                        evbest = -1;
                        ev = __ffs(pending) - 1;
                        lo = 0; hi = hs; glo = st.g_start(p, ev); ghi = g1[ev];
                        if (!(glo <= (R)0)) glo = 0;
                        side = 0; it = 0;
                        newton = false;
                        fin = false;
                        if constexpr (NEWTON) {
                            const R d0 = (R)st.g_rate_start(ev), d1 = (R)st.g_rate(ev);
                            if (d0 >= (R)0 && d1 > (R)0) {
                                newton = true;
                                R s0 = hs - ghi / d1;
                                if (!(s0 > (R)0 && s0 < hs)) s0 = hs * (-glo / (ghi - glo));
                                if (!(s0 > (R)0 && s0 < hs)) s0 = (R)0.5 * hs;
                                snext = s0;
                            }
                        }
                        phase = PH_CROSS;
                    }
                }
            } else if (phase == PH_CROSS) {
                bool done = false;
                if (!(s > lo && s < hi)) {
                    done = true;
                } else if (NEWTON && newton) {
                    // safeguarded Newton: keep the bracket, bisect when the step would leave it
                    const R gs = st.g_end(p, ev);
                    if (gs > (R)0) { hi = s; ghi = gs; } else { lo = s; glo = gs; }
                    ++it;
                    const R gtol = (R)CROSS_G_TOL * (R)cross_g_scale(p, ev);
                    if (fin || fabs(gs) <= gtol) {
                        // on the surface to rounding, or the trial point of a Newton correction below
                        // NEWTON_LAST x the step: quadratic convergence put it within ~1e-12 of the step
                        lo = s;
                        hi = s;
                        done = true;
                    } else {
                        R dg = (R)1;
                        if constexpr (NEWTON) dg = (R)st.g_rate(ev);
                        R sn = s - gs * rcp_nr(dg);
                        if (!(sn > lo && sn < hi)) sn = (R)0.5 * (lo + hi);
                        else if (fabs(sn - s) <= (R)NEWTON_LAST * hs) fin = true;
                        snext = sn;
                        if (hi - lo <= conv * hi || it >= 100) done = true;
                    }
                } else {
                    R gs = st.g_end(p, ev);
                    if (it < prefix) {
                        if (gs > (R)0) { hi = s; ghi = gs; } else { lo = s; glo = gs; }
                    } else if (gs > (R)0) {
                        hi = s; ghi = gs;
                        if (side == 1) glo *= (R)0.5;
                        side = 1;
                    } else {
                        lo = s; glo = gs;
                        if (side == -1) ghi *= (R)0.5;
                        side = -1;
                    }
                    ++it;
                    if (it >= prefix && hi - lo <= conv * hi) done = true;
                    // or a regula falsi trial point lies on the surface to rounding (Illinois approaches
                    // the root from one side, so the far end of the bracket may lag for many iterations)
                    const R gtol = (R)CROSS_G_TOL * (R)cross_g_scale(p, ev);
                    if (!done && it > prefix && fabs(gs) <= gtol) {
                        lo = s;
                        hi = s;
                        done = true;
                    }
                    if (it >= prefix + 200) done = true;
                }
                if (done) {
                    R se = ev == EV_METAL ? lo : hi;
                    if (se < sbest) { sbest = se; evbest = ev; }
                    pending &= ~(1u << ev);
                    if (pending) {
                        ev = __ffs(pending) - 1;
                        lo = 0; hi = hs; glo = st.g_start(p, ev); ghi = g1[ev];
                        if (!(glo <= (R)0)) glo = 0;
                        side = 0; it = 0;
                        newton = false;  // the coarse step's end point is gone: bisection for further surfaces
                    } else if (PREC == 0 && sbest == s && evbest == ev) {
                        land = true;  // the last trial step ended on the crossing: no re-evaluation
                    } else {
                        phase = PH_FINAL;
                    }
                }
            } else {
                land = true;  // PH_FINAL: the evaluation landed on the crossing
            }
            if (land) {
                st.take_crossing();
                t += sbest;
                h = hs * fac;
                phase = PH_STEP;
                if (evbest == EV_METAL) {
                    if ((VAR == V_RADIAL && MODE == M_ORD) || (VAR == V_ANY && st.vm == 0)) {
                        st.mirror();
                        metal = true;
                    } else {
                        status = CLOAK_RAY_SINGULAR;
                    }
                } else {
                    status = metal ? CLOAK_RAY_HIT_METAL_EXITED : CLOAK_RAY_EXITED;
                }
            }
        }
        if (status >= 0) {  // ray finished: write back (in the queue's state format), lane becomes idle
            st.store(q, slot);
            q.t[slot] = (double)t;
            q.status[slot] = status;
            q.steps[slot] = steps;
            q.face[slot] = evbest;
            phase = PH_IDLE;
        }
    }
}

// The FP64 integrator keeps the compiler's register choice (148-151 registers, three blocks of 128
// threads per SM); the mixed one is held to 128 registers for four blocks per SM -- its FP32 steps are
// latency-bound and gain from the extra warps, while the rare band steps near R1 may spill.
template <int VAR, int MODE, int INTEG, int PREC>
__global__ void __launch_bounds__(128) k_wf_integrate(Params p, Queue q) {
    wf_integrate_body<VAR, MODE, INTEG, PREC>(p, q);
}
template <int VAR, int MODE, int INTEG, int PREC>
__global__ void __launch_bounds__(128, 4) k_wf_integrate_mixed(const __grid_constant__ Params p, Queue q) {
    wf_integrate_body<VAR, MODE, INTEG, PREC>(p, q);
}
template <int VAR, int MODE, int INTEG, int PREC>
constexpr auto wf_integrate_kernel() {
    if constexpr (PREC == 0) return k_wf_integrate<VAR, MODE, INTEG, PREC>;
    else return k_wf_integrate_mixed<VAR, MODE, INTEG, PREC>;
}

// Exit of queue slot k: refraction into vacuum at the crossed face, the Eq. 12 factor of the exit face
// times the stored factor of the entry face, room lookup.  d_cam: the camera ray (kept as the
// direction of rays that do not leave).
__device__ __forceinline__ void exit_slot(const Params &p, int mode, const Queue &q, unsigned int k, const double d_cam[3],
                                          cloak_record &rec, float rgb[3]) {
    double y[6];
    get_state(p.precision != 0, q, k, y);
    int status = q.status[k];
    rec.mode = mode;
    rec.tile_id = -1;
    rec.weight = 0.0;
    rec.steps = q.steps[k];
    rec.tof = q.t[k];
    rgb[0] = rgb[1] = rgb[2] = 0.f;
    if (status == CLOAK_RAY_EXITED || status == CLOAK_RAY_HIT_METAL_EXITED) {
        double x[3] = {y[0], y[1], y[2]}, nrm[3], eo, ee, c[3], kk[3];
        face_normal(q.face[k], x, nrm);
        local_material(p, x, eo, ee, c);
        if (p.formulation) set_vec(kk, y + 3);  // the Hamiltonian state carries the wave vector
        else wave_from_velocity(mode, eo, ee, c, y + 3, kk);
        double kn = dot3(kk, nrm), kt[3];
        for (int a = 0; a < 3; ++a) kt[a] = kk[a] - kn * nrm[a];
        double kt2 = dot3(kt, kt);
        set_vec(rec.exit_pos, x);
        if (kt2 > 1.0) {
            rec.status = CLOAK_RAY_TIR;
            set_vec(rec.exit_dir, d_cam);
        } else {
            double qn = sqrt(1.0 - kt2), dout[3], mdout[3];
            for (int a = 0; a < 3; ++a) {
                dout[a] = fma(qn, nrm[a], kt[a]);
                mdout[a] = -dout[a];
            }
            double tin = exit_factor(p, mode, eo, ee, c, nrm, mdout, qn);
            rec.weight = tin * q.w_out[k];
            rec.status = status;
            set_vec(rec.exit_dir, dout);
            rec.tile_id = room_hit(p, x, dout, rgb);
        }
    } else {  // STEP_LIMIT or SINGULAR
        rec.status = status;
        rec.exit_pos[0] = y[0]; rec.exit_pos[1] = y[1]; rec.exit_pos[2] = y[2];
        set_vec(rec.exit_dir, d_cam);
    }
}

template <int VAR, int MODE>
__global__ void __launch_bounds__(128) k_wf_exit(Params p, int spp, unsigned long long seed, Queue q,
                                                 float4 *samples, cloak_record *recs) {
    const unsigned int n = q.count[0];
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if (q.key[k] < 0) continue;  // finished before the integration (learned surrogate)
        long long idx = q.id[k];
        long long pix = idx / spp;
        int s = (int)(idx - pix * spp);
        int i = (int)(pix % p.W), j = (int)(pix / p.W);
        double o[3], d[3];
        camera_ray(p, i, j, s, spp, seed, o, d);
        cloak_record rec;
        float rgb[3];
        exit_slot(p, MODE, q, k, d, rec, rgb);
        store_sample(samples, recs, idx, rec, rgb);
    }
}

__global__ void k_wf_resolve(int npix, int spp, const float4 *samples, float4 *out);

}  // namespace ck

namespace ck {

template <int V, int M, int I, int PREC>
static cudaError_t wavefront_vmip(const Params &p, int spp, unsigned long long seed, const Queue &q, float4 *samples,
                                 cloak_record *recs, int packet, cudaStream_t st, cudaEvent_t *ev, const WfHook *hook) {
    long long n = (long long)p.W * p.Hp * spp;
    const int bs = 128;
    k_wf_entry<V, M><<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(p, spp, seed, q, samples, recs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (hook && (e = hook->fn(hook->ctx, q, st)) != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int pk = packet > 0 ? packet : 128;
    // the slowest rays go to the warps of LONG_RAY_BLOCKS blocks that have their SMs to themselves
    k_wf_sort_scan<<<1, 32, 0, st>>>(q, NBINS, (unsigned int)(p.long_ray_blocks * pk * p.reserve_per_thread));
    k_wf_sort_scatter<<<sms * 8, 256, 0, st>>>(q);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], st);
    // persistent integrator: exactly the resident grid
    int nb = 0;
    constexpr auto kern = wf_integrate_kernel<V, M, I, PREC>();
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, pk, 0);
    if (e != cudaSuccess) return e;
    Params pl = p;
    pl.dedicated_blocks = p.long_ray_blocks;
    kern<<<(nb > 0 ? nb : 1) * sms, pk, 0, st>>>(pl, q);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[2], st);
    k_wf_exit<V, M><<<sms * 16, 128, 0, st>>>(p, spp, seed, q, samples, recs);
    e = cudaGetLastError();
    if (ev) cudaEventRecord(ev[3], st);
    return e;
}

template <int V, int M, int I>
static cudaError_t wavefront_vmi(const Params &p, int spp, unsigned long long seed, const Queue &q, float4 *samples,
                                 cloak_record *recs, int packet, cudaStream_t st, cudaEvent_t *ev, const WfHook *hook) {
    if (p.precision != 0) return wavefront_vmip<V, M, I, 1>(p, spp, seed, q, samples, recs, packet, st, ev, hook);
    return wavefront_vmip<V, M, I, 0>(p, spp, seed, q, samples, recs, packet, st, ev, hook);
}

template <int V>
cudaError_t launch_wavefront_v(const Params &p, int mode, int spp, unsigned long long seed, const Queue &q,
                               float4 *samples, cloak_record *recs, int packet, cudaStream_t st, cudaEvent_t *ev,
                               const WfHook *hook) {
    if (mode == M_ORD && p.integ == I_RK4)
        return wavefront_vmi<V, M_ORD, I_RK4>(p, spp, seed, q, samples, recs, packet, st, ev, hook);
    if (mode == M_ORD && p.integ == I_DP45)
        return wavefront_vmi<V, M_ORD, I_DP45>(p, spp, seed, q, samples, recs, packet, st, ev, hook);
    if (mode == M_EXT && p.integ == I_RK4)
        return wavefront_vmi<V, M_EXT, I_RK4>(p, spp, seed, q, samples, recs, packet, st, ev, hook);
    if (mode == M_EXT && p.integ == I_DP45)
        return wavefront_vmi<V, M_EXT, I_DP45>(p, spp, seed, q, samples, recs, packet, st, ev, hook);
    return cudaErrorInvalidValue;
}

#define CK_INSTANTIATE_WAVEFRONT(V)                                                                        \
    template cudaError_t launch_wavefront_v<V>(const Params &, int, int, unsigned long long, const Queue &, \
                                               float4 *, cloak_record *, int, cudaStream_t, cudaEvent_t *, const WfHook *);

}  // namespace ck
