// capi.cu -- the C ABI of include/cloak.h: handle lifetime, argument checks, launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "batch.h"
#include "internal.h"
#include "surrogate.h"
#include "wavefront.cuh"

struct cloak {
    int variant;
    double R1, R2, H;
    double eo_t, ee_t, c_t[3];
    unsigned long long scene_seed;
    double eye[3], target[3], up[3], hfov;
    int W, Hp;
    int integ;
    double h_or_tol;
    int precision;
    long max_steps;
    int schedule, packet, steps_per_round;
    int long_ray_blocks, reserve_per_thread;  // schedule knobs (cloak_set_schedule_tuning)
    double cost_scale;
    int tuned;  // the knobs were set explicitly; until then the mixed precisions use their own defaults
    int analyzer;     // CLOAK_ANALYZER_*
    int formulation;  // CLOAK_FORM_*
    int device;
    // library-owned scratch of the wavefront schedule (queue + per-sample buffer), grown on demand
    void *scratch;
    size_t scratch_bytes;
    // stage timing: events recorded around the stages of the last render call
    int timing;        // 0 off, 1 on
    int timed_calls;   // renders since timing was enabled
    int timed_sched;   // schedule of the last timed render
    cudaEvent_t ev[5];
    // batched render: view table (pinned host staging + device copy) and the captured graph
    void *batch_host, *batch_dev;
    size_t batch_bytes;
    cudaStream_t cap_stream;
    cudaGraphExec_t graph_exec;
    cudaEvent_t graph_done;
    unsigned long long graph_key;
    // learned surrogate of the exit state (created by training, loading or setting parameters)
    ck::SurNet *sur;
    // the two polarisation images behind the unpolarised panel
    void *panel_img;
    size_t panel_bytes;
    // first-order reflections in the unpolarised and polariser panels: the reflected rays' queue and
    // their per-sample results
    int reflections;
    void *refl_scratch;
    size_t refl_bytes;
};

static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}
static int cuda_fail(cudaError_t e, const char *where) {
    return fail(CLOAK_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}
static bool finite3(const double *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

// Threads per block of the persistent integration kernel: the handle's setting, or the precision's default
// (128 for FP64, 64 for the mixed precisions)
static int eff_packet(const cloak *h) {
    if (h->packet > 0) return h->packet;
    return h->precision == CLOAK_MIXED || h->precision == CLOAK_MIXED_FF ? 64 : 0;
}

// Camera frame and material constants for the kernels.
static int make_params(const cloak *h, ck::Params &p) {
    memset(&p, 0, sizeof(p));
    p.variant = h->variant == CLOAK_RADIAL ? ck::V_RADIAL : h->variant == CLOAK_AZIMUTHAL ? ck::V_AZIMUTHAL : ck::V_TEST;
    p.R1 = h->R1;
    p.R2 = h->R2;
    p.H = h->H;
    p.halfH = 0.5 * h->H;
    double kk = h->R2 / (h->R2 - h->R1);
    p.K = kk * kk;
    p.invK = 1.0 / p.K;
    p.R1x2 = 2.0 * h->R1;
    p.R1sq = h->R1 * h->R1;
    p.R2sq = h->R2 * h->R2;
    p.eo_t = h->eo_t;
    p.ee_t = h->ee_t;
    double cl = std::sqrt(h->c_t[0] * h->c_t[0] + h->c_t[1] * h->c_t[1] + h->c_t[2] * h->c_t[2]);
    for (int i = 0; i < 3; ++i) p.c_t[i] = h->c_t[i] / cl;
    p.scene_seed = h->scene_seed;
    p.integ = h->integ == CLOAK_RK4 ? ck::I_RK4 : ck::I_DP45;
    p.precision = h->precision == CLOAK_MIXED ? 1 : h->precision == CLOAK_MIXED_FF ? 2 : 0;
    p.mixed_band = h->precision == CLOAK_MIXED || h->precision == CLOAK_MIXED_FF ? 0.02 : 0.0;
    p.band_df = h->precision == CLOAK_MIXED_FF;
    p.R1f = (float)p.R1;
    p.R2f = (float)p.R2;
    p.halfHf = (float)p.halfH;
    p.Kf = (float)p.K;
    p.invKf = (float)p.invK;
    p.R1sq_hf = (float)p.R1sq;
    p.R1sq_lf = (float)(p.R1sq - (double)p.R1sq_hf);
    p.R2sq_hf = (float)p.R2sq;
    p.R2sq_lf = (float)(p.R2sq - (double)p.R2sq_hf);
    p.halfH_hf = (float)p.halfH;
    p.halfH_lf = (float)(p.halfH - (double)p.halfH_hf);
    p.band_limf = p.mixed_band > 0.0 ? (float)(p.R1 + p.mixed_band) : 0.f;
    p.h_or_tol = h->h_or_tol;
    p.max_steps = h->max_steps;
    if (h->tuned || !(h->precision == CLOAK_MIXED || h->precision == CLOAK_MIXED_FF)) {
        p.long_ray_blocks = h->long_ray_blocks;
        p.reserve_per_thread = h->reserve_per_thread;
        p.cost_scale = (float)h->cost_scale;
    } else {  // the mixed precisions' defaults: the best settings the tuner found on the twelve-view step
        p.long_ray_blocks = 16;
        p.reserve_per_thread = 4;
        p.cost_scale = 3.0f;
    }
    double w[3], u[3], v[3];
    for (int i = 0; i < 3; ++i) w[i] = h->target[i] - h->eye[i];
    double l = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (!(l > 0)) return fail(CLOAK_EINVAL, "camera eye and target coincide");
    for (int i = 0; i < 3; ++i) w[i] /= l;
    u[0] = w[1] * h->up[2] - w[2] * h->up[1];
    u[1] = w[2] * h->up[0] - w[0] * h->up[2];
    u[2] = w[0] * h->up[1] - w[1] * h->up[0];
    l = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (!(l > 1e-300)) return fail(CLOAK_EINVAL, "camera up vector is parallel to the view direction");
    for (int i = 0; i < 3; ++i) u[i] /= l;
    v[0] = u[1] * w[2] - u[2] * w[1];
    v[1] = u[2] * w[0] - u[0] * w[2];
    v[2] = u[0] * w[1] - u[1] * w[0];
    for (int i = 0; i < 3; ++i) {
        p.eye[i] = h->eye[i];
        p.fw[i] = w[i];
        p.rt[i] = u[i];
        p.up[i] = v[i];
    }
    p.tx = std::tan(0.5 * h->hfov * M_PI / 180.0);
    p.ty = p.tx * (double)h->Hp / (double)h->W;
    p.W = h->W;
    p.Hp = h->Hp;
    p.analyzer = h->analyzer;
    p.formulation = h->formulation == CLOAK_FORM_HAMILTONIAN ? 1 : 0;
    return CLOAK_OK;
}

// Carve the wavefront queue (SoA, cap slots) and the per-sample buffer out of the handle's scratch.
static int wavefront_scratch(cloak *h, long long cap, ck::Queue &q, float4 **samples) {
    size_t need = ck::queue_bytes(cap);
    if (h->scratch_bytes < need) {
        if (h->scratch) {
            cudaError_t e = cudaFree(h->scratch);
            h->scratch = nullptr;
            h->scratch_bytes = 0;
            if (e != cudaSuccess) return cuda_fail(e, "cudaFree(scratch)");
        }
        cudaError_t e = cudaMalloc(&h->scratch, need);
        if (e != cudaSuccess) {
            h->scratch = nullptr;
            cudaGetLastError();
            return fail(CLOAK_ENOMEM, "cannot allocate %zu bytes of wavefront scratch: %s", need, cudaGetErrorString(e));
        }
        h->scratch_bytes = need;
    }
    ck::carve_queue((char *)h->scratch, cap, q, samples);
    return CLOAK_OK;
}

static int run_wavefront(cloak *h, const ck::Params &p, int pol, int spp, unsigned long long seed, float4 *out,
                         cloak_record *recs, cudaStream_t st) {
    long long cap = (long long)p.W * p.Hp * spp;
    if (cap > 2147483647LL) return fail(CLOAK_EINVAL, "width*height*spp = %lld exceeds 2^31-1", cap);
    ck::Queue q;
    float4 *samples = nullptr;
    int rc = wavefront_scratch(h, cap, q, &samples);
    if (rc) return rc;
    // learned surrogate: only for the geometry it was trained on (elsewhere every ray is integrated)
    ck::SurRenderCtx sctx;
    ck::WfHook hook{ck::sur_render_hook, &sctx};
    const ck::WfHook *hk = nullptr;
    if (h->precision == CLOAK_SURROGATE) {
        if (!h->sur || !h->sur->trained) return fail(CLOAK_ESTATE, "CLOAK_SURROGATE needs a trained surrogate");
        const ck::SurNet *sn = h->sur;
        const bool same = std::fabs(sn->R1 - h->R1) <= 1e-12 * h->R2 && std::fabs(sn->R2 - h->R2) <= 1e-12 * h->R2 &&
                          std::fabs(sn->H - h->H) <= 1e-12 * h->H &&
                          (h->variant == CLOAK_RADIAL || h->variant == CLOAK_AZIMUTHAL);
        if (same) {
            sctx.s = h->sur;
            sctx.p = p;
            sctx.mode = pol;
            sctx.spp = spp;
            sctx.seed = seed;
            sctx.samples = recs ? nullptr : samples;
            sctx.recs = recs;
            sctx.cap = cap;
            hk = &hook;
        }
    }
    cudaEvent_t *ev = h->timing ? h->ev : nullptr;
    if (ev) cudaEventRecord(ev[0], st);
    cudaError_t e = cudaMemsetAsync(q.count, 0, ck::QUEUE_HEADER_BYTES, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    e = ck::launch_wavefront(p, pol, spp, seed, q, recs ? nullptr : samples, recs, eff_packet(h), st, ev, hk);
    if (e != cudaSuccess) return cuda_fail(e, "wavefront launch");
    if (!recs) {
        e = ck::launch_resolve(p.W * p.Hp, spp, samples, out, st);
        if (e != cudaSuccess) return cuda_fail(e, "resolve launch");
    }
    if (ev) {
        cudaEventRecord(ev[4], st);
        h->timed_calls++;
        h->timed_sched = CLOAK_SCHED_WAVEFRONT;
    }
    return CLOAK_OK;
}

static int use_device(const cloak *h) {
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return CLOAK_OK;
}

extern "C" {

const char *cloak_last_error(void) { return g_err.c_str(); }

cloak_t *cloak_create(int variant, double R1, double R2, double height) {
    if (variant != CLOAK_RADIAL && variant != CLOAK_AZIMUTHAL && variant != CLOAK_TEST_UNIAXIAL_CONST) {
        fail(CLOAK_EINVAL, "unknown variant %d", variant);
        return nullptr;
    }
    if (!(std::isfinite(R1) && std::isfinite(R2) && std::isfinite(height) && height > 0 && R2 > 0)) {
        fail(CLOAK_EINVAL, "geometry must be finite with R2 > 0 and height > 0");
        return nullptr;
    }
    if (variant == CLOAK_TEST_UNIAXIAL_CONST ? (R1 != 0.0) : !(R1 > 0 && R1 < R2)) {
        fail(CLOAK_EINVAL, variant == CLOAK_TEST_UNIAXIAL_CONST ? "test medium needs R1 = 0" : "need 0 < R1 < R2");
        return nullptr;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cuda_fail(e, "cudaGetDevice");
        return nullptr;
    }
    cloak *h = new (std::nothrow) cloak();
    if (!h) {
        fail(CLOAK_ENOMEM, "out of host memory");
        return nullptr;
    }
    h->variant = variant;
    h->R1 = R1;
    h->R2 = R2;
    h->H = height;
    h->eo_t = h->ee_t = 1.0;
    h->c_t[0] = 0; h->c_t[1] = 0; h->c_t[2] = 1;
    h->scene_seed = 0;
    h->eye[0] = 5; h->eye[1] = 0; h->eye[2] = 0;
    h->target[0] = h->target[1] = h->target[2] = 0;
    h->up[0] = 0; h->up[1] = 0; h->up[2] = 1;
    h->hfov = 60.0;
    h->W = 128;
    h->Hp = 96;
    h->integ = CLOAK_RK4;
    h->h_or_tol = 1e-3;
    h->precision = CLOAK_FP64;
    h->max_steps = 1000000;
    h->schedule = CLOAK_SCHED_PLAIN;
    h->packet = 0;
    h->long_ray_blocks = ck::LONG_RAY_BLOCKS;
    h->reserve_per_thread = 1;
    h->cost_scale = 4.0;
    h->steps_per_round = 0;
    h->analyzer = CLOAK_ANALYZER_NONE;
    h->formulation = CLOAK_FORM_FERMAT;
    h->device = dev;
    h->scratch = nullptr;
    h->scratch_bytes = 0;
    h->timing = 0;
    h->timed_calls = 0;
    h->timed_sched = 0;
    h->batch_host = h->batch_dev = nullptr;
    h->batch_bytes = 0;
    h->cap_stream = nullptr;
    h->graph_exec = nullptr;
    h->graph_done = nullptr;
    h->graph_key = 0;
    h->sur = nullptr;
    h->panel_img = nullptr;
    h->panel_bytes = 0;
    g_err.clear();
    return h;
}

void cloak_destroy(cloak_t *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->graph_done) cudaEventSynchronize(h->graph_done);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph_done) cudaEventDestroy(h->graph_done);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->batch_host) cudaFreeHost(h->batch_host);
    if (h->batch_dev) cudaFree(h->batch_dev);
    if (h->scratch) cudaFree(h->scratch);
    ck::sur_destroy(h->sur);
    if (h->panel_img) cudaFree(h->panel_img);
    if (h->refl_scratch) cudaFree(h->refl_scratch);
    if (h->timing)
        for (int i = 0; i < 5; ++i) cudaEventDestroy(h->ev[i]);
    delete h;
}

int cloak_set_stage_timing(cloak_t *h, int on) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    int rc = use_device(h);
    if (rc) return rc;
    if (on && !h->timing) {
        for (int i = 0; i < 5; ++i) {
            cudaError_t e = cudaEventCreate(&h->ev[i]);
            if (e != cudaSuccess) {
                for (int j = 0; j < i; ++j) cudaEventDestroy(h->ev[j]);
                return cuda_fail(e, "cudaEventCreate");
            }
        }
        h->timing = 1;
        h->timed_calls = 0;
    } else if (!on && h->timing) {
        cudaError_t e = cudaDeviceSynchronize();
        for (int i = 0; i < 5; ++i) cudaEventDestroy(h->ev[i]);
        h->timing = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    }
    return CLOAK_OK;
}

int cloak_stage_times(cloak_t *h, float ms[4]) {
    if (!h || !ms) return fail(CLOAK_EINVAL, "null argument");
    if (!h->timing || h->timed_calls == 0) return fail(CLOAK_ESTATE, "stage timing is off or nothing was timed");
    int rc = use_device(h);
    if (rc) return rc;
    cudaError_t e = cudaEventSynchronize(h->ev[4]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    for (int i = 0; i < 4; ++i) ms[i] = 0.f;
    if (h->timed_sched == CLOAK_SCHED_WAVEFRONT) {
        for (int i = 0; i < 4; ++i) {
            e = cudaEventElapsedTime(&ms[i], h->ev[i], h->ev[i + 1]);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        }
    } else {
        e = cudaEventElapsedTime(&ms[1], h->ev[0], h->ev[4]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    }
    return CLOAK_OK;
}

int cloak_camera_set(cloak_t *h, const double eye[3], const double target[3], const double up[3], double hfov_deg,
                     int width, int height) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (!eye || !target || !up) return fail(CLOAK_EINVAL, "null camera vector");
    if (!finite3(eye) || !finite3(target) || !finite3(up)) return fail(CLOAK_EINVAL, "camera vectors must be finite");
    if (!(hfov_deg > 0 && hfov_deg < 180)) return fail(CLOAK_EINVAL, "hfov must be in (0, 180) degrees");
    if (width < 1 || height < 1 || (long long)width * height > 2147483647LL)
        return fail(CLOAK_EINVAL, "image size %dx%d out of range", width, height);
    cloak tmp = *h;
    for (int i = 0; i < 3; ++i) { tmp.eye[i] = eye[i]; tmp.target[i] = target[i]; tmp.up[i] = up[i]; }
    tmp.hfov = hfov_deg;
    tmp.W = width;
    tmp.Hp = height;
    ck::Params p;
    int rc = make_params(&tmp, p);
    if (rc != CLOAK_OK) return rc;
    *h = tmp;
    return CLOAK_OK;
}

int cloak_set_integrator(cloak_t *h, int kind, double h_or_tol, int precision, long max_steps) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (kind != CLOAK_RK4 && kind != CLOAK_DP45) return fail(CLOAK_EINVAL, "unknown integrator %d", kind);
    if (!(std::isfinite(h_or_tol) && h_or_tol > 0)) return fail(CLOAK_EINVAL, "step / tolerance must be > 0");
    if (precision != CLOAK_FP64 && precision != CLOAK_MIXED && precision != CLOAK_MIXED_FF &&
        precision != CLOAK_SURROGATE)
        return fail(CLOAK_EINVAL, "unknown precision %d", precision);
    if (max_steps < 1 || max_steps > 2000000000L) return fail(CLOAK_EINVAL, "max_steps out of range");
    if (h->formulation == CLOAK_FORM_HAMILTONIAN && (precision == CLOAK_MIXED || precision == CLOAK_MIXED_FF))
        return fail(CLOAK_EINVAL, "the Hamiltonian form runs in FP64");
    h->integ = kind;
    h->h_or_tol = h_or_tol;
    h->precision = precision;
    h->max_steps = max_steps;
    return CLOAK_OK;
}

int cloak_set_test_medium(cloak_t *h, double eps_o, double eps_e, const double c_hat[3]) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (h->variant != CLOAK_TEST_UNIAXIAL_CONST) return fail(CLOAK_ESTATE, "not a test-medium handle");
    if (!c_hat || !finite3(c_hat)) return fail(CLOAK_EINVAL, "optic axis must be finite");
    double l = std::sqrt(c_hat[0] * c_hat[0] + c_hat[1] * c_hat[1] + c_hat[2] * c_hat[2]);
    if (!(l > 0) || !(eps_o > 0) || !(eps_e > 0) || !std::isfinite(eps_o) || !std::isfinite(eps_e))
        return fail(CLOAK_EINVAL, "need eps_o, eps_e > 0 and a nonzero optic axis");
    h->eo_t = eps_o;
    h->ee_t = eps_e;
    for (int i = 0; i < 3; ++i) h->c_t[i] = c_hat[i];
    return CLOAK_OK;
}

int cloak_set_formulation(cloak_t *h, int formulation) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (formulation != CLOAK_FORM_FERMAT && formulation != CLOAK_FORM_HAMILTONIAN)
        return fail(CLOAK_EINVAL, "unknown formulation %d", formulation);
    if (formulation == CLOAK_FORM_HAMILTONIAN) {
        if (h->variant != CLOAK_RADIAL && h->variant != CLOAK_AZIMUTHAL)
            return fail(CLOAK_ESTATE, "the Hamiltonian form needs a radial or azimuthal cloak handle");
        if (h->precision == CLOAK_MIXED || h->precision == CLOAK_MIXED_FF)
            return fail(CLOAK_ESTATE, "the Hamiltonian form runs in FP64");
    }
    h->formulation = formulation;
    return CLOAK_OK;
}

int cloak_set_reflections(cloak_t *h, int on) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (on != 0 && on != 1) return fail(CLOAK_EINVAL, "reflections must be 0 or 1");
    h->reflections = on;
    return CLOAK_OK;
}

int cloak_set_analyzer(cloak_t *h, int analyzer) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (analyzer != CLOAK_ANALYZER_NONE && analyzer != CLOAK_ANALYZER_RIGHT && analyzer != CLOAK_ANALYZER_UP)
        return fail(CLOAK_EINVAL, "unknown analyzer %d", analyzer);
    h->analyzer = analyzer;
    return CLOAK_OK;
}

int cloak_set_scene_seed(cloak_t *h, unsigned long long seed) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    h->scene_seed = seed;
    return CLOAK_OK;
}

int cloak_set_schedule_tuning(cloak_t *h, int long_ray_blocks, int reserve_per_thread, double cost_scale) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (long_ray_blocks < 0 || long_ray_blocks > 64) return fail(CLOAK_EINVAL, "long_ray_blocks must be in [0, 64]");
    if (reserve_per_thread < 1 || reserve_per_thread > 8)
        return fail(CLOAK_EINVAL, "reserve_per_thread must be in [1, 8]");
    if (!(cost_scale >= 1.0 && cost_scale <= 16.0)) return fail(CLOAK_EINVAL, "cost_scale must be in [1, 16]");
    h->long_ray_blocks = long_ray_blocks;
    h->reserve_per_thread = reserve_per_thread;
    h->cost_scale = cost_scale;
    h->tuned = 1;
    return CLOAK_OK;
}

int cloak_set_schedule(cloak_t *h, int schedule, int packet, int steps_per_round) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (schedule != CLOAK_SCHED_PLAIN && schedule != CLOAK_SCHED_WAVEFRONT)
        return fail(CLOAK_EINVAL, "unknown schedule %d", schedule);
    if (packet != 0 && (packet < 32 || packet > 128 || packet % 32))
        return fail(CLOAK_EINVAL, "packet must be 0 or a multiple of 32 in [32, 128]");
    if (steps_per_round < 0) return fail(CLOAK_EINVAL, "steps_per_round must be >= 0");
    h->schedule = schedule;
    h->packet = packet;
    h->steps_per_round = steps_per_round;
    return CLOAK_OK;
}

int cloak_render(cloak_t *h, int polarization, int spp, unsigned long long seed, void *dev_rgba, size_t bytes,
                 void *cuda_stream) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (polarization != CLOAK_POL_ORDINARY && polarization != CLOAK_POL_EXTRAORDINARY)
        return fail(CLOAK_EINVAL, "unknown polarization %d", polarization);
    if (spp < 1 || spp > 65536) return fail(CLOAK_EINVAL, "spp must be in [1, 65536]");
    size_t need = (size_t)h->W * h->Hp * 16;
    if (!dev_rgba) return fail(CLOAK_EINVAL, "null output buffer");
    if (bytes < need) return fail(CLOAK_EINVAL, "output buffer holds %zu bytes, needs %zu", bytes, need);
    ck::Params p;
    int rc = make_params(h, p);
    if (rc) return rc;
    if ((rc = use_device(h))) return rc;
    if (h->schedule == CLOAK_SCHED_WAVEFRONT)
        return run_wavefront(h, p, polarization, spp, seed, (float4 *)dev_rgba, nullptr, (cudaStream_t)cuda_stream);
    if (h->precision != CLOAK_FP64) return fail(CLOAK_EINVAL, "this precision needs the wavefront schedule");
    if (h->timing) cudaEventRecord(h->ev[0], (cudaStream_t)cuda_stream);
    cudaError_t e = ck::launch_render_plain(p, polarization, spp, seed, (float4 *)dev_rgba, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "render launch");
    if (h->timing) {
        cudaEventRecord(h->ev[4], (cudaStream_t)cuda_stream);
        h->timed_calls++;
        h->timed_sched = CLOAK_SCHED_PLAIN;
    }
    return CLOAK_OK;
}

int cloak_render_records(cloak_t *h, int polarization, int spp, unsigned long long seed, void *dev_records,
                         size_t bytes, void *cuda_stream) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (polarization != CLOAK_POL_ORDINARY && polarization != CLOAK_POL_EXTRAORDINARY)
        return fail(CLOAK_EINVAL, "unknown polarization %d", polarization);
    if (spp < 1 || spp > 65536) return fail(CLOAK_EINVAL, "spp must be in [1, 65536]");
    size_t need = (size_t)h->W * h->Hp * spp * sizeof(cloak_record);
    if (!dev_records) return fail(CLOAK_EINVAL, "null output buffer");
    if (bytes < need) return fail(CLOAK_EINVAL, "record buffer holds %zu bytes, needs %zu", bytes, need);
    ck::Params p;
    int rc = make_params(h, p);
    if (rc) return rc;
    if ((rc = use_device(h))) return rc;
    if (h->schedule == CLOAK_SCHED_WAVEFRONT)
        return run_wavefront(h, p, polarization, spp, seed, nullptr, (cloak_record *)dev_records,
                             (cudaStream_t)cuda_stream);
    if (h->precision != CLOAK_FP64) return fail(CLOAK_EINVAL, "this precision needs the wavefront schedule");
    if (h->timing) cudaEventRecord(h->ev[0], (cudaStream_t)cuda_stream);
    cudaError_t e = ck::launch_records_plain(p, polarization, spp, seed, (cloak_record *)dev_records,
                                             (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "records launch");
    if (h->timing) {
        cudaEventRecord(h->ev[4], (cudaStream_t)cuda_stream);
        h->timed_calls++;
        h->timed_sched = CLOAK_SCHED_PLAIN;
    }
    return CLOAK_OK;
}

int cloak_trace_rays(cloak_t *h, int polarization, const double *dev_rays, long n, void *dev_records,
                     void *cuda_stream) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (polarization != CLOAK_POL_ORDINARY && polarization != CLOAK_POL_EXTRAORDINARY)
        return fail(CLOAK_EINVAL, "unknown polarization %d", polarization);
    if (n < 0) return fail(CLOAK_EINVAL, "n must be >= 0");
    if (n == 0) return CLOAK_OK;
    if (!dev_rays || !dev_records) return fail(CLOAK_EINVAL, "null buffer");
    ck::Params p;
    int rc = make_params(h, p);
    if (rc) return rc;
    p.analyzer = 0;  // rays without a camera: no camera polariser
    if ((rc = use_device(h))) return rc;
    cudaError_t e = ck::launch_trace_rays(p, polarization, dev_rays, n, (cloak_record *)dev_records,
                                          (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "trace launch");
    return CLOAK_OK;
}

int cloak_eval_rhs(cloak_t *h, int polarization, const double *dev_y, long n, double *dev_dy, void *cuda_stream) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (polarization != CLOAK_POL_ORDINARY && polarization != CLOAK_POL_EXTRAORDINARY)
        return fail(CLOAK_EINVAL, "unknown polarization %d", polarization);
    if (h->variant != CLOAK_RADIAL && h->variant != CLOAK_AZIMUTHAL)
        return fail(CLOAK_ESTATE, "the equations of motion are evaluated for the radial and azimuthal cloaks");
    if (n < 0) return fail(CLOAK_EINVAL, "n must be >= 0");
    if (n == 0) return CLOAK_OK;
    if (!dev_y || !dev_dy) return fail(CLOAK_EINVAL, "null buffer");
    ck::Params p;
    int rc = make_params(h, p);
    if (rc) return rc;
    if ((rc = use_device(h))) return rc;
    cudaError_t e = ck::launch_eval_rhs(p, polarization, dev_y, n, dev_dy, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "rhs launch");
    return CLOAK_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Batched render
// ---------------------------------------------------------------------------------------------
static int view_frame(const cloak_view &v, ck::ViewDev &d) {
    if (v.variant != CLOAK_RADIAL && v.variant != CLOAK_AZIMUTHAL) return fail(CLOAK_EINVAL, "view variant %d", v.variant);
    if (v.polarization != CLOAK_POL_ORDINARY && v.polarization != CLOAK_POL_EXTRAORDINARY)
        return fail(CLOAK_EINVAL, "view polarization %d", v.polarization);
    if (!finite3(v.eye) || !finite3(v.target) || !finite3(v.up)) return fail(CLOAK_EINVAL, "view camera not finite");
    if (!(v.hfov_deg > 0 && v.hfov_deg < 180)) return fail(CLOAK_EINVAL, "view hfov out of (0, 180)");
    if (v.width < 1 || v.height < 1 || (long long)v.width * v.height > 2147483647LL)
        return fail(CLOAK_EINVAL, "view size %dx%d out of range", v.width, v.height);
    if (!v.dev_rgba) return fail(CLOAK_EINVAL, "view without output buffer");
    double w[3], u[3], up[3];
    for (int i = 0; i < 3; ++i) w[i] = v.target[i] - v.eye[i];
    double l = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (!(l > 0)) return fail(CLOAK_EINVAL, "view eye and target coincide");
    for (int i = 0; i < 3; ++i) w[i] /= l;
    u[0] = w[1] * v.up[2] - w[2] * v.up[1];
    u[1] = w[2] * v.up[0] - w[0] * v.up[2];
    u[2] = w[0] * v.up[1] - w[1] * v.up[0];
    l = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (!(l > 1e-300)) return fail(CLOAK_EINVAL, "view up vector parallel to the view direction");
    for (int i = 0; i < 3; ++i) u[i] /= l;
    up[0] = u[1] * w[2] - u[2] * w[1];
    up[1] = u[2] * w[0] - u[0] * w[2];
    up[2] = u[0] * w[1] - u[1] * w[0];
    for (int i = 0; i < 3; ++i) { d.eye[i] = v.eye[i]; d.fw[i] = w[i]; d.rt[i] = u[i]; d.up[i] = up[i]; }
    d.tx = std::tan(0.5 * v.hfov_deg * M_PI / 180.0);
    d.ty = d.tx * (double)v.height / (double)v.width;
    d.W = v.width;
    d.Hp = v.height;
    d.vm = 2 * v.variant + v.polarization;
    d.pad = 0;
    d.out = (float4 *)v.dev_rgba;
    return CLOAK_OK;
}

static unsigned long long fnv1a(unsigned long long hsh, const void *data, size_t n) {
    const unsigned char *b = (const unsigned char *)data;
    for (size_t i = 0; i < n; ++i) { hsh ^= b[i]; hsh *= 1099511628211ull; }
    return hsh;
}

// The batched render (views validated, device table, graph capture or replay); samples_out (nullable)
// receives the per-sample buffer of the batch.
static int batch_core(cloak_t *h, const cloak_view *views, int nviews, int spp, unsigned long long seed,
                      void *cuda_stream, float4 **samples_out, int analyzer, int tof = 0, ck::Queue *q_out = nullptr);

extern "C" int cloak_set_wait_limit(long long polls) {
    g_err.clear();
    if (polls < 0 || polls > 0xffffffffll) return fail(CLOAK_EINVAL, "cloak_set_wait_limit: polls must be in [0, 2^32 - 1]");
    ck::set_wait_limit((unsigned int)polls);
    return CLOAK_OK;
}

extern "C" int cloak_fma_peak(int precision, int blocks, int threads, long long iters, void *dev_sink,
                              double *flops, void *cuda_stream) {
    g_err.clear();
    if (precision != CLOAK_FP64 && precision != CLOAK_MIXED)
        return fail(CLOAK_EINVAL, "cloak_fma_peak: precision must be CLOAK_FP64 or CLOAK_MIXED");
    if (blocks < 1 || threads < 32 || threads > 256 || threads % 32 != 0 || iters < 1)
        return fail(CLOAK_EINVAL, "cloak_fma_peak: need blocks >= 1, threads a multiple of 32 in [32, 256], iters >= 1");
    if (!dev_sink || !flops) return fail(CLOAK_EINVAL, "cloak_fma_peak: null sink or flops");
    cudaError_t e = ck::launch_fma_peak(precision == CLOAK_FP64, blocks, threads, iters, dev_sink, flops,
                                        (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? CLOAK_OK : cuda_fail(e, "cloak_fma_peak");
}

extern "C" int cloak_render_batch(cloak_t *h, const cloak_view *views, int nviews, int spp, unsigned long long seed,
                                  void *cuda_stream) {
    return batch_core(h, views, nviews, spp, seed, cuda_stream, nullptr, h ? h->analyzer : 0);
}

static int batch_core(cloak_t *h, const cloak_view *views, int nviews, int spp, unsigned long long seed,
                      void *cuda_stream, float4 **samples_out, int analyzer, int tof, ck::Queue *q_out) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (h->variant != CLOAK_RADIAL && h->variant != CLOAK_AZIMUTHAL)
        return fail(CLOAK_ESTATE, "batched rendering needs a radial or azimuthal cloak handle");
    if (!views || nviews < 1 || nviews > 65536) return fail(CLOAK_EINVAL, "need 1..65536 views");
    if (spp < 1 || spp > 65536) return fail(CLOAK_EINVAL, "spp must be in [1, 65536]");
    ck::Params p;
    int rc = make_params(h, p);
    if (rc) return rc;
    p.analyzer = analyzer;
    p.tof = tof;
    // learned surrogate: rays it is confident about leave the queue before the integration (the
    // integrator handles the rest, and everything when the network was trained on another geometry)
    const bool sur = h->precision == CLOAK_SURROGATE && tof == 0 && h->sur && h->sur->trained &&
                     std::fabs(h->sur->R1 - h->R1) <= 1e-12 * h->R2 && std::fabs(h->sur->R2 - h->R2) <= 1e-12 * h->R2 &&
                     std::fabs(h->sur->H - h->H) <= 1e-12 * h->H;
    if (h->precision == CLOAK_SURROGATE && !(h->sur && h->sur->trained))
        return fail(CLOAK_ESTATE, "CLOAK_SURROGATE needs a trained surrogate");
    std::vector<ck::ViewDev> table((size_t)nviews);
    long long total = 0, total_pix = 0;
    for (int i = 0; i < nviews; ++i) {
        if ((rc = view_frame(views[i], table[i]))) return rc;
        table[i].ray_begin = total;
        table[i].pix_begin = total_pix;
        total += (long long)views[i].width * views[i].height * spp;
        total_pix += (long long)views[i].width * views[i].height;
    }
    if (total > 2147483647LL) return fail(CLOAK_EINVAL, "batch holds %lld samples, more than 2^31-1", total);
    if ((rc = use_device(h))) return rc;
    ck::Queue q;
    float4 *samples = nullptr;
    if ((rc = wavefront_scratch(h, total, q, &samples))) return rc;
    if (q_out) *q_out = q;
    if (sur) {  // the network's buffers for every queued ray and its kernel set up, before any capture
        cudaError_t e = ck::sur_ensure_inference(h->sur, total);
        if (e == cudaSuccess) e = ck::mlp_fused_prepare();
        if (e != cudaSuccess) return cuda_fail(e, "surrogate buffers");
    }
    size_t tbytes = table.size() * sizeof(ck::ViewDev);
    unsigned long long key = 1469598103934665603ull;
    key = fnv1a(key, table.data(), tbytes);
    key = fnv1a(key, &p, sizeof(p));
    int extra[5] = {spp, eff_packet(h), nviews, h->timing, sur ? 1 : 0};
    key = fnv1a(key, extra, sizeof(extra));
    key = fnv1a(key, &seed, sizeof(seed));
    key = fnv1a(key, &h->scratch, sizeof(h->scratch));
    if (sur) {  // the captured launches hold the network's buffers and the gate
        const void *bufs[3] = {h->sur->X, h->sur->Y, h->sur->elig};
        key = fnv1a(key, bufs, sizeof(bufs));
        key = fnv1a(key, &h->sur->gate, sizeof(h->sur->gate));
        key = fnv1a(key, &h->sur->inf_f16, sizeof(h->sur->inf_f16));
        const unsigned int lim = ck::wait_limit();  // baked into the captured network launch
        key = fnv1a(key, &lim, sizeof(lim));
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaError_t e;
    if (!h->graph_exec || key != h->graph_key) {
        // the previous graph may still read the staging buffer
        if (h->graph_done && (e = cudaEventSynchronize(h->graph_done)) != cudaSuccess)
            return cuda_fail(e, "cudaEventSynchronize");
        if (h->batch_bytes < tbytes) {
            if (h->batch_host) cudaFreeHost(h->batch_host);
            if (h->batch_dev) cudaFree(h->batch_dev);
            h->batch_host = h->batch_dev = nullptr;
            h->batch_bytes = 0;
            if ((e = cudaHostAlloc(&h->batch_host, tbytes, cudaHostAllocDefault)) != cudaSuccess)
                return fail(CLOAK_ENOMEM, "pinned view table: %s", cudaGetErrorString(e));
            if ((e = cudaMalloc(&h->batch_dev, tbytes)) != cudaSuccess) {
                cudaFreeHost(h->batch_host);
                h->batch_host = nullptr;
                return fail(CLOAK_ENOMEM, "device view table: %s", cudaGetErrorString(e));
            }
            h->batch_bytes = tbytes;
        }
        memcpy(h->batch_host, table.data(), tbytes);
        if (!h->cap_stream && (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreate");
        if (!h->graph_done && (e = cudaEventCreateWithFlags(&h->graph_done, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate");
        if (h->graph_exec) {
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
        }
        if ((e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamBeginCapture");
        cudaError_t e1 = cudaMemcpyAsync(h->batch_dev, h->batch_host, tbytes, cudaMemcpyHostToDevice, h->cap_stream);
        ck::SurRenderCtx sctx;
        ck::WfHook hook{ck::sur_render_hook, &sctx};
        if (sur) {
            sctx.s = h->sur;
            sctx.p = p;
            sctx.mode = 0;
            sctx.spp = spp;
            sctx.seed = seed;
            sctx.samples = samples;
            sctx.recs = nullptr;
            sctx.cap = total;
            sctx.views = (const ck::ViewDev *)h->batch_dev;
            sctx.nviews = nviews;
        }
        cudaError_t e2 = e1 == cudaSuccess ? ck::launch_batch(p, (const ck::ViewDev *)h->batch_dev, nviews, spp, seed,
                                                             total, total_pix, q, samples, eff_packet(h), h->cap_stream,
                                                             h->timing ? h->ev : nullptr, sur ? &hook : nullptr)
                                           : e1;
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (e2 != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return cuda_fail(e2 != cudaSuccess ? e2 : e, "batch capture");
        }
        e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            h->graph_exec = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        h->graph_key = key;
    }
    if ((e = cudaGraphLaunch(h->graph_exec, st)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    if ((e = cudaEventRecord(h->graph_done, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if (h->timing) {
        h->timed_calls++;
        h->timed_sched = CLOAK_SCHED_WAVEFRONT;
    }
    if (samples_out) *samples_out = samples;
    return CLOAK_OK;
}

// ---------------------------------------------------------------------------------------------
// Panels of the paper's figures
// ---------------------------------------------------------------------------------------------
extern "C" int cloak_render_panel(cloak_t *h, int panel, int spp, unsigned long long seed, void *dev_rgba,
                                  size_t bytes, void *cuda_stream) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (panel != CLOAK_PANEL_ROOM && panel != CLOAK_PANEL_METAL && panel != CLOAK_PANEL_UNPOLARIZED &&
        panel != CLOAK_PANEL_POLARIZER_RIGHT && panel != CLOAK_PANEL_POLARIZER_UP && panel != CLOAK_PANEL_TOF)
        return fail(CLOAK_EINVAL, "unknown panel %d", panel);
    if (spp < 1 || spp > 65536) return fail(CLOAK_EINVAL, "spp must be in [1, 65536]");
    const size_t npix = (size_t)h->W * h->Hp;
    if (!dev_rgba) return fail(CLOAK_EINVAL, "null output buffer");
    if (bytes < npix * 16) return fail(CLOAK_EINVAL, "output buffer holds %zu bytes, needs %zu", bytes, npix * 16);
    ck::Params p;
    int rc = make_params(h, p);
    if (rc) return rc;
    if ((rc = use_device(h))) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (panel == CLOAK_PANEL_ROOM || panel == CLOAK_PANEL_METAL) {
        cudaError_t e = ck::launch_panel(p, panel, spp, seed, (float4 *)dev_rgba, st);
        return e == cudaSuccess ? CLOAK_OK : cuda_fail(e, "panel launch");
    }
    // the TOF image keeps the handle's own camera polariser
    const int analyzer = panel == CLOAK_PANEL_POLARIZER_RIGHT ? CLOAK_ANALYZER_RIGHT
                         : panel == CLOAK_PANEL_POLARIZER_UP  ? CLOAK_ANALYZER_UP
                         : panel == CLOAK_PANEL_TOF           ? h->analyzer
                                                              : CLOAK_ANALYZER_NONE;
    const int tof = panel == CLOAK_PANEL_TOF ? 1 : 0;
    p.analyzer = analyzer;
    p.tof = tof;
    if (h->variant != CLOAK_RADIAL && h->variant != CLOAK_AZIMUTHAL)
        return fail(CLOAK_ESTATE, "the unpolarised and TOF panels need a radial or azimuthal cloak handle");
    if (h->precision == CLOAK_SURROGATE)
        return fail(CLOAK_EINVAL, "the panels run the integrator: set the FP64 or mixed precision");
    // both polarisations in one batched render (their images go to handle scratch), then the sum
    if (h->panel_bytes < 2 * npix * 16) {
        if (h->panel_img) cudaFree(h->panel_img);
        h->panel_img = nullptr;
        h->panel_bytes = 0;
        cudaError_t e = cudaMalloc(&h->panel_img, 2 * npix * 16);
        if (e != cudaSuccess) {
            h->panel_img = nullptr;
            cudaGetLastError();
            return fail(CLOAK_ENOMEM, "panel scratch: %s", cudaGetErrorString(e));
        }
        h->panel_bytes = 2 * npix * 16;
    }
    cloak_view v[2];
    for (int m = 0; m < 2; ++m) {
        v[m].variant = h->variant;
        v[m].polarization = m;
        for (int k = 0; k < 3; ++k) { v[m].eye[k] = h->eye[k]; v[m].target[k] = h->target[k]; v[m].up[k] = h->up[k]; }
        v[m].hfov_deg = h->hfov;
        v[m].width = h->W;
        v[m].height = h->Hp;
        v[m].dev_rgba = (char *)h->panel_img + m * npix * 16;
    }
    float4 *samples = nullptr;
    const bool refl = h->reflections && !tof;
    const long long total = 2LL * (long long)npix * spp;
    if (refl && 2 * total > 2147483647LL)
        return fail(CLOAK_EINVAL, "reflections: 2 x %lld samples exceed 2^31-1", total);
    ck::Queue q;
    if ((rc = batch_core(h, v, 2, spp, seed, cuda_stream, &samples, analyzer, tof, &q))) return rc;
    float4 *rs = nullptr;
    if (refl) {
        // the reflected rays' queue; its per-sample buffer (2 x samples) holds their results
        const size_t need = ck::queue_bytes(2 * total);
        if (h->refl_bytes < need) {
            if (h->refl_scratch) cudaFree(h->refl_scratch);
            h->refl_scratch = nullptr;
            h->refl_bytes = 0;
            cudaError_t e = cudaMalloc(&h->refl_scratch, need);
            if (e != cudaSuccess) {
                h->refl_scratch = nullptr;
                cudaGetLastError();
                return fail(CLOAK_ENOMEM, "reflection scratch: %s", cudaGetErrorString(e));
            }
            h->refl_bytes = need;
        }
        ck::Queue q2;
        ck::carve_queue((char *)h->refl_scratch, 2 * total, q2, &rs);
        cudaError_t e = ck::launch_reflections(p, q, q2, rs, 2 * total, eff_packet(h), st);
        if (e != cudaSuccess) return cuda_fail(e, "reflections");
    }
    cudaError_t e = tof ? ck::launch_tof_resolve(p, (const ck::ViewDev *)h->batch_dev, spp, seed, (long long)npix,
                                                 samples, (float4 *)dev_rgba, st)
                        : ck::launch_unpol_resolve(p, (const ck::ViewDev *)h->batch_dev, spp, seed, (long long)npix,
                                                   samples, rs, (float4 *)dev_rgba, st);
    return e == cudaSuccess ? CLOAK_OK : cuda_fail(e, tof ? "TOF resolve" : "unpolarised resolve");
}

// ---------------------------------------------------------------------------------------------
// Allocation-free render (cloak_render_noalloc).  The wavefront queue and per-sample buffer live in
// a fixed file-scope device array instead of handle scratch, for callers that may not allocate
// device memory.  The array is part of this module: every GPU that loads the library holds it until
// the process exits.  Host code must not use the array's name as a device address; its address is
// resolved once per device with cudaGetSymbolAddress and passed to the kernels.
// ---------------------------------------------------------------------------------------------
static constexpr long long NOALLOC_MAX_SAMPLES = 1LL << 20;  // width * height * spp
static constexpr size_t NOALLOC_BYTES = ck::queue_bytes(NOALLOC_MAX_SAMPLES);
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

static constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[NOALLOC_MAX_DEVICES];

// Device address of the array on the current device (resolved on the first call per device).
static int noalloc_scratch_ptr(int dev, void **out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(CLOAK_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        if (!ptr) return fail(CLOAK_ECUDA, "cudaGetSymbolAddress returned a null address for the no-alloc scratch");
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return CLOAK_OK;
}

extern "C" int cloak_render_noalloc(cloak_t *h, int polarization, int spp, unsigned long long seed, void *dev_rgba,
                                    size_t bytes, void *cuda_stream) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (polarization != CLOAK_POL_ORDINARY && polarization != CLOAK_POL_EXTRAORDINARY)
        return fail(CLOAK_EINVAL, "unknown polarization %d", polarization);
    if (spp < 1 || spp > 65536) return fail(CLOAK_EINVAL, "spp must be in [1, 65536]");
    if (!dev_rgba) return fail(CLOAK_EINVAL, "null output buffer");
    size_t need = (size_t)h->W * h->Hp * 16;
    if (bytes < need) return fail(CLOAK_EINVAL, "output buffer holds %zu bytes, needs %zu", bytes, need);
    long long cap = (long long)h->W * h->Hp * spp;
    if (cap > NOALLOC_MAX_SAMPLES)
        return fail(CLOAK_EINVAL, "width*height*spp = %lld exceeds the no-alloc limit of %lld samples", cap,
                    NOALLOC_MAX_SAMPLES);
    if (h->precision == CLOAK_SURROGATE)
        return fail(CLOAK_EINVAL, "the learned surrogate allocates its scratch; use cloak_render");
    ck::Params p;
    int rc = make_params(h, p);
    if (rc) return rc;
    if ((rc = use_device(h))) return rc;
    void *base = nullptr;
    if ((rc = noalloc_scratch_ptr(h->device, &base))) return rc;
    // same layout as the handle scratch of the wavefront schedule
    ck::Queue q;
    float4 *samples = nullptr;
    ck::carve_queue((char *)base, cap, q, &samples);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the queue header (counters, sort bins) must start at zero; everything else is written before it is read
    cudaError_t e = cudaMemsetAsync(q.count, 0, ck::QUEUE_HEADER_BYTES, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    e = ck::launch_wavefront(p, polarization, spp, seed, q, samples, nullptr, eff_packet(h), st, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "wavefront launch");
    e = ck::launch_resolve(p.W * p.Hp, spp, samples, (float4 *)dev_rgba, st);
    if (e != cudaSuccess) return cuda_fail(e, "resolve launch");
    return CLOAK_OK;
}

// ---------------------------------------------------------------------------------------------
// Learned surrogate
// ---------------------------------------------------------------------------------------------
static int ensure_surrogate(cloak *h) {
    if (h->sur) return CLOAK_OK;
    if (h->variant != CLOAK_RADIAL && h->variant != CLOAK_AZIMUTHAL)
        return fail(CLOAK_ESTATE, "the surrogate needs a radial or azimuthal cloak handle");
    const char *why = "";
    h->sur = ck::sur_create(h->R1, h->R2, h->H, 0x5eedull, &why);
    if (!h->sur) return fail(CLOAK_ENOMEM, "%s", why);
    return CLOAK_OK;
}

extern "C" int cloak_surrogate_train(cloak_t *h, long n_rays, unsigned long long seed, int epochs, void *cuda_stream) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (n_rays < 19456 || n_rays > 2147483647L) return fail(CLOAK_EINVAL, "n_rays must be in [19456, 2^31 - 1]");
    if (epochs < 1 || epochs > 100000) return fail(CLOAK_EINVAL, "epochs must be in [1, 100000]");
    int rc = use_device(h);
    if (rc) return rc;
    if ((rc = ensure_surrogate(h))) return rc;
    ck::Params p;
    if ((rc = make_params(h, p))) return rc;
    h->sur->R1 = h->R1;
    h->sur->R2 = h->R2;
    h->sur->H = h->H;
    std::string why;
    rc = ck::sur_train(h->sur, p, n_rays, seed, epochs, (cudaStream_t)cuda_stream, why);
    if (rc) return fail(rc, "surrogate training: %s", why.c_str());
    return CLOAK_OK;
}

extern "C" int cloak_surrogate_save(cloak_t *h, const char *path) {
    if (!h || !path) return fail(CLOAK_EINVAL, "null argument");
    if (!h->sur) return fail(CLOAK_ESTATE, "the handle has no surrogate");
    int rc = use_device(h);
    if (rc) return rc;
    std::string why;
    rc = ck::sur_save(h->sur, path, why);
    return rc ? fail(rc, "%s", why.c_str()) : CLOAK_OK;
}

extern "C" int cloak_surrogate_load(cloak_t *h, const char *path) {
    if (!h || !path) return fail(CLOAK_EINVAL, "null argument");
    int rc = use_device(h);
    if (rc) return rc;
    if ((rc = ensure_surrogate(h))) return rc;
    std::string why;
    rc = ck::sur_load(h->sur, path, why);
    return rc ? fail(rc, "%s", why.c_str()) : CLOAK_OK;
}

extern "C" int cloak_surrogate_set_gate(cloak_t *h, double max_log10_err) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (!std::isfinite(max_log10_err)) return fail(CLOAK_EINVAL, "gate must be finite");
    if (!h->sur) return fail(CLOAK_ESTATE, "the handle has no surrogate");
    h->sur->gate = (float)max_log10_err;
    return CLOAK_OK;
}

extern "C" int cloak_surrogate_set_precision(cloak_t *h, int fp16) {
    if (!h) return fail(CLOAK_EINVAL, "null handle");
    if (fp16 != 0 && fp16 != 1) return fail(CLOAK_EINVAL, "fp16 must be 0 (BF16) or 1 (FP16)");
    int rc = use_device(h);
    if (rc) return rc;
    if ((rc = ensure_surrogate(h))) return rc;
    h->sur->inf_f16 = fp16;
    return CLOAK_OK;
}

extern "C" int cloak_surrogate_train_timing(cloak_t *h, double out[4]) {
    if (!h || !out) return fail(CLOAK_EINVAL, "null argument");
    if (!h->sur || !h->sur->trained || !(h->sur->train_ms[0] > 0.0))
        return fail(CLOAK_ESTATE, "the handle's surrogate was not trained by cloak_surrogate_train");
    const double B = h->sur->info[7];
    out[0] = h->sur->train_ms[0];
    out[1] = h->sur->train_ms[1];
    // algorithmic multiply-adds x 2 of a stage-1 step, unpadded: forward, backward data (layers 4..1) and
    // weight gradients (all layers) of 7 -> 256 -> 256 -> 256 -> 256 -> 5
    const double fwd = 7.0 * 256 + 3.0 * 256 * 256 + 256.0 * 5, bwd_data = 256.0 * 5 + 3.0 * 256 * 256;
    out[2] = 2.0 * B * (2.0 * fwd + bwd_data);
    out[3] = B;
    return CLOAK_OK;
}

extern "C" int cloak_surrogate_info(cloak_t *h, double info[8]) {
    if (!h || !info) return fail(CLOAK_EINVAL, "null argument");
    if (!h->sur || !h->sur->trained) return fail(CLOAK_ESTATE, "the handle has no trained surrogate");
    for (int i = 0; i < 8; ++i) info[i] = h->sur->info[i];
    return CLOAK_OK;
}

extern "C" int cloak_surrogate_params(cloak_t *h, float *host, long n, int set) {
    if (!h || !host) return fail(CLOAK_EINVAL, "null argument");
    if (n != ck::sur_nparams()) return fail(CLOAK_EINVAL, "the network has %lld parameters", ck::sur_nparams());
    int rc = use_device(h);
    if (rc) return rc;
    if ((rc = ensure_surrogate(h))) return rc;
    cudaError_t e = set ? ck::sur_set_params(h->sur, host) : ck::sur_get_params(h->sur, host);
    return e == cudaSuccess ? CLOAK_OK : cuda_fail(e, "surrogate parameters");
}

extern "C" int cloak_surrogate_forward(cloak_t *h, const float *dev_x, long n, float *dev_y, void *cuda_stream) {
    if (!h || !dev_x || !dev_y) return fail(CLOAK_EINVAL, "null argument");
    if (n < 1 || n > 2147483647L) return fail(CLOAK_EINVAL, "n out of range");
    if (!h->sur) return fail(CLOAK_ESTATE, "the handle has no surrogate");
    int rc = use_device(h);
    if (rc) return rc;
    std::string why;
    rc = ck::sur_forward_rows(h->sur, dev_x, n, dev_y, (cudaStream_t)cuda_stream, why);
    return rc ? fail(rc, "%s", why.c_str()) : CLOAK_OK;
}

extern "C" int cloak_surrogate_step(cloak_t *h, const float *dev_x, const float *dev_t, long n, int stage, double lr,
                                    float *host_grad, void *cuda_stream) {
    if (!h || !dev_x || !dev_t) return fail(CLOAK_EINVAL, "null argument");
    if (n < 128 || n % 128 || n > (1L << 24)) return fail(CLOAK_EINVAL, "n must be a multiple of 128 in [128, 2^24]");
    if (stage != 1 && stage != 2) return fail(CLOAK_EINVAL, "stage must be 1 or 2");
    if (!(lr >= 0) || !std::isfinite(lr)) return fail(CLOAK_EINVAL, "lr must be >= 0");
    if (!h->sur) return fail(CLOAK_ESTATE, "the handle has no surrogate");
    int rc = use_device(h);
    if (rc) return rc;
    std::string why;
    rc = ck::sur_batch_grad(h->sur, dev_x, dev_t, n, stage, lr, host_grad, (cudaStream_t)cuda_stream, why);
    return rc ? fail(rc, "%s", why.c_str()) : CLOAK_OK;
}
