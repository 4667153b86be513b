// surrogate.cu -- the learned surrogate: parameters, BF16 tensor-core training (forward, backward, Adam)
// and inference, and its C ABI.  See surrogate.h for the network.
//
// Training step on a batch of B rays (B a multiple of 128), every GEMM on the tensor cores (mlp_tc.cuh):
//   forward  Z_l = H_{l-1} W_l^T + b_l, H_l = GELU(Z_l)          (H_{-1} = X; the last layer is affine)
//   loss     dY = dL/dY                                           (k_sur_loss)
//   backward dW_l = dZ_l^T H_{l-1}   (split over the batch, FP32 atomics)
//            dZ_{l-1} = (dZ_l W_l) * GELU'(Z_{l-1})                (fused into the GEMM epilogue)
//            db_l = column sums of dZ_l                            (k_sur_rowsum on the transposed copy)
//   update   Adam on the FP32 masters, then their BF16 copies W_l and W_l^T (k_sur_adam)
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cloak.h"
#include "mlp_tc.cuh"
#include "sur_physics.cuh"
#include "surrogate.h"
#include "tc_ptx.cuh"
#include "wavefront.cuh"

namespace ck {

namespace {
__device__ unsigned int g_gemm_err;  // timeout flag of the GEMM kernels launched from this file

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Optimiser schedule kept on the device, so that a captured training step replays unchanged: step
// counter (batch choice and Adam bias corrections) and the learning rate of the current step.
struct SurSched {
    long long step;   // steps taken (this one included, after k_sur_sched_next)
    long long total;  // length of the cosine schedule
    float lr0, floor; // peak rate; the cosine decays to floor * lr0
    int warm;         // linear warm-up steps
    float lr, c1, c2; // this step: rate, 1 - beta1^step, 1 - beta2^step
};

__global__ void k_sur_sched_next(SurSched *sc) {
    const long long k = sc->step;
    sc->step = k + 1;
    const float w = fminf(1.f, (float)(k + 1) / (float)sc->warm);
    const float cs = 0.5f * (1.f + cospif(fminf((float)k / (float)sc->total, 1.f)));
    sc->lr = sc->lr0 * w * (sc->floor + (1.f - sc->floor) * cs);
    sc->c1 = 1.f - powf(0.9f, (float)(k + 1));
    sc->c2 = 1.f - powf(0.999f, (float)(k + 1));
}

// An input enters the first GEMM as a BF16 pair (hi, lo), hi + lo = x to about 16 significant bits, in
// columns j and SUR_IN + j; both columns carry the same weight, so the product is W x without the 8-bit
// rounding of x (a quantisation of the direction angles by up to 2^-8 of pi/2 otherwise).
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// batch rows from the training set: random rows (sc: step counter) or rows i0 .. i0 + B - 1 (sc null)
__global__ void k_sur_gather(const float *X_all, const float *T_all, long long n, unsigned long long seed,
                             const SurSched *sc, int B, long long i0, __nv_bfloat16 *Xb, __nv_bfloat16 *XTb,
                             float *Tb) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    long long idx = !sc ? i0 + b : (long long)(mix64(mix64(seed) ^ (uint64_t)(sc->step * B + b)) % (uint64_t)n);
    if (idx >= n) idx = n - 1;
    const float *x = X_all + idx * SUR_XSTRIDE;
#pragma unroll
    for (int j = 0; j < SUR_IN; ++j) {
        __nv_bfloat16 hi, lo;
        split_bf16(x[j], hi, lo);
        Xb[(size_t)b * 64 + j] = hi;
        Xb[(size_t)b * 64 + SUR_IN + j] = lo;
        XTb[(size_t)j * B + b] = hi;
        XTb[(size_t)(SUR_IN + j) * B + b] = lo;
    }
    const float *t = T_all + idx * SUR_TSTRIDE;
#pragma unroll
    for (int j = 0; j < SUR_TSTRIDE; ++j) Tb[(size_t)b * SUR_TSTRIDE + j] = t[j];
}

// Loss and dL/dY (stage 1: masked weighted squared error of outputs 0..3; stage 2: L1 of the
// confidence output 4), both as means over the batch.
__global__ void k_sur_loss(const float *Y, const float *Tb, int B, int stage, __nv_bfloat16 *dY,
                           __nv_bfloat16 *dYT, double *loss) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    double L = 0.0;
    if (b < B) {
        const float *y = Y + (size_t)b * 16, *t = Tb + (size_t)b * SUR_TSTRIDE;
        const float w[4] = {1.f, 1.f, 1.f, 0.1f}, invB = 1.f / (float)B, mask = t[5];
        float g[SUR_OUT] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (stage == 1) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float e = y[j] - t[j];
                L += (double)(mask * w[j] * e * e * invB);
                g[j] = 2.f * mask * w[j] * e * invB;
            }
        } else {
            const float e = y[4] - t[4];
            L += (double)(fabsf(e) * invB);
            g[4] = (e > 0.f ? 1.f : (e < 0.f ? -1.f : 0.f)) * invB;
        }
#pragma unroll
        for (int j = 0; j < SUR_OUT; ++j) {
            const __nv_bfloat16 v = __float2bfloat16_rn(g[j]);
            dY[(size_t)b * 64 + j] = v;
            dYT[(size_t)j * B + b] = v;
        }
    }
    for (int o = 16; o > 0; o >>= 1) L += __shfl_down_sync(0xffffffffu, L, o);
    if ((threadIdx.x & 31) == 0 && L != 0.0) atomicAdd(loss, L);
}

// out[r] = sum over the columns of row r of a BF16 matrix (bias gradients from a transposed dZ)
// out[i] = sum over the slices s = 0, 1, ... of part[s * n + i], in that order: the weight gradients of the
// batch-split GEMMs, summed the same way on every run (atomic accumulation made training order-dependent)
__global__ void k_sum_slices(const float *part, int slices, long long n, float *out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int k = 0; k < slices; ++k) acc += part[(size_t)k * n + i];
        out[i] = acc;
    }
}

__global__ void k_sur_rowsum(const __nv_bfloat16 *M, int cols, float *out) {
    const __nv_bfloat16 *row = M + (size_t)blockIdx.x * cols;
    float s = 0.f;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) s += __bfloat162float(row[c]);
    __shared__ float part[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) out[blockIdx.x] = s;
    }
}

// One Adam step (beta1 0.9, beta2 0.999, eps 1e-8; rate and bias corrections from the schedule) of
// layer l (weights r < out, c < in, and the bias), then the BF16 copies W (nout x kin) and W^T
// (kin x kb).  One thread per element of the mw x kin grid plus one per bias; sc null: copies only.
// First layer: the weight of input j also multiplies its low part (column SUR_IN + j) and its gradient is
// the sum of both columns'; the entry height and azimuth (inputs 0, 1) keep their weights (zero after
// initialisation: the exit does not depend on them by the symmetry of the media).
__global__ void k_sur_adam(SurDims dm, float *W, float *b, float *mW, float *vW, float *mb, float *vb,
                           const float *gW, const float *gb, __nv_bfloat16 *Wb, __nv_bfloat16 *WTb, __half *Wh,
                           __half *bh, const SurSched *sc) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nW = (long long)dm.mw * dm.kin;
    const bool update = sc != nullptr;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float lr = update ? sc->lr : 0.f, c1 = update ? sc->c1 : 1.f, c2 = update ? sc->c2 : 1.f;
    if (e < nW) {
        const int r = (int)(e / dm.kin), c = (int)(e % dm.kin);
        const bool first = dm.in == SUR_IN;
        if (first && c >= SUR_IN && c < 2 * SUR_IN) return;  // low-part column: written with its input's
        if (update && r < dm.out && c < dm.in && !(first && c < 2)) {
            const float g = first ? gW[e] + gW[e + SUR_IN] : gW[e];
            const float m = b1 * mW[e] + (1.f - b1) * g, v = b2 * vW[e] + (1.f - b2) * g * g;
            mW[e] = m;
            vW[e] = v;
            W[e] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
        }
        const __nv_bfloat16 wb = __float2bfloat16_rn(W[e]);
        const __half wh = __float2half_rn(W[e]);
        if (r < dm.nout) {
            Wb[(size_t)r * dm.kin + c] = wb;
            Wh[(size_t)r * dm.kin + c] = wh;
            if (first && c < SUR_IN) {
                Wb[(size_t)r * dm.kin + SUR_IN + c] = wb;
                Wh[(size_t)r * dm.kin + SUR_IN + c] = wh;
            }
        }
        if (r < dm.kb) WTb[(size_t)c * dm.kb + r] = wb;
    } else if (e < nW + dm.mw) {
        const int r = (int)(e - nW);
        if (update && r < dm.out) {
            const float g = gb[r];
            const float m = b1 * mb[r] + (1.f - b1) * g, v = b2 * vb[r] + (1.f - b2) * g * g;
            mb[r] = m;
            vb[r] = v;
            b[r] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
        }
        bh[r] = __float2half_rn(b[r]);
    }
}

// FP32 inputs (n x 7) into the padded input rows of the inference scratch as (hi, lo) pairs, BF16 or FP16
__global__ void k_sur_pack(const float *x, long long n, uint16_t *X, int f16) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int j = 0; j < SUR_IN; ++j) sur_split_pair(x[i * SUR_IN + j], f16, X + (size_t)i * 64 + j, X + (size_t)i * 64 + SUR_IN + j);
}
__global__ void k_sur_unpack(const float *Y, long long n, float *y) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int j = 0; j < SUR_OUT; ++j) y[i * SUR_OUT + j] = Y[(size_t)i * 16 + j];
}
// FP32 targets (n x 8) into the batch target buffer, and FP32 inputs into the batch input buffers
__global__ void k_sur_pack_batch(const float *x, const float *t, int B, __nv_bfloat16 *Xb, __nv_bfloat16 *XTb,
                                 float *Tb) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
#pragma unroll
    for (int j = 0; j < SUR_IN; ++j) {
        __nv_bfloat16 hi, lo;
        split_bf16(x[(size_t)b * SUR_IN + j], hi, lo);
        Xb[(size_t)b * 64 + j] = hi;
        Xb[(size_t)b * 64 + SUR_IN + j] = lo;
        XTb[(size_t)j * B + b] = hi;
        XTb[(size_t)(SUR_IN + j) * B + b] = lo;
    }
#pragma unroll
    for (int j = 0; j < SUR_TSTRIDE; ++j) Tb[(size_t)b * SUR_TSTRIDE + j] = t[(size_t)b * SUR_TSTRIDE + j];
}
}  // namespace

// ------------------------------------------------------------------ host helpers
static uint64_t host_mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double host_uniform(uint64_t seed, uint64_t i) {
    return (double)(host_mix64(host_mix64(seed) ^ i) >> 11) * 0x1.0p-53;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static cudaError_t gemm(const CUtensorMap &ta, const CUtensorMap &tb, GemmArgs g, cudaStream_t st) {
    return launch_gemm_tc(ta, tb, g, st);
}
// Polls of the tensor-core kernels' waits that decide a timeout (process-wide; cloak_set_wait_limit).
static std::atomic<unsigned int> g_wait_limit{MBAR_DEFAULT_LIMIT};
unsigned int wait_limit() { return g_wait_limit.load(); }
void set_wait_limit(unsigned int polls) { g_wait_limit.store(polls ? polls : MBAR_DEFAULT_LIMIT); }

static GemmArgs gemm_args(int M, int N, int K, int epi, unsigned int *err) {
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.M = M; g.N = N; g.K = K; g.ksplit = 1; g.epi = epi; g.err = err;
    g.wait_limit = wait_limit();
    return g;
}
static bool tmap(CUtensorMap *m, const void *base, long long rows, int cols, int box_rows) {
    return make_tmap_bf16(m, base, (int)rows, cols, box_rows) == CUDA_SUCCESS;
}

SurNet *sur_create(double R1, double R2, double H, unsigned long long seed, const char **why) {
    SurNet *s = new SurNet();
    memset(s, 0, sizeof(*s));
    s->R1 = R1; s->R2 = R2; s->H = H;
    s->gate = -3.0f;
    size_t bytes = 0;
    for (int l = 0; l < SUR_L; ++l) {
        SurDims d = sur_dims(l);
        const size_t w = align256((size_t)d.mw * d.kin * 4), bb = align256((size_t)d.mw * 4);
        bytes += 4 * w + 4 * bb;                                        // W, mW, vW, gW ; b, mb, vb, gb
        bytes += align256((size_t)d.nout * d.kin * 2) + align256((size_t)d.kin * d.kb * 2);
        bytes += align256((size_t)d.nout * d.kin * 2) + align256((size_t)d.mw * 2);  // Wh, bh
    }
    bytes += 256;  // error flag
    cudaError_t e = cudaMalloc(&s->arena, bytes);
    if (e != cudaSuccess) {
        *why = "cannot allocate the surrogate's parameters";
        delete s;
        return nullptr;
    }
    // zeroed before any stream uses it: cudaMemset runs on the legacy default stream, which the library's
    // non-blocking streams do not wait for
    if (cudaMemset(s->arena, 0, bytes) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        *why = "cannot clear the surrogate's parameters";
        cudaFree(s->arena);
        delete s;
        return nullptr;
    }
    char *p = s->arena;
    // gradients first, contiguous (zeroed before every step)
    s->grad_begin = p;
    for (int l = 0; l < SUR_L; ++l) {
        SurDims d = sur_dims(l);
        s->gW[l] = (float *)p; p += align256((size_t)d.mw * d.kin * 4);
        s->gb[l] = (float *)p; p += align256((size_t)d.mw * 4);
    }
    s->grad_bytes = (size_t)(p - s->grad_begin);
    for (int l = 0; l < SUR_L; ++l) {
        SurDims d = sur_dims(l);
        const size_t w = align256((size_t)d.mw * d.kin * 4), bb = align256((size_t)d.mw * 4);
        s->W[l] = (float *)p; p += w;
        s->mW[l] = (float *)p; p += w;
        s->vW[l] = (float *)p; p += w;
        s->b[l] = (float *)p; p += bb;
        s->mb[l] = (float *)p; p += bb;
        s->vb[l] = (float *)p; p += bb;
        s->Wb[l] = (__nv_bfloat16 *)p; p += align256((size_t)d.nout * d.kin * 2);
        s->WTb[l] = (__nv_bfloat16 *)p; p += align256((size_t)d.kin * d.kb * 2);
        s->Wh[l] = (__half *)p; p += align256((size_t)d.nout * d.kin * 2);
        s->bh[l] = (__half *)p; p += align256((size_t)d.mw * 2);
        if (!tmap(&s->tWb[l], s->Wb[l], d.nout, d.kin, d.nout) || !tmap(&s->tWTb[l], s->WTb[l], d.kin, d.kb, d.kin) ||
            make_tmap_f16(&s->tWh[l], s->Wh[l], d.nout, d.kin, d.nout) != CUDA_SUCCESS) {
            *why = "cannot encode the weight tensor maps";
            cudaFree(s->arena);
            delete s;
            return nullptr;
        }
    }
    s->err = (unsigned int *)p;
    // initial weights: normal with variance 1/in (Box-Muller on splitmix64 uniforms), last layer x 0.1
    std::vector<float> host;
    for (int l = 0; l < SUR_L; ++l) {
        SurDims d = sur_dims(l);
        host.assign((size_t)d.mw * d.kin, 0.f);
        const double sd = (l == SUR_L - 1 ? 0.1 : 1.0) / std::sqrt((double)d.in);
        for (int r = 0; r < d.out; ++r)
            for (int c = (l == 0 ? 2 : 0); c < d.in; ++c) {
                const uint64_t k = ((uint64_t)l << 40) ^ ((uint64_t)r << 20) ^ (uint64_t)c;
                const double u1 = host_uniform(seed, 2 * k) + 0x1.0p-54, u2 = host_uniform(seed, 2 * k + 1);
                host[(size_t)r * d.kin + c] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2));
            }
        cudaMemcpy(s->W[l], host.data(), host.size() * 4, cudaMemcpyHostToDevice);
    }
    if (sur_refresh_bf16(s, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        *why = "cannot initialise the surrogate's weights";
        cudaFree(s->arena);
        delete s;
        return nullptr;
    }
    return s;
}

void sur_destroy(SurNet *s) {
    if (!s) return;
    if (s->inf_arena) cudaFree(s->inf_arena);
    if (s->arena) cudaFree(s->arena);
    delete s;
}

static cudaError_t adam_all(SurNet *s, const SurSched *sc, int first_layer, cudaStream_t st) {
    for (int l = first_layer; l < SUR_L; ++l) {
        SurDims d = sur_dims(l);
        const long long n = (long long)d.mw * d.kin + d.mw;
        k_sur_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, s->W[l], s->b[l], s->mW[l], s->vW[l], s->mb[l],
                                                               s->vb[l], s->gW[l], s->gb[l], s->Wb[l], s->WTb[l],
                                                               s->Wh[l], s->bh[l], sc);
    }
    return cudaGetLastError();
}

cudaError_t sur_refresh_bf16(SurNet *s, cudaStream_t st) { return adam_all(s, nullptr, 0, st); }

cudaError_t sur_ensure_inference(SurNet *s, long long rows) {
    rows = (rows + 127) / 128 * 128;
    if (rows <= s->inf_rows) return cudaSuccess;
    if (s->inf_arena) {
        cudaFree(s->inf_arena);
        s->inf_arena = nullptr;
        s->inf_rows = 0;
    }
    const size_t xb = align256((size_t)rows * 64 * 2), yb = align256((size_t)rows * 16 * 4), eb = align256((size_t)rows);
    cudaError_t e = cudaMalloc(&s->inf_arena, xb + yb + eb);
    if (e != cudaSuccess) return e;
    char *p = s->inf_arena;
    s->X = (uint16_t *)p; p += xb;
    s->Y = (float *)p; p += yb;
    s->elig = (unsigned char *)p;
    // columns 14..63 stay zero; cleared before any stream uses the buffer (cudaMemset runs on the legacy default
    // stream, which the library's non-blocking streams do not wait for)
    if ((e = cudaMemset(s->X, 0, xb)) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    s->inf_rows = rows;
    return cudaSuccess;
}

cudaError_t sur_forward(SurNet *s, long long n, const unsigned int *m_count, cudaStream_t st) {
    return launch_mlp_fused(s, n, m_count, st);
}

// ------------------------------------------------------------------ training workspace
struct TrainWS {
    int B;
    char *arena;
    __nv_bfloat16 *Xb, *XTb, *H[4], *HT[4], *dY, *dYT, *dZ[2], *dZT[2];
    float *Tb, *Z[4], *Y;
    double *loss;
    SurSched *sched;
    float *partials;  // per-slice partial weight gradients (k_sum_slices)
    CUtensorMap tXb, tXTb, tH[4], tHT[4], tdY, tdYT, tdZ[2], tdZT[2];
};

static int ksplit_for(int B, int mtiles);
static cudaError_t ws_create(TrainWS &w, int B, cudaStream_t st) {
    memset(&w, 0, sizeof(w));
    w.B = B;
    size_t part = 0;  // the largest per-slice partial gradients of a layer
    for (int l = 0; l < SUR_L; ++l) {
        const SurDims d = sur_dims(l);
        part = std::max(part, (size_t)ksplit_for(B, d.mw / GEMM_TILE_M) * d.mw * d.kin * 4);
    }
    part = align256(part);
    const size_t x = align256((size_t)B * 64 * 2), z = align256((size_t)B * SUR_W * 4),
                 h = align256((size_t)B * SUR_W * 2), t = align256((size_t)B * SUR_TSTRIDE * 4),
                 y = align256((size_t)B * 16 * 4), dyt = align256((size_t)128 * B * 2);
    const size_t bytes = 2 * x + t + 4 * z + 8 * h + y + x + dyt + 4 * h + 512 + part;
    cudaError_t e = cudaMalloc(&w.arena, bytes);
    if (e != cudaSuccess) return e;
    // cleared on the stream that uses it (a cudaMemset on the legacy default stream can still be running
    // when the first kernels of a non-blocking stream start)
    if ((e = cudaMemsetAsync(w.arena, 0, bytes, st)) != cudaSuccess) return e;
    char *p = w.arena;
    w.Xb = (__nv_bfloat16 *)p; p += x;
    w.XTb = (__nv_bfloat16 *)p; p += x;
    w.Tb = (float *)p; p += t;
    for (int l = 0; l < 4; ++l) { w.Z[l] = (float *)p; p += z; }
    for (int l = 0; l < 4; ++l) { w.H[l] = (__nv_bfloat16 *)p; p += h; }
    for (int l = 0; l < 4; ++l) { w.HT[l] = (__nv_bfloat16 *)p; p += h; }
    w.Y = (float *)p; p += y;
    w.dY = (__nv_bfloat16 *)p; p += x;
    w.dYT = (__nv_bfloat16 *)p; p += dyt;
    for (int j = 0; j < 2; ++j) { w.dZ[j] = (__nv_bfloat16 *)p; p += h; }
    for (int j = 0; j < 2; ++j) { w.dZT[j] = (__nv_bfloat16 *)p; p += h; }
    w.loss = (double *)p;
    w.sched = (SurSched *)(p + 256);
    w.partials = (float *)(p + 512);
    bool ok = tmap(&w.tXb, w.Xb, B, 64, GEMM_TILE_M) && tmap(&w.tXTb, w.XTb, 64, B, 64) &&
              tmap(&w.tdY, w.dY, B, 64, GEMM_TILE_M) && tmap(&w.tdYT, w.dYT, 128, B, GEMM_TILE_M);
    for (int l = 0; l < 4; ++l)
        ok = ok && tmap(&w.tH[l], w.H[l], B, SUR_W, GEMM_TILE_M) && tmap(&w.tHT[l], w.HT[l], SUR_W, B, SUR_W);
    for (int j = 0; j < 2; ++j)
        ok = ok && tmap(&w.tdZ[j], w.dZ[j], B, SUR_W, GEMM_TILE_M) && tmap(&w.tdZT[j], w.dZT[j], SUR_W, B, GEMM_TILE_M);
    return ok ? cudaSuccess : cudaErrorInvalidValue;
}
static void ws_destroy(TrainWS &w) {
    if (w.arena) cudaFree(w.arena);
    w.arena = nullptr;
}

// split of the batch dimension for the weight-gradient GEMMs: about one CTA per SM
static int ksplit_for(int B, int mtiles) {
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int chunks = B / GEMM_KCHUNK;
    int best = 1;
    for (int k = 1; k <= chunks; ++k)
        if (chunks % k == 0 && k * mtiles <= sms) best = k;
    return best;
}

static cudaError_t train_forward(SurNet *s, TrainWS &w, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < SUR_L && e == cudaSuccess; ++l) {
        SurDims d = sur_dims(l);
        const CUtensorMap &ta = l == 0 ? w.tXb : w.tH[l - 1];
        GemmArgs g = gemm_args(w.B, d.nout, d.kin, l < SUR_L - 1 ? EPI_BIAS_GELU : EPI_BIAS, s->err);
        g.bias = s->b[l];
        if (l < SUR_L - 1) {
            g.Z = w.Z[l]; g.ldz = SUR_W;
            g.H = w.H[l]; g.ldh = SUR_W;
            g.HT = w.HT[l]; g.ldht = w.B;
        } else {
            g.Z = w.Y; g.ldz = 16;
        }
        e = gemm(ta, s->tWb[l], g, st);
    }
    return e;
}

// dW = dZ^T H over the batch: the batch is split into K slices (about one CTA per SM), each slice stores
// its partial product, and the slices are summed in a fixed order
static cudaError_t weight_grad(SurNet *s, TrainWS &w, const SurDims &d, const CUtensorMap &tdz, const CUtensorMap &th,
                               float *gW, cudaStream_t st) {
    GemmArgs g = gemm_args(d.mw, d.kin, w.B, EPI_STORE, s->err);
    g.ksplit = ksplit_for(w.B, d.mw / GEMM_TILE_M);
    g.C = w.partials;
    g.ldc = d.kin;
    g.slice_stride = (long long)d.mw * d.kin;
    cudaError_t e = gemm(tdz, th, g, st);
    if (e != cudaSuccess) return e;
    const long long n = (long long)d.mw * d.kin;
    k_sum_slices<<<(unsigned)std::min<long long>((n + 255) / 256, 1184), 256, 0, st>>>(w.partials, g.ksplit, n, gW);
    return cudaGetLastError();
}

// gradients of the loss of the batch in w (after train_forward and k_sur_loss); layers >= first only
static cudaError_t train_backward(SurNet *s, TrainWS &w, int first, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(s->grad_begin, 0, s->grad_bytes, st);
    const int B = w.B;
    // output layer
    {
        SurDims d = sur_dims(SUR_L - 1);
        if (e == cudaSuccess) e = weight_grad(s, w, d, w.tdYT, w.tHT[SUR_L - 2], s->gW[SUR_L - 1], st);
        k_sur_rowsum<<<d.out, 256, 0, st>>>(w.dYT, B, s->gb[SUR_L - 1]);
    }
    int cur = 0;
    for (int l = SUR_L - 1; l > first && e == cudaSuccess; --l) {
        // dZ_{l-1} = (dZ_l W_l) * GELU'(Z_{l-1})
        SurDims d = sur_dims(l), dp = sur_dims(l - 1);
        const CUtensorMap &ta = l == SUR_L - 1 ? w.tdY : w.tdZ[cur ^ 1];
        GemmArgs g = gemm_args(B, d.kin, d.kb, EPI_GELU_BWD, s->err);
        g.Z = w.Z[l - 1]; g.ldz = SUR_W;
        g.H = w.dZ[cur]; g.ldh = SUR_W;
        g.HT = w.dZT[cur]; g.ldht = B;
        e = gemm(ta, s->tWTb[l], g, st);
        if (e != cudaSuccess) break;
        // dW_{l-1} = dZ_{l-1}^T H_{l-2}, db_{l-1} = column sums of dZ_{l-1}
        const CUtensorMap &tb = l - 1 == 0 ? w.tXTb : w.tHT[l - 2];
        e = weight_grad(s, w, dp, w.tdZT[cur], tb, s->gW[l - 1], st);
        k_sur_rowsum<<<dp.out, 256, 0, st>>>(w.dZT[cur], B, s->gb[l - 1]);
        cur ^= 1;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

// One optimiser step on the batch already in w (schedule advanced by k_sur_sched_next first).
static cudaError_t train_step(SurNet *s, TrainWS &w, int stage, cudaStream_t st) {
    cudaError_t e = train_forward(s, w, st);
    if (e != cudaSuccess) return e;
    k_sur_loss<<<(w.B + 255) / 256, 256, 0, st>>>(w.Y, w.Tb, w.B, stage, w.dY, w.dYT, w.loss);
    e = train_backward(s, w, stage == 1 ? 0 : SUR_L - 1, st);
    if (e != cudaSuccess) return e;
    return adam_all(s, w.sched, stage == 1 ? 0 : SUR_L - 1, st);
}

static cudaError_t sched_init(TrainWS &w, long long step0, long long total, float lr0, float floor, int warm,
                              cudaStream_t st) {
    SurSched h;
    memset(&h, 0, sizeof(h));
    h.step = step0; h.total = total > 0 ? total : 1; h.lr0 = lr0; h.floor = floor; h.warm = warm > 0 ? warm : 1;
    cudaError_t e = cudaMemcpyAsync(w.sched, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
}

// `steps` optimiser steps on random batches of the training set: the first eagerly, the rest as
// replays of a captured CUDA graph of one step (schedule, batch, forward, loss, backward, Adam).  The
// loss accumulator is cleared before the last `tail` steps.
static cudaError_t run_steps(SurNet *s, TrainWS &w, int stage, long long steps, long long tail, const float *X_all,
                             const float *T_all, long long n, unsigned long long seed, cudaStream_t st) {
    const int B = w.B;
    auto one = [&](cudaStream_t cs) -> cudaError_t {
        k_sur_sched_next<<<1, 1, 0, cs>>>(w.sched);
        k_sur_gather<<<(B + 255) / 256, 256, 0, cs>>>(X_all, T_all, n, seed, w.sched, B, 0, w.Xb, w.XTb, w.Tb);
        return train_step(s, w, stage, cs);
    };
    if (steps <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(w.loss, 0, 8, st);
    if (e == cudaSuccess && steps <= tail) e = cudaMemsetAsync(w.loss, 0, 8, st);
    if (e == cudaSuccess) e = one(st);  // eager: sets the kernels' attributes outside any capture
    if (e != cudaSuccess || steps == 1) return e;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    cudaError_t ec = one(st);
    e = cudaStreamEndCapture(st, &g);
    if (ec != cudaSuccess) e = ec;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    for (long long k = 1; k < steps && e == cudaSuccess; ++k) {
        if (steps - k == tail) e = cudaMemsetAsync(w.loss, 0, 8, st);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, st);
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    return e;
}

static cudaError_t d2h(void *dst, const void *src, size_t bytes, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
    return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
}

static unsigned int *gemm_err_flag() {
    unsigned int *p = nullptr;
    cudaGetSymbolAddress((void **)&p, g_gemm_err);
    return p;
}

}  // namespace ck

// ------------------------------------------------------------------ C ABI building block
extern "C" int cloak_mlp_gemm(const void *dev_a, const void *dev_b, float *dev_c, int M, int N, int K,
                              void *cuda_stream) {
    if (!dev_a || !dev_b || !dev_c) return CLOAK_EINVAL;
    if (M <= 0 || M % 128 || N < 16 || N > 256 || N % 16 || K <= 0 || K % 64) return CLOAK_EINVAL;
    if (((uintptr_t)dev_a | (uintptr_t)dev_b) & 15) return CLOAK_EINVAL;
    CUtensorMap ta, tb;
    if (ck::make_tmap_bf16(&ta, dev_a, M, K, ck::GEMM_TILE_M) != CUDA_SUCCESS) return CLOAK_ECUDA;
    if (ck::make_tmap_bf16(&tb, dev_b, N, K, N) != CUDA_SUCCESS) return CLOAK_ECUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned int *err = ck::gemm_err_flag();
    if (!err) return CLOAK_ECUDA;
    if (cudaMemsetAsync(err, 0, sizeof(unsigned int), st) != cudaSuccess) return CLOAK_ECUDA;
    ck::GemmArgs g = ck::gemm_args(M, N, K, ck::EPI_STORE, err);
    g.C = dev_c;
    g.ldc = N;
    if (ck::launch_gemm_tc(ta, tb, g, st) != cudaSuccess) return CLOAK_ECUDA;
    unsigned int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CLOAK_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CLOAK_ECUDA;
    return h ? CLOAK_ETIMEOUT : CLOAK_OK;
}

// ------------------------------------------------------------------ surrogate entry points (called by capi.cu)
namespace ck {

// layout of the flat FP32 parameter vector of the C ABI: per layer W_l (out x in, row-major), then b_l
long long sur_nparams() {
    long long n = 0;
    for (int l = 0; l < SUR_L; ++l) {
        SurDims d = sur_dims(l);
        n += (long long)d.out * d.in + d.out;
    }
    return n;
}

cudaError_t sur_get_params(SurNet *s, float *host) {
    cudaError_t e0 = cudaDeviceSynchronize();
    if (e0 != cudaSuccess) return e0;
    std::vector<float> buf;
    long long o = 0;
    for (int l = 0; l < SUR_L; ++l) {
        SurDims d = sur_dims(l);
        buf.resize((size_t)d.mw * d.kin);
        cudaError_t e = cudaMemcpy(buf.data(), s->W[l], buf.size() * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        for (int r = 0; r < d.out; ++r)
            for (int c = 0; c < d.in; ++c) host[o++] = buf[(size_t)r * d.kin + c];
        e = cudaMemcpy(host + o, s->b[l], (size_t)d.out * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        o += d.out;
    }
    return cudaSuccess;
}

cudaError_t sur_set_params(SurNet *s, const float *host) {
    cudaError_t e0 = cudaDeviceSynchronize();
    if (e0 != cudaSuccess) return e0;
    std::vector<float> buf;
    long long o = 0;
    for (int l = 0; l < SUR_L; ++l) {
        SurDims d = sur_dims(l);
        buf.assign((size_t)d.mw * d.kin, 0.f);
        for (int r = 0; r < d.out; ++r)
            for (int c = 0; c < d.in; ++c) buf[(size_t)r * d.kin + c] = host[o++];
        cudaError_t e = cudaMemcpy(s->W[l], buf.data(), buf.size() * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        std::vector<float> bb((size_t)d.mw, 0.f);
        for (int r = 0; r < d.out; ++r) bb[r] = host[o++];
        if ((e = cudaMemcpy(s->b[l], bb.data(), bb.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        const size_t wb = (size_t)d.mw * d.kin * 4, bbytes = (size_t)d.mw * 4;
        if ((e = cudaMemset(s->mW[l], 0, wb)) != cudaSuccess || (e = cudaMemset(s->vW[l], 0, wb)) != cudaSuccess ||
            (e = cudaMemset(s->mb[l], 0, bbytes)) != cudaSuccess || (e = cudaMemset(s->vb[l], 0, bbytes)) != cudaSuccess)
            return e;
    }
    s->adam_step = 0;
    cudaError_t e = sur_refresh_bf16(s, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e;
}

// forward pass of n FP32 input rows (n x 7) into FP32 outputs (n x 5)
int sur_forward_rows(SurNet *s, const float *dev_x, long long n, float *dev_y, cudaStream_t st, std::string &why) {
    cudaError_t e = sur_ensure_inference(s, n);
    if (e != cudaSuccess) { why = "cannot allocate the inference scratch"; return CLOAK_ENOMEM; }
    const long long rows = (n + 127) / 128 * 128;
    unsigned int *err = s->err;  // this network's own timeout flag
    cudaMemsetAsync(err, 0, 4, st);
    k_sur_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dev_x, n, s->X, s->inf_f16);
    if ((e = sur_forward(s, rows, nullptr, st)) != cudaSuccess) { why = cudaGetErrorString(e); return CLOAK_ECUDA; }
    k_sur_unpack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->Y, n, dev_y);
    unsigned int h = 0;
    cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { why = cudaGetErrorString(e); return CLOAK_ECUDA; }
    if (h) { why = "tensor-core GEMM timed out"; return CLOAK_ETIMEOUT; }
    return CLOAK_OK;
}

// gradients (host, flat layout) of one batch, and optionally one Adam step with learning rate lr
int sur_batch_grad(SurNet *s, const float *dev_x, const float *dev_t, long long n, int stage, double lr,
                   float *host_grad, cudaStream_t st, std::string &why) {
    TrainWS w;
    cudaError_t e = ws_create(w, (int)n, st);
    if (e != cudaSuccess) { ws_destroy(w); why = "cannot allocate the training workspace"; return CLOAK_ENOMEM; }
    unsigned int *err = s->err;  // this network's own timeout flag
    cudaMemsetAsync(err, 0, 4, st);
    cudaMemsetAsync(w.loss, 0, 8, st);
    k_sur_pack_batch<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dev_x, dev_t, (int)n, w.Xb, w.XTb, w.Tb);
    if (lr > 0) {
        // a constant rate: warm-up of one step, floor 1
        e = sched_init(w, s->adam_step, 1, (float)lr, 1.f, 1, st);
        if (e == cudaSuccess) {
            k_sur_sched_next<<<1, 1, 0, st>>>(w.sched);
            e = train_step(s, w, stage, st);
        }
        s->adam_step++;
    } else {
        e = train_forward(s, w, st);
        if (e == cudaSuccess) {
            k_sur_loss<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w.Y, w.Tb, (int)n, stage, w.dY, w.dYT, w.loss);
            e = train_backward(s, w, 0, st);
        }
    }
    unsigned int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && host_grad) {
        std::vector<float> buf;
        long long o = 0;
        for (int l = 0; l < SUR_L && e == cudaSuccess; ++l) {
            SurDims d = sur_dims(l);
            buf.resize((size_t)d.mw * d.kin);
            e = cudaMemcpy(buf.data(), s->gW[l], buf.size() * 4, cudaMemcpyDeviceToHost);
            for (int r = 0; r < d.out; ++r)
                for (int c = 0; c < d.in; ++c)
                    host_grad[o++] = buf[(size_t)r * d.kin + c] + (l == 0 ? buf[(size_t)r * d.kin + SUR_IN + c] : 0.f);
            if (e == cudaSuccess) e = cudaMemcpy(host_grad + o, s->gb[l], (size_t)d.out * 4, cudaMemcpyDeviceToHost);
            o += d.out;
        }
    }
    ws_destroy(w);
    if (e != cudaSuccess) { why = cudaGetErrorString(e); return CLOAK_ECUDA; }
    if (h) { why = "tensor-core GEMM timed out"; return CLOAK_ETIMEOUT; }
    return CLOAK_OK;
}

// Train on n rays traced by the integrator (parameters p: geometry, integrator, precision).
int sur_train(SurNet *s, const Params &p, long long n, unsigned long long seed, int epochs, cudaStream_t caller,
              std::string &why) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    const int B = 19456;  // 152 x 128: one 128-row tile per SM in the forward GEMMs
    cudaError_t e = cudaStreamSynchronize(caller);
    if (e != cudaSuccess) { why = cudaGetErrorString(e); return CLOAK_ECUDA; }
    cudaStream_t st = nullptr;  // private stream: graph capture is not possible on the legacy default stream
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
        why = cudaGetErrorString(e);
        return CLOAK_ECUDA;
    }
    // 1. training set: the integrator traces n seeded rays
    const size_t qb = queue_bytes(n), xb = (size_t)n * SUR_XSTRIDE * 4, tb = (size_t)n * SUR_TSTRIDE * 4;
    char *data = nullptr;
    e = cudaMalloc(&data, qb + xb + tb);
    if (e != cudaSuccess) {
        cudaStreamDestroy(st);
        why = "cannot allocate the training set";
        return CLOAK_ENOMEM;
    }
    Queue q;
    float4 *unused = nullptr;
    carve_queue(data, n, q, &unused);
    float *X_all = (float *)(data + qb), *T_all = (float *)(data + qb + xb);
    e = launch_sur_data(p, n, seed, q, X_all, T_all, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const auto t1 = clk::now();
    // fraction of lateral exits (the surrogate's support)
    double lateral = 0.0;
    if (e == cudaSuccess) {
        std::vector<float> T((size_t)std::min<long long>(n, 1 << 20) * SUR_TSTRIDE);
        e = d2h(T.data(), T_all, T.size() * 4, st);
        for (size_t i = 0; i < T.size() / SUR_TSTRIDE; ++i) lateral += T[i * SUR_TSTRIDE + 5];
        lateral /= (double)(T.size() / SUR_TSTRIDE);
    }
    TrainWS w;
    memset(&w, 0, sizeof(w));
    if (e == cudaSuccess) e = ws_create(w, B, st);
    unsigned int *err = s->err;  // this network's own timeout flag
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, st);
    // 2. stage 1: regression outputs, Adam, linear warm-up then cosine decay to 2 % of the peak rate
    const long long steps_per_epoch = std::max<long long>(1, n / B);
    const long long total1 = steps_per_epoch * std::max(epochs, 1);
    double loss1 = 0.0, loss2 = 0.0, acc = 0.0;
    if (e == cudaSuccess) e = sched_init(w, 0, total1, 2e-3f, 0.02f, 200, st);
    // device time of the optimizer steps of each stage (CUDA events around the replayed step graphs)
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = run_steps(s, w, 1, total1, steps_per_epoch, X_all, T_all, n, seed ^ 0x7261696eull, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = d2h(&acc, w.loss, 8, st);
    loss1 = acc / (double)std::min(steps_per_epoch, total1);
    // 3. confidence targets: the exit error of the trained regression on every training ray
    for (long long i0 = 0; i0 < n && e == cudaSuccess; i0 += B) {
        k_sur_gather<<<(B + 255) / 256, 256, 0, st>>>(X_all, T_all, n, 0, nullptr, B, i0, w.Xb, w.XTb, w.Tb);
        e = train_forward(s, w, st);
        if (e == cudaSuccess) e = launch_sur_conf_targets(p.R2, p.H, seed, i0, std::min<long long>(B, n - i0), w.Y, T_all, st);
    }
    // 4. stage 2: the confidence head alone (output layer, fresh Adam moments), L1 loss
    if (e == cudaSuccess) {
        SurDims d = sur_dims(SUR_L - 1);
        cudaMemsetAsync(s->mW[SUR_L - 1], 0, (size_t)d.mw * d.kin * 4, st);
        cudaMemsetAsync(s->vW[SUR_L - 1], 0, (size_t)d.mw * d.kin * 4, st);
        cudaMemsetAsync(s->mb[SUR_L - 1], 0, (size_t)d.mw * 4, st);
        cudaMemsetAsync(s->vb[SUR_L - 1], 0, (size_t)d.mw * 4, st);
    }
    const long long total2 = steps_per_epoch * std::max(1, epochs / 3);
    if (e == cudaSuccess) e = sched_init(w, 0, total2, 1e-3f, 0.f, 1, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], st);
    if (e == cudaSuccess) e = run_steps(s, w, 2, total2, steps_per_epoch, X_all, T_all, n, seed ^ 0x636f6e66ull, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
    float ms1 = 0.f, ms2 = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms1, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms2, ev[2], ev[3]);
    for (int i = 0; i < 4; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    acc = 0.0;
    if (e == cudaSuccess) e = d2h(&acc, w.loss, 8, st);
    loss2 = acc / (double)std::min(steps_per_epoch, total2);
    unsigned int h = 0;
    if (e == cudaSuccess) e = d2h(&h, err, 4, st);
    ws_destroy(w);
    cudaFree(data);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) { why = cudaGetErrorString(e); return CLOAK_ECUDA; }
    if (h) { why = "tensor-core GEMM timed out"; return CLOAK_ETIMEOUT; }
    const auto t2 = clk::now();
    s->trained = 1;
    s->adam_step = total2;
    s->info[0] = loss1;
    s->info[1] = loss2;
    s->info[2] = lateral;
    s->info[3] = (double)n;
    s->info[4] = std::chrono::duration<double>(t2 - t0).count();
    s->info[5] = std::chrono::duration<double>(t1 - t0).count();
    s->info[6] = (double)(total1 + total2);
    s->info[7] = (double)B;
    s->train_ms[0] = total1 > 0 ? ms1 / (double)total1 : 0.0;
    s->train_ms[1] = total2 > 0 ? ms2 / (double)total2 : 0.0;
    return CLOAK_OK;
}

// ------------------------------------------------------------------ checkpoint: flat binary with a header
struct SurFileHeader {
    char magic[8];       // "CKSURR01"
    int version, layers;
    int dims[SUR_L + 1];
    double R1, R2, H;
    float gate;
    int trained;
    long long adam_step;
    double info[8];
};

int sur_save(SurNet *s, const char *path, std::string &why) {
    SurFileHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "CKSURR01", 8);
    hd.version = 1;
    hd.layers = SUR_L;
    for (int l = 0; l < SUR_L; ++l) hd.dims[l] = sur_dims(l).in;
    hd.dims[SUR_L] = SUR_OUT;
    hd.R1 = s->R1; hd.R2 = s->R2; hd.H = s->H;
    hd.gate = s->gate;
    hd.trained = s->trained;
    hd.adam_step = s->adam_step;
    memcpy(hd.info, s->info, sizeof(hd.info));
    FILE *f = fopen(path, "wb");
    if (!f) { why = std::string("cannot open ") + path; return CLOAK_EINVAL; }
    bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1;
    std::vector<float> buf;
    for (int l = 0; l < SUR_L && ok; ++l) {
        SurDims d = sur_dims(l);
        const size_t nw = (size_t)d.mw * d.kin, nb = (size_t)d.mw;
        float *arrs[6] = {s->W[l], s->mW[l], s->vW[l], s->b[l], s->mb[l], s->vb[l]};
        size_t sizes[6] = {nw, nw, nw, nb, nb, nb};
        for (int a = 0; a < 6 && ok; ++a) {
            buf.resize(sizes[a]);
            ok = cudaMemcpy(buf.data(), arrs[a], sizes[a] * 4, cudaMemcpyDeviceToHost) == cudaSuccess &&
                 fwrite(buf.data(), 4, sizes[a], f) == sizes[a];
        }
    }
    ok = (fclose(f) == 0) && ok;
    if (!ok) { why = std::string("cannot write ") + path; return CLOAK_ECUDA; }
    return CLOAK_OK;
}

int sur_load(SurNet *s, const char *path, std::string &why) {
    FILE *f = fopen(path, "rb");
    if (!f) { why = std::string("cannot open ") + path; return CLOAK_EINVAL; }
    SurFileHeader hd;
    bool ok = fread(&hd, sizeof(hd), 1, f) == 1 && memcmp(hd.magic, "CKSURR01", 8) == 0 && hd.version == 1 &&
              hd.layers == SUR_L;
    for (int l = 0; l < SUR_L && ok; ++l) ok = hd.dims[l] == sur_dims(l).in;
    ok = ok && hd.dims[SUR_L] == SUR_OUT;
    if (!ok) { fclose(f); why = "not a surrogate checkpoint of this network"; return CLOAK_EINVAL; }
    std::vector<float> buf;
    for (int l = 0; l < SUR_L && ok; ++l) {
        SurDims d = sur_dims(l);
        const size_t nw = (size_t)d.mw * d.kin, nb = (size_t)d.mw;
        float *arrs[6] = {s->W[l], s->mW[l], s->vW[l], s->b[l], s->mb[l], s->vb[l]};
        size_t sizes[6] = {nw, nw, nw, nb, nb, nb};
        for (int a = 0; a < 6 && ok; ++a) {
            buf.resize(sizes[a]);
            ok = fread(buf.data(), 4, sizes[a], f) == sizes[a] &&
                 cudaMemcpy(arrs[a], buf.data(), sizes[a] * 4, cudaMemcpyHostToDevice) == cudaSuccess;
        }
    }
    fclose(f);
    if (!ok) { why = std::string("truncated checkpoint ") + path; return CLOAK_EINVAL; }
    s->R1 = hd.R1; s->R2 = hd.R2; s->H = hd.H;
    s->gate = hd.gate;
    s->trained = hd.trained;
    s->adam_step = hd.adam_step;
    memcpy(s->info, hd.info, sizeof(hd.info));
    cudaError_t e = sur_refresh_bf16(s, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { why = cudaGetErrorString(e); return CLOAK_ECUDA; }
    return CLOAK_OK;
}

// render hook: features of the queued rays, inference, gate

cudaError_t sur_render_hook(void *ctx, const Queue &q, cudaStream_t st) {
    SurRenderCtx *c = (SurRenderCtx *)ctx;
    SurNet *s = c->s;
    cudaError_t e = sur_ensure_inference(s, c->cap);
    if (e != cudaSuccess) return e;
    // The network's timeout flag is cleared before its forward pass and read by the gate: if a bounded wait
    // of the tensor-core kernel ran out, its outputs are incomplete and the gate leaves every ray to the
    // integrator (the render stays exact, at the integrator's cost).
    if ((e = cudaMemsetAsync(s->err, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
    if (c->views) {  // batched render (captured in a graph): per-ray view, mode and variant
        if ((e = launch_sur_features_batch(c->p, c->views, c->nviews, c->spp, c->seed, q, s, st)) != cudaSuccess)
            return e;
        if ((e = sur_forward(s, s->inf_rows, q.count, st)) != cudaSuccess) return e;
        return launch_sur_gate_batch(c->p, c->views, c->nviews, c->spp, c->seed, q, s, c->samples, st);
    }
    if ((e = launch_sur_features(c->p, c->mode, c->spp, c->seed, q, s, st)) != cudaSuccess) return e;
    if ((e = sur_forward(s, s->inf_rows, q.count, st)) != cudaSuccess) return e;
    return launch_sur_gate(c->p, c->mode, c->spp, c->seed, q, s, c->samples, c->recs, st);
}

}  // namespace ck
