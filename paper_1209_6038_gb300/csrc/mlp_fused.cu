// mlp_fused.cu -- the surrogate network's forward pass as ONE persistent tcgen05 kernel.
//
// Each CTA (one per SM) takes pairs of 128-row tiles through all five layers without their activations
// leaving the SM.  Warp-specialised, the two tiles of a pair in ping-pong; the jobs are (tile 0, layer 0),
// (tile 1, layer 0), (tile 0, layer 1), ...:
//   * the copy warp (one thread) streams the jobs' weights from L2 by TMA in 64-wide K chunks (32 KB,
//     128-byte swizzle) through a 3-slot ring, refilling a slot as soon as the MMAs that read it are done,
//     and loads each tile's inputs (the K-major layout the MMA reads) once the tile's previous last-layer
//     MMAs are done -- after the weight chunk of the tile's first job, so that chunk is already on its way;
//   * the MMA warp (one thread) issues, per chunk, the four tcgen05.mma (M = 128, K = 16) of the job's tile
//     (one for the first layer, whose 14 input columns fit one K step) into its TMEM columns (tile t:
//     256 t .. 256 t + 255) and frees the slot by a commit.  Before a job's
//     first MMA it waits only for the epilogue of the same tile's previous layer, so the MMAs of one tile
//     run while the epilogue of the other tile runs.  The two roles are separate threads because one
//     thread doing both spent longer per chunk on its barrier waits and bookkeeping than the tensor core
//     spent on the chunk's four MMAs;
//   * 16 epilogue warps take the jobs in the same order (warp w: TMEM lanes 32 (w % 4) .., column quarter
//     w / 4): they read the tile's accumulators once its MMAs completed (16 columns per TMEM load), round
//     them to half-precision pairs, add the half-precision bias (read through L1), apply GELU in the
//     same pairs and write the activations back into the swizzled shared-memory layout as the tile's
//     next A operand (the last layer writes the FP32 outputs, its bias added in FP32), then arrive on the
//     tile's barrier.
// Operands (weights, inputs as (hi, lo) pairs, activations) are BF16, the precision the network is trained
// in, or -- selected per network -- FP16: the GELU is evaluated in half-precision pairs in both forms, and
// in FP16 its result is stored as it is (no conversion back through FP32 to BF16: faster, and 11
// significant bits instead of 8).  Accumulation is FP32 in both.
// Barriers: full/empty per ring slot; per tile the inputs' barrier, "MMAs done" (committed by the MMA
// warp) and "activations ready" (16 arrivals).  Shared memory: activations 2 x 64 KB, weight ring
// 3 x 32 KB.  Every mbarrier wait is bounded; on a timeout the kernel sets the error flag, lets its MMAs and
// copies in flight complete, frees TMEM and returns.
#include "device_once.h"
#include "surrogate.h"
#include "tc_ptx.cuh"

namespace ck {

namespace {
constexpr int F_EPI_WARPS = 16;
constexpr int F_COPY_WARP = F_EPI_WARPS;                       // warp index of the TMA copy thread
constexpr int F_MMA_WARP = F_EPI_WARPS + 1;                    // warp index of the MMA thread
constexpr int F_THREADS = 32 * (F_EPI_WARPS + 2);
constexpr int F_PARTS = F_EPI_WARPS / 4;                       // epilogue warps per row quarter (column parts)
constexpr uint32_t F_ACT_CHUNK = 128 * 128;                  // 128 rows x 64 BF16 = 16 KB
constexpr uint32_t F_ACT_BYTES = 2 * 4 * F_ACT_CHUNK;         // 2 tiles x 4 K chunks
constexpr uint32_t F_RING_SLOT = 256 * 128;                   // up to 256 weight rows x 64 BF16
constexpr int F_SLOTS = 3;                                     // weight ring depth
constexpr size_t F_SMEM = 1024 + F_ACT_BYTES + F_SLOTS * F_RING_SLOT;

struct FusedArgs {
    const float *bias[SUR_L];    // FP32 biases (the output layer's are used)
    const __half *bias_h[SUR_L - 1]; // hidden layers' biases in half precision (both forms)
    float *Y;                    // outputs, 16 FP32 per row
    long long n;                 // rows of X and Y (a multiple of 128)
    const unsigned int *m_count; // optional live row count
    unsigned int *err;
    unsigned int wait_limit;     // polls of the waits that decide a timeout
};

// bias, GELU and the store of 16 columns from c (a multiple of 16) of row r: u the FP32 accumulators,
// b0, b1 the 16 half-precision biases; the result goes into the 128-byte-swizzled K-major layout of chunk
// c / 64 of the tile's activations (16-byte units (c % 64) / 8 and + 1 of the row, each XOR-ed with r % 8)
template <bool F16>
__device__ __forceinline__ void epi_piece(const uint32_t (&u)[16], uint4 b0, uint4 b1, unsigned char *act_t, int c,
                                          int r) {
    const uint32_t bw[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
    uint32_t pk[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const __half2 bias = *reinterpret_cast<const __half2 *>(&bw[k]);
        pk[k] = F16 ? gelu2_f16(__uint_as_float(u[2 * k]), __uint_as_float(u[2 * k + 1]), bias)
                    : gelu2_bf16(__uint_as_float(u[2 * k]), __uint_as_float(u[2 * k + 1]), bias);
    }
    unsigned char *chunk = act_t + (c / 64) * F_ACT_CHUNK + (r >> 3) * 1024 + (r & 7) * 128;
    const int u0 = (c & 63) >> 3;
    *(uint4 *)(chunk + ((u0 ^ (r & 7)) << 4)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *(uint4 *)(chunk + (((u0 + 1) ^ (r & 7)) << 4)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

template <bool F16>
__global__ void __launch_bounds__(F_THREADS, 1)
    k_mlp_fused(const __grid_constant__ CUtensorMap tX, const __grid_constant__ CUtensorMap tW0,
                const __grid_constant__ CUtensorMap tW1, const __grid_constant__ CUtensorMap tW2,
                const __grid_constant__ CUtensorMap tW3, const __grid_constant__ CUtensorMap tW4, FusedArgs a) {
    extern __shared__ unsigned char fsm_raw[];
    __shared__ __align__(8) uint64_t full_bar[F_SLOTS], empty_bar[F_SLOTS], x_bar[2], done_bar[2], act_bar[2], drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    unsigned char *sm = (unsigned char *)(((uintptr_t)fsm_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *act = sm, *ring = sm + F_ACT_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long live = a.m_count ? min(a.n, (long long)__ldg(a.m_count)) : a.n;
    volatile int *vfailed = &failed;
    const uint32_t lim = a.wait_limit;

    if (tid == 0) {
        for (int s = 0; s < F_SLOTS; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int t = 0; t < 2; ++t) {
            mbar_init(smem_u32(&x_bar[t]), 1);
            mbar_init(smem_u32(&done_bar[t]), 1);
            mbar_init(smem_u32(&act_bar[t]), F_EPI_WARPS);
        }
        mbar_init(smem_u32(&drain_bar), 1);
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    const long long stride = (long long)gridDim.x * 256;

    if (warp == F_COPY_WARP) {
        if (lane == 0) {
            uint32_t s = 0, ph = 0;  // ring slot of the next load and its use count's parity
            uint32_t loads = 0;      // weight chunks loaded
            uint32_t Lx = 0;         // tile pairs whose inputs were loaded (x_bar phase)
            bool x_pending[2] = {false, false};
            uint32_t x_phase[2] = {0, 0};
            bool ok = true;
            for (long long base = (long long)blockIdx.x * 256; base < live && ok; base += stride) {
                for (int job = 0; job < 2 * SUR_L && ok; ++job) {
                    const int l = job >> 1, t = job & 1;
                    const int nk = l == 0 ? 1 : 4;
                    const uint32_t bytes = l == SUR_L - 1 ? 16u * 128u : 256u * 128u;
                    const CUtensorMap *map = l == 0 ? &tW0 : l == 1 ? &tW1 : l == 2 ? &tW2 : l == 3 ? &tW3 : &tW4;
                    for (int j = 0; j < nk; ++j) {
                        // the slot is free once the MMAs of the chunk loaded F_SLOTS chunks ago are done
                        if (loads >= F_SLOTS) ok = mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, lim);
                        if (!ok) break;
                        mbar_expect_tx(smem_u32(&full_bar[s]), bytes);
                        tma_load_2d(smem_u32(ring + s * F_RING_SLOT), map, j * 64, 0, smem_u32(&full_bar[s]));
                        ++loads;
                        if (++s == F_SLOTS) { s = 0; ph ^= 1u; }
                    }
                    if (!ok) break;
                    if (l == 0) {
                        // the tile's inputs overwrite its activations, which its previous last-layer MMAs read
                        // ("MMAs done" completes SUR_L times per tile and pair)
                        if (Lx > 0) ok = mbar_wait(smem_u32(&done_bar[t]), (SUR_L * Lx - 1) & 1, lim);
                        if (!ok || *vfailed) { ok = false; break; }
                        mbar_expect_tx(smem_u32(&x_bar[t]), F_ACT_CHUNK);
                        tma_load_2d(smem_u32(act + t * 4 * F_ACT_CHUNK), &tX, 0, (int)(base + 128 * t), smem_u32(&x_bar[t]));
                        x_pending[t] = true;
                        x_phase[t] = Lx & 1;
                    }
                }
                ++Lx;
            }
            if (!ok) {
                *vfailed = 1;
                if (a.err) atomicExch(a.err, 1u);
            }
            // every copy has landed before the shared memory is released: the last load into each slot and
            // the last inputs of each tile (at once on a normal exit, where the MMAs consumed them; bounded by
            // the default limit after a timeout)
            for (uint32_t k = 0; k < F_SLOTS && k < loads; ++k) {
                const uint32_t g = loads - 1 - k;  // one of the last F_SLOTS loads, each in its own slot
                mbar_wait(smem_u32(&full_bar[g % F_SLOTS]), (g / F_SLOTS) & 1);
            }
            for (int t = 0; t < 2; ++t)
                if (x_pending[t]) mbar_wait(smem_u32(&x_bar[t]), x_phase[t]);
        }
    } else if (warp == F_MMA_WARP) {
        if (lane == 0) {
            uint32_t s = 0, ph = 0;  // ring slot of the next chunk and its fill parity
            uint32_t Lt[2] = {0, 0}; // jobs committed per tile (phases of done_bar[t] / act_bar[t])
            uint32_t iters = 0;      // tile pairs started (phase of x_bar[t])
            bool ok = true;
            const uint32_t ring0 = smem_u32(ring), act0 = smem_u32(act);
            for (long long base = (long long)blockIdx.x * 256; base < live && ok; base += stride) {
                for (int job = 0; job < 2 * SUR_L && ok; ++job) {
                    const int l = job >> 1, t = job & 1;
                    const int nk = l == 0 ? 1 : 4;
                    const uint32_t idesc = F16 ? f16_idesc(l == SUR_L - 1 ? 16 : SUR_W) : bf16_idesc(l == SUR_L - 1 ? 16 : SUR_W);
                    const uint32_t d_tmem = tmem + t * 256;
                    for (int j = 0; j < nk; ++j) {
                        ok = mbar_wait(smem_u32(&full_bar[s]), ph, lim);
                        if (ok && j == 0) {
                            // the tile's previous epilogue has read its accumulators and written these inputs
                            if (Lt[t] > 0) ok = mbar_wait(smem_u32(&act_bar[t]), (Lt[t] - 1) & 1, lim);
                            if (ok && l == 0) ok = mbar_wait(smem_u32(&x_bar[t]), iters & 1, lim);
                            if (ok && *vfailed) ok = false;
                        }
                        if (!ok) break;
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const uint64_t bd = sw128_desc(ring0 + s * F_RING_SLOT);
                        const uint64_t ad = sw128_desc(act0 + (uint32_t)(t * 4 + j) * F_ACT_CHUNK);
                        // the first layer's inputs (7 values as hi/lo pairs) and weights fill K columns 0..13 of
                        // the chunk and are zero beyond: one MMA covers them
                        const int nmma = l == 0 ? 1 : 4;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            if (kk >= nmma) break;
                            const uint32_t acc = (j > 0 || kk > 0) ? 1u : 0u;
                            asm volatile(
                                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
                                "l"(ad + (uint64_t)(2 * kk)), "l"(bd + (uint64_t)(2 * kk)), "r"(idesc), "r"(acc));
                        }
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            smem_u32(&empty_bar[s])));
                        if (++s == F_SLOTS) { s = 0; ph ^= 1u; }
                    }
                    if (!ok) break;
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&done_bar[t])));
                    ++Lt[t];
                }
                ++iters;
            }
            if (!ok) {
                *vfailed = 1;
                if (a.err) atomicExch(a.err, 1u);
                // the MMAs already issued complete before the accumulators are freed (a commit arrives once every
                // earlier MMA of this thread is done); bounded by the default limit
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&drain_bar)));
                mbar_wait(smem_u32(&drain_bar), 0);
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (one row per thread), column quarter w / 4
        const int q = warp & 3, r = q * 32 + lane, part = warp >> 2;
        uint32_t Lt[2] = {0, 0};
        bool ok = true;
        for (long long base = (long long)blockIdx.x * 256; base < live && ok; base += stride) {
            for (int job = 0; job < 2 * SUR_L; ++job) {
                const int l = job >> 1, t = job & 1;
                const int N = l == SUR_L - 1 ? 16 : SUR_W;
                const int cw = max(16, N / F_PARTS), c0 = part * cw, c1 = min(N, c0 + cw);
                // the half-precision biases of the warp's columns, 16 per piece (two 16-byte loads through L1);
                // the first piece's are read while the MMAs run
                const uint4 *bias8 = reinterpret_cast<const uint4 *>(a.bias_h[l < SUR_L - 1 ? l : 0] + c0);
                uint4 b0 = make_uint4(0, 0, 0, 0), b1 = b0;
                if (l < SUR_L - 1) {
                    b0 = __ldg(bias8);
                    b1 = __ldg(bias8 + 1);
                }
                ok = mbar_wait(smem_u32(&done_bar[t]), Lt[t] & 1, lim) && !*vfailed;
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * 256);
                if (l < SUR_L - 1) {
                    // four 16-column pieces, one TMEM load each (loads kept in flight across the GELU of the
                    // previous piece measured slower: 32 more live registers per thread)
                    unsigned char *act_t = act + t * 4 * F_ACT_CHUNK;
#pragma unroll 1
                    for (int pc = 0; pc < 4; ++pc) {
                        if (pc) {
                            b0 = __ldg(bias8 + 2 * pc);
                            b1 = __ldg(bias8 + 2 * pc + 1);
                        }
                        uint32_t u[16];
                        tmem_ld16(taddr + (uint32_t)(c0 + 16 * pc), u);
                        tmem_wait16(u);
                        epi_piece<F16>(u, b0, b1, act_t, c0 + 16 * pc, r);
                    }
                } else if (c0 < c1) {  // the 16 outputs in FP32
                    uint32_t u[16];
                    tmem_ld16(taddr, u);
                    tmem_wait16(u);
                    const long long row = base + t * 128 + r;
                    if (row < live) {
                        float4 *y = (float4 *)(a.Y + row * 16);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            y[i] = make_float4(__uint_as_float(u[4 * i]) + __ldg(a.bias[SUR_L - 1] + 4 * i),
                                               __uint_as_float(u[4 * i + 1]) + __ldg(a.bias[SUR_L - 1] + 4 * i + 1),
                                               __uint_as_float(u[4 * i + 2]) + __ldg(a.bias[SUR_L - 1] + 4 * i + 2),
                                               __uint_as_float(u[4 * i + 3]) + __ldg(a.bias[SUR_L - 1] + 4 * i + 3));
                    }
                }
                // the shared-memory writes must be visible to the tensor cores' (async) reads, and the TMEM
                // reads complete, before the producer's next MMAs of this tile
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&act_bar[t]));
                ++Lt[t];
            }
        }
        if (!ok) {
            *vfailed = 1;
            if (lane == 0 && a.err) atomicExch(a.err, 1u);  // this warp's rows were not written
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}
}  // namespace

static DeviceOnce g_fused_once;
static int g_fused_sms[MAX_DEVICES];

// one-time setup of the kernel on the current device (also before a stream capture)
cudaError_t mlp_fused_prepare() {
    return g_fused_once.run([](int dev) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&g_fused_sms[dev], cudaDevAttrMultiProcessorCount, dev);
        for (auto kern : {k_mlp_fused<false>, k_mlp_fused<true>}) {
            cudaFuncAttributes fa;
            cudaError_t e = cudaFuncGetAttributes(&fa, kern);
            if (e != cudaSuccess) return e;
            if ((size_t)(optin - (int)fa.sharedSizeBytes) < F_SMEM) return cudaErrorInvalidValue;
            if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F_SMEM)) != cudaSuccess)
                return e;
        }
        return cudaSuccess;
    });
}

// forward pass of rows [0, n) of s->X into s->Y (rows beyond *m_count skipped when it is set)
cudaError_t launch_mlp_fused(SurNet *s, long long n, const unsigned int *m_count, cudaStream_t st) {
    cudaError_t e0 = mlp_fused_prepare();
    if (e0 != cudaSuccess) return e0;
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = g_fused_sms[dev];
    if (n <= 0 || n % 128) return cudaErrorInvalidValue;
    CUtensorMap tx;
    const bool f16 = s->inf_f16 != 0;
    if ((f16 ? make_tmap_f16(&tx, s->X, (int)n, 64, GEMM_TILE_M) : make_tmap_bf16(&tx, s->X, (int)n, 64, GEMM_TILE_M)) !=
        CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    FusedArgs a;
    for (int l = 0; l < SUR_L; ++l) a.bias[l] = s->b[l];
    for (int l = 0; l < SUR_L - 1; ++l) a.bias_h[l] = s->bh[l];
    a.Y = s->Y;
    a.n = n;
    a.m_count = m_count;
    a.err = s->err;
    a.wait_limit = wait_limit();
    const long long pairs = (n + 255) / 256;
    const int grid = (int)std::min<long long>(pairs, (long long)sms);
    if (f16)
        k_mlp_fused<true><<<grid, F_THREADS, F_SMEM, st>>>(tx, s->tWh[0], s->tWh[1], s->tWh[2], s->tWh[3], s->tWh[4], a);
    else
        k_mlp_fused<false><<<grid, F_THREADS, F_SMEM, st>>>(tx, s->tWb[0], s->tWb[1], s->tWb[2], s->tWb[3], s->tWb[4], a);
    return cudaGetLastError();
}

}  // namespace ck
