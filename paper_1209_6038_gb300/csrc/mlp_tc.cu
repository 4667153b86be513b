// mlp_tc.cu -- tcgen05 / TMEM / TMA BF16 GEMM (see mlp_tc.cuh).
#include <cudaTypedefs.h>

#include "device_once.h"
#include "mlp_tc.cuh"
#include "tc_ptx.cuh"

namespace ck {

// 16 consecutive values of one row as BF16 into H, and into the transposed copy HT when it is set
__device__ __forceinline__ void store_bf16_row(const GemmArgs &g, int row, int c, const float v[16]) {
    __nv_bfloat162 hv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) hv[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    uint4 *dh = (uint4 *)(g.H + (size_t)row * g.ldh + c);
    dh[0] = *(uint4 *)&hv[0];
    dh[1] = *(uint4 *)&hv[4];
    if (g.HT) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            g.HT[(size_t)(c + 2 * i) * g.ldht + row] = hv[i].x;
            g.HT[(size_t)(c + 2 * i + 1) * g.ldht + row] = hv[i].y;
        }
    }
}

__global__ void __launch_bounds__(128, 1) k_gemm_tc(const __grid_constant__ CUtensorMap ta,
                                                    const __grid_constant__ CUtensorMap tb, GemmArgs g) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[GEMM_STAGES], empty_bar[GEMM_STAGES], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    const int m0 = blockIdx.x * GEMM_TILE_M;
    if (g.m_count && g.m_base + m0 >= (long long)__ldg(g.m_count)) return;  // whole tile beyond the live rows
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int kslice = g.K / g.ksplit, kbase = blockIdx.y * kslice;
    const int N = g.N, nk = kslice / GEMM_KCHUNK;
    const uint32_t a_bytes = GEMM_TILE_M * 128, b_bytes = (uint32_t)N * 128;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t ncols = 32;
    while ((int)ncols < N) ncols <<= 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < GEMM_STAGES; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&done_bar), 1);
        failed = 0;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;

    if (threadIdx.x == 0) {
        const uint32_t idesc = bf16_idesc(N);
        bool ok = true;
        int loaded = 0, consumed = 0;  // chunks whose TMA loads were issued / whose full barrier was seen
        for (int it = 0; it < nk + GEMM_STAGES - 1 && ok; ++it) {
            if (it < nk) {  // load chunk `it`
                const int s = it % GEMM_STAGES;
                if (it >= GEMM_STAGES) ok = mbar_wait(smem_u32(&empty_bar[s]), ((it / GEMM_STAGES) - 1) & 1, g.wait_limit);
                if (!ok) break;
                unsigned char *sa = smem + s * (a_bytes + b_bytes), *sb = sa + a_bytes;
                mbar_expect_tx(smem_u32(&full_bar[s]), a_bytes + b_bytes);
                tma_load_2d(smem_u32(sa), &ta, kbase + it * GEMM_KCHUNK, m0, smem_u32(&full_bar[s]));
                tma_load_2d(smem_u32(sb), &tb, kbase + it * GEMM_KCHUNK, 0, smem_u32(&full_bar[s]));
                loaded = it + 1;
            }
            const int j = it - (GEMM_STAGES - 1);
            if (j >= 0 && j < nk) {  // multiply chunk j
                const int s = j % GEMM_STAGES;
                ok = mbar_wait(smem_u32(&full_bar[s]), (j / GEMM_STAGES) & 1, g.wait_limit);
                if (!ok) break;
                consumed = j + 1;
                asm volatile("tcgen05.fence::after_thread_sync;");
                unsigned char *sa = smem + s * (a_bytes + b_bytes), *sb = sa + a_bytes;
                const uint64_t ad = sw128_desc(smem_u32(sa)), bd = sw128_desc(smem_u32(sb));
#pragma unroll
                for (int kk = 0; kk < GEMM_KCHUNK / 16; ++kk) {
                    const uint32_t acc = (j > 0 || kk > 0) ? 1u : 0u;
                    // advance 16 K-elements (32 bytes) inside the swizzled 128-byte row
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(ad + (uint64_t)(2 * kk)), "l"(bd + (uint64_t)(2 * kk)), "r"(idesc), "r"(acc));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&empty_bar[s])));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&done_bar)));
        if (!ok) {
            failed = 1;
            // let the copies still in flight land before the CTA's shared memory is released (bounded)
            for (int c = consumed; c < loaded; ++c)
                if (!mbar_wait(smem_u32(&full_bar[c % GEMM_STAGES]), (c / GEMM_STAGES) & 1)) break;
        }
    }
    __syncwarp();
    const bool done = mbar_wait(smem_u32(&done_bar), 0);
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (!done || failed) {
        if (threadIdx.x == 0 && g.err) atomicExch(g.err, 1u);
    } else {
        const int row = m0 + warp * 32 + lane;
        for (int c = 0; c < N; c += 16) {
            uint32_t r[16];
            const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
            if (row < g.M) {
                if (g.epi == EPI_STORE || g.epi == EPI_ATOMIC) {
                    float4 *dst = (float4 *)(g.C + (size_t)blockIdx.y * (size_t)g.slice_stride + (size_t)row * g.ldc + c);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        float4 q = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                        if (g.epi == EPI_STORE) dst[i] = q;
                        else atomicAdd(dst + i, q);
                    }
                } else if (g.epi == EPI_GELU_BWD) {
                    const float4 *zi = (const float4 *)(g.Z + (size_t)row * g.ldz + c);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        float4 z = zi[i];
                        v[4 * i] *= gelu_tanh_grad(z.x);
                        v[4 * i + 1] *= gelu_tanh_grad(z.y);
                        v[4 * i + 2] *= gelu_tanh_grad(z.z);
                        v[4 * i + 3] *= gelu_tanh_grad(z.w);
                    }
                    store_bf16_row(g, row, c, v);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += g.bias[c + i];
                    if (g.Z) {
                        float4 *dz = (float4 *)(g.Z + (size_t)row * g.ldz + c);
#pragma unroll
                        for (int i = 0; i < 4; ++i) dz[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                    }
                    if (g.epi == EPI_BIAS_GELU) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = gelu_tanh(v[i]);
                        store_bf16_row(g, row, c, v);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ------------------------------------------------------------------ host
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

static CUresult make_tmap_16bit(CUtensorMap *map, CUtensorMapDataType type, const void *base, int rows, int cols,
                                int box_rows) {
    auto enc = get_encode();
    if (!enc) return CUDA_ERROR_NOT_SUPPORTED;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)GEMM_KCHUNK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, type, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}
CUresult make_tmap_bf16(CUtensorMap *map, const void *base, int rows, int cols, int box_rows) {
    return make_tmap_16bit(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, rows, cols, box_rows);
}
CUresult make_tmap_f16(CUtensorMap *map, const void *base, int rows, int cols, int box_rows) {
    return make_tmap_16bit(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, base, rows, cols, box_rows);
}

cudaError_t launch_gemm_tc(const CUtensorMap &ta, const CUtensorMap &tb, const GemmArgs &g, cudaStream_t st) {
    if (g.M <= 0 || g.M % GEMM_TILE_M || g.N < 16 || g.N > 256 || g.N % 16 || g.ksplit < 1 || g.K <= 0 ||
        g.K % (GEMM_KCHUNK * g.ksplit))
        return cudaErrorInvalidValue;
    // Shared memory per CTA: the ring, padded so that no more CTAs share an SM than its 512 TMEM columns
    // hold (each allocates the power of two >= N, at least 32) -- an allocation never has to wait.
    static DeviceOnce once;
    static int smem_sm_of[MAX_DEVICES], reserved_of[MAX_DEVICES], max_dyn_of[MAX_DEVICES];
    cudaError_t e0 = once.run([](int dev) {
        int optin = 0;
        cudaDeviceGetAttribute(&smem_sm_of[dev], cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&reserved_of[dev], cudaDevAttrReservedSharedMemoryPerBlock, dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, k_gemm_tc);
        if (e != cudaSuccess) return e;
        max_dyn_of[dev] = optin - (int)fa.sharedSizeBytes;  // the barriers are static shared memory
        return cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_of[dev]);
    });
    if (e0 != cudaSuccess) return e0;
    int dev = 0;
    cudaGetDevice(&dev);
    const int smem_sm = smem_sm_of[dev], reserved = reserved_of[dev], max_dyn = max_dyn_of[dev];
    int ncols = 32;
    while (ncols < g.N) ncols <<= 1;
    const int max_ctas = 512 / ncols;
    size_t smem = gemm_smem_bytes(g.N);
    const size_t floor_b = (size_t)smem_sm / (size_t)(max_ctas + 1) + 1;
    if (smem + (size_t)reserved < floor_b) smem = floor_b - (size_t)reserved;
    if (smem > (size_t)max_dyn) return cudaErrorInvalidValue;
    k_gemm_tc<<<dim3(g.M / GEMM_TILE_M, g.ksplit), 128, smem, st>>>(ta, tb, g);
    return cudaGetLastError();
}

}  // namespace ck
