// mlp_tc.cuh -- BF16 tensor-core GEMM for the learned surrogate (sm_103a: tcgen05 + TMEM + TMA).
//
//   C[M x N] = A[M x K] * B[N x K]^T      A, B row-major BF16 (K contiguous), FP32 accumulation.
//
// One CTA (4 warps) computes a 128 x N tile (N <= 256, multiple of 16) over one slice of K (split-K:
// gridDim.y slices).  K is consumed in chunks of 64 elements (128 bytes, one 128B-swizzle row): warp 0 /
// lane 0 issues the TMA loads of A and B chunks into a 3-stage shared-memory ring and the tcgen05.mma
// instructions (M = 128, K = 16 each, accumulator in tensor memory), committing each stage back to its
// "empty" barrier.  After the last MMA completes, every warp reads its 32 accumulator lanes with
// tcgen05.ld and applies the epilogue (row r, column c, accumulator a):
//   EPI_STORE     C[r, c] = a
//   EPI_ATOMIC    C[r, c] += a                                (split-K partial sums, FP32 atomics)
//   EPI_BIAS      Z[r, c] = a + bias[c]
//   EPI_BIAS_GELU z = a + bias[c]; Z[r, c] = z (if Z); H[r, c] = GELU(z) (BF16); HT[c, r] = H[r, c] (if HT)
//   EPI_GELU_BWD  g = a * GELU'(Z[r, c]); H[r, c] = g (BF16); HT[c, r] = g (if HT)
// With m_count set, tiles whose first row (+ m_base) is at or beyond *m_count are skipped (device-side row
// count).
// Every mbarrier wait is bounded; on timeout the kernel records an error code and skips ahead.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ck {

enum { EPI_STORE = 0, EPI_BIAS_GELU = 1, EPI_BIAS = 2, EPI_ATOMIC = 3, EPI_GELU_BWD = 4 };

struct GemmArgs {
    int M, N, K;                 // M % 128 == 0, N % 16 == 0 (16..256), K % (64 * ksplit) == 0
    int ksplit;                  // slices of K (gridDim.y)
    const unsigned int *m_count; // optional device row count
    long long m_base;            // row of this GEMM's row 0 in the count's numbering (chunked inference)
    float *C;                    // EPI_STORE / EPI_ATOMIC: C[M x ldc]
    int ldc;
    const float *bias;           // [N]
    float *Z;                    // EPI_BIAS*: output (optional for GELU); EPI_GELU_BWD: input
    int ldz;
    __nv_bfloat16 *H;            // EPI_BIAS_GELU / EPI_GELU_BWD: H[M x ldh]
    int ldh;
    __nv_bfloat16 *HT;           // optional transposed copy HT[N x ldht]
    int ldht;
    int epi;
    unsigned int *err;           // error flag (0 = ok)
    unsigned int wait_limit;     // polls of the waits that decide a timeout (MBAR_DEFAULT_LIMIT)
    long long slice_stride;      // EPI_STORE with ksplit > 1: slice y of K writes its partial product to
                                 // C + y * slice_stride (summed afterwards in a fixed order), 0 otherwise
};

constexpr int GEMM_TILE_M = 128;
constexpr int GEMM_KCHUNK = 64;
constexpr int GEMM_STAGES = 2;  // K of the network's layers is at most 256: four chunks, double-buffered

inline size_t gemm_smem_bytes(int N) {
    return 1024 + (size_t)GEMM_STAGES * (GEMM_TILE_M * 128 + (size_t)N * 128);
}

// host: TMA descriptors for a row-major BF16 matrix [rows x cols] with box (64 cols x box_rows)
CUresult make_tmap_bf16(CUtensorMap *map, const void *base, int rows, int cols, int box_rows);
// the same for a half-precision (FP16) matrix
CUresult make_tmap_f16(CUtensorMap *map, const void *base, int rows, int cols, int box_rows);
cudaError_t launch_gemm_tc(const CUtensorMap &ta, const CUtensorMap &tb, const GemmArgs &g, cudaStream_t st);

}  // namespace ck
