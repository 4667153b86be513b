// surrogate.cu -- C ABI of the learned surrogate's tensor-core building blocks.
#include <cstdio>
#include <string>

#include "cloak.h"
#include "mlp_tc.cuh"

namespace {
__device__ unsigned int g_gemm_err;  // timeout flag of the last cloak_mlp_gemm call
}

extern "C" int cloak_mlp_gemm(const void *dev_a, const void *dev_b, float *dev_c, int M, int N, int K,
                              void *cuda_stream) {
    if (!dev_a || !dev_b || !dev_c) return CLOAK_EINVAL;
    if (M <= 0 || M % 128 || N < 16 || N > 256 || N % 16 || K <= 0 || K % 64) return CLOAK_EINVAL;
    if (((uintptr_t)dev_a | (uintptr_t)dev_b) & 15) return CLOAK_EINVAL;
    CUtensorMap ta, tb;
    if (ck::make_tmap_bf16(&ta, dev_a, M, K, ck::GEMM_TILE_M) != CUDA_SUCCESS) return CLOAK_ECUDA;
    if (ck::make_tmap_bf16(&tb, dev_b, N, K, N) != CUDA_SUCCESS) return CLOAK_ECUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned int *err = nullptr;
    if (cudaGetSymbolAddress((void **)&err, g_gemm_err) != cudaSuccess) return CLOAK_ECUDA;
    if (cudaMemsetAsync(err, 0, sizeof(unsigned int), st) != cudaSuccess) return CLOAK_ECUDA;
    ck::GemmArgs g{};
    g.M = M; g.N = N; g.K = K; g.C = dev_c; g.ldc = N; g.epi = ck::EPI_STORE; g.err = err;
    if (ck::launch_gemm_tc(ta, tb, g, st) != cudaSuccess) return CLOAK_ECUDA;
    unsigned int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CLOAK_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CLOAK_ECUDA;
    return h ? CLOAK_ETIMEOUT : CLOAK_OK;
}
