// alu_peak.cu -- FMA throughput microbenchmark: the measured denominators of the ALU rooflines
// (FP64 for the integrator, FP32 for the mixed-precision form).  The paper has no counterpart.
//
// Every thread runs CHAINS independent fused multiply-add chains x <- x * a + b (no dependence between
// chains, so the pipe, not the FMA latency, bounds the rate).  With |a| < 1 the chains settle on the
// fixed point b / (1 - a): no overflow, no subnormals.  The result is stored only when a condition the
// compiler cannot decide holds, so the chains stay live without a memory write per thread.
#include <cuda_runtime.h>

namespace {

constexpr int CHAINS = 8;
constexpr int UNROLL = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T *sink, long long iters, T a, T b) {
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == T(-1)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true for a in (0, 1), b > 0
}

}  // namespace

namespace ck {
// Launch of the microbenchmark (argument checks in the C ABI): returns the launch status and the
// operations the launch performs.
cudaError_t launch_fma_peak(int fp64, int blocks, int threads, long long iters, void *sink, double *flops,
                            cudaStream_t st) {
    if (fp64)
        k_fma_peak<double><<<blocks, threads, 0, st>>>(static_cast<double *>(sink), iters, 0.999999, 1e-7);
    else
        k_fma_peak<float><<<blocks, threads, 0, st>>>(static_cast<float *>(sink), iters, 0.9999f, 1e-4f);
    *flops = 2.0 * CHAINS * UNROLL * double(iters) * double(blocks) * double(threads);
    return cudaGetLastError();
}
}  // namespace ck
