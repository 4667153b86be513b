// tc_ptx.cuh -- sm_103a building blocks of the tensor-core kernels: mbarriers with bounded waits, TMA
// tile loads, tcgen05 shared-memory and instruction descriptors, GELU.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ck {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Polls of one bounded mbarrier wait before it gives up (the default; cloak_set_wait_limit can lower the
// bound of the waits that decide a timeout, never of those that let in-flight work land before an exit).
constexpr uint32_t MBAR_DEFAULT_LIMIT = 1u << 22;
// bounded wait for the phase with the given parity; false on timeout.  The first poll does not block
// (test_wait), later ones may suspend briefly (try_wait): a bound of one poll gives up unless the phase is
// already complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit = MBAR_DEFAULT_LIMIT) {
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        if (it == 0)
            asm volatile(
                "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(ok)
                : "r"(bar), "r"(parity)
                : "memory");
        else
            asm volatile(
                "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(ok)
                : "r"(bar), "r"(parity)
                : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);        // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // layout: 128-byte swizzle
    return d;
}
// instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both operands K-major, M = 128
__host__ __device__ constexpr uint32_t bf16_idesc(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
// the same for FP16 x FP16 -> FP32 (operand formats 0)
__host__ __device__ constexpr uint32_t f16_idesc(int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// GELU, tanh form, with the hardware tanh approximation (tanh.approx.f32, relative error about 2^-11: below
// the BF16 rounding of the activations it feeds), and its derivative (FP32)
__device__ __forceinline__ float tanh_fast(float u) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
    return t;
}
__device__ __forceinline__ float gelu_tanh(float x) {
    const float k0 = 0.7978845608028654f, k1 = 0.044715f;
    float u = k0 * (x + k1 * x * x * x);
    return 0.5f * x * (1.f + tanh_fast(u));
}
// 16 consecutive TMEM columns of the warp's 32 lanes (one lane per thread) into u; the load is
// asynchronous: read u only after tmem_wait16(u)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&u)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
                   "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
                 : "r"(taddr));
}
// waits for every TMEM load of the thread; u as operands, so that no use of u moves above the wait
__device__ __forceinline__ void tmem_wait16(uint32_t (&u)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(u[0]), "+r"(u[1]), "+r"(u[2]), "+r"(u[3]), "+r"(u[4]), "+r"(u[5]), "+r"(u[6]), "+r"(u[7]),
                   "+r"(u[8]), "+r"(u[9]), "+r"(u[10]), "+r"(u[11]), "+r"(u[12]), "+r"(u[13]), "+r"(u[14]), "+r"(u[15])
                 :
                 : "memory");
}
// GELU (tanh form) of x = (a, b) + bias in half-precision pair arithmetic: x rounded to a half pair, the
// bias added, then x (1 + tanh(u)) / 2 with u = x (k0 + k0 k1 x^2), k0 = sqrt(2/pi), k1 = 0.044715 (one
// hardware tanh, tanh.approx.f16x2, for two values).  Half precision carries 11 significant bits;
// inputs must stay below its range (|x| < 65504), where x^2 overflowing only saturates tanh.
__device__ __forceinline__ __half2 gelu2_h2(float a, float b, __half2 bias) {
    const __half2 x = __hadd2(__floats2half2_rn(a, b), bias);
    const __half2 c1 = __float2half2_rn(0.7978845608028654f * 0.044715f), c0 = __float2half2_rn(0.7978845608028654f),
                  half = __float2half2_rn(0.5f);
    const __half2 u = __hmul2(x, __hfma2(c1, __hmul2(x, x), c0));
    __half2 th;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(*(uint32_t *)&th) : "r"(*(const uint32_t *)&u));
    const __half2 hx = __hmul2(half, x);
    return __hfma2(hx, th, hx);
}
// the same packed as BF16x2 (8 significant bits): the BF16 activations of the fused inference kernel
__device__ __forceinline__ uint32_t gelu2_bf16(float a, float b, __half2 bias) {
    const float2 g = __half22float2(gelu2_h2(a, b, bias));
    const __nv_bfloat162 o = __floats2bfloat162_rn(g.x, g.y);
    return *(const uint32_t *)&o;
}
// the same as a half-precision pair: the FP16 activations
__device__ __forceinline__ uint32_t gelu2_f16(float a, float b, __half2 bias) {
    const __half2 o = gelu2_h2(a, b, bias);
    return *(const uint32_t *)&o;
}
__device__ __forceinline__ float gelu_tanh_grad(float x) {
    const float k0 = 0.7978845608028654f, k1 = 0.044715f;
    float th = tanhf(k0 * (x + k1 * x * x * x));
    return 0.5f * (1.f + th) + 0.5f * x * (1.f - th * th) * k0 * (1.f + 3.f * k1 * x * x);
}

}  // namespace ck
