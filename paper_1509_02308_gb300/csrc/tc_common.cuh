// Device helpers shared by the tcgen05 kernels of the learned inverse
// (conv_tc.cu at inference, train_tc.cu in the training step): shared-memory
// matrix descriptors, mbarrier waits with a time limit, MMA issue, TMEM
// loads, packed FP32 pairs and the tanh form of GELU.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>

namespace pchase {
namespace {

// every mbarrier wait gives up after 2 s of %globaltimer
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128
// bytes in 8-row atoms of 1024 bytes (stride byte offset 1024), descriptor
// version 1 (bits 46-47), layout type 2 = SWIZZLE_128B (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(16u >> 4) << 16) |
           ((uint64_t)(1024u >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    const int n = valid ? 16 : 0;  // 0: zero-fill (padding, rows past the end)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait1() {
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = globaltimer();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (globaltimer() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// tcgen05.mma .kind::f16 (BF16 operands from shared memory, FP32
// accumulator in TMEM) with instruction descriptor idesc; acc = 0 overwrites
// the accumulator, else adds to it
__device__ __forceinline__ void mma_bf16_id(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                            uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// TMA tile loads: the mbarrier expects `bytes`, the loads complete it
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
// a 2-D TMA tile load (coordinates: column, row) into shared memory,
// completing on mbarrier bar with its byte count
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// OR of v over the 256 threads that meet at named barrier bar_id
__device__ __forceinline__ bool group_any(int bar_id, bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n"
        " bar.red.or.pred p, %2, 256, q;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(bar_id)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

// Two FP32 lanes in one 64-bit register pair (low = first).  The f32x2
// forms issue one instruction for two IEEE operations with the same
// rounding as their scalar forms, so results are bit-identical.
__device__ __forceinline__ uint64_t f2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2split(uint64_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// tanh form of GELU (Hendrycks & Gimpel 2016) on both lanes, rounded to a
// BF16 pair (low lane in the low half), with the hardware tanh
// (tanh.approx.f32, relative error about 2^-11, below the BF16 output's
// 2^-8), arranged per lane as h + h tanh(x (k0 + k0 k1 x^2)), h = x / 2:
// four f32x2 operations, two tanh and one conversion per pair
__device__ __forceinline__ uint32_t gelu2_bf16(uint64_t x) {
    const float k0 = 0.7978845608028654f, k01 = 0.7978845608028654f * 0.044715f;
    const uint64_t u = mul2(x, fma2(f2(k01, k01), mul2(x, x), f2(k0, k0)));
    float u0, u1, t0, t1;
    f2split(u, u0, u1);
    asm("tanh.approx.f32 %0, %1;" : "=f"(t0) : "f"(u0));
    asm("tanh.approx.f32 %0, %1;" : "=f"(t1) : "f"(u1));
    const uint64_t h = mul2(f2(0.5f, 0.5f), x);
    float r0, r1;
    f2split(fma2(h, f2(t0, t1), h), r0, r1);
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(r1), "f"(r0));
    return d;
}

// gelu2_bf16 of 2 xh, given xh (both lanes halved exactly): with x = 2 xh,
// h = xh and u = xh (2 k0 + 8 k0 k1 xh^2), the same values as gelu2_bf16
// computes, one multiply fewer
__device__ __forceinline__ uint32_t gelu2h_bf16(uint64_t xh) {
    const float k0 = 0.7978845608028654f, k01 = 0.7978845608028654f * 0.044715f;
    const uint64_t u = mul2(xh, fma2(f2(8.0f * k01, 8.0f * k01), mul2(xh, xh), f2(2.0f * k0, 2.0f * k0)));
    float u0, u1, t0, t1;
    f2split(u, u0, u1);
    asm("tanh.approx.f32 %0, %1;" : "=f"(t0) : "f"(u0));
    asm("tanh.approx.f32 %0, %1;" : "=f"(t1) : "f"(u1));
    float r0, r1;
    f2split(fma2(xh, f2(t0, t1), xh), r0, r1);
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(r1), "f"(r0));
    return d;
}

// The tanh form of GELU (Hendrycks & Gimpel 2016), 0.5 x (1 + tanh(u)) with
// u = k0 (x + k1 x^3), written as x s with s = 1 / (1 + exp(-2u)) (the same
// function: 1 + tanh(u) = 2 / (1 + exp(-2u))), and its derivative
// s + 2 x s (1 - s) k0 (1 + 3 k1 x^2), with 1 - s = exp(-2u) s.  One ex2.approx
// and one rcp.approx (a few ulp each) per value and no cancellation in either
// tail; exp(-2u) is capped at 2^126 so that it stays finite.
__device__ __forceinline__ float gelu_sig_parts(float x, float &e) {
    const float k0 = 0.7978845608028654f, k1 = 0.044715f, log2e = 1.4426950408889634f;
    const float c0 = -2.0f * k0 * log2e, c1 = -2.0f * k0 * k1 * log2e;
    const float v = fminf(x * fmaf(c1, x * x, c0), 126.0f);  // -2u log2(e)
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(v));
    float s;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(1.0f + e));
    return s;
}
__device__ __forceinline__ float gelu_t(float x) {
    float e;
    return x * gelu_sig_parts(x, e);
}
__device__ __forceinline__ float gelu_grad_t(float x) {
    const float k0 = 0.7978845608028654f, k1 = 0.044715f;
    float e;
    const float s = gelu_sig_parts(x, e);
    return fmaf(2.0f * k0 * x * s * (e * s), fmaf(3.0f * k1, x * x, 1.0f), s);
}

}  // namespace
}  // namespace pchase
