// The learned inverse's training step (S7), backward through the four
// convolution layers (kernel 5, stride 2, zero padding 2, 64 output channels):
//
//   out[b][lo][co] = GELU(pre[b][lo][co]),
//   pre[b][lo][co] = bias[co] + sum_kk sum_ci W[co][kk*cin + ci] * x[b][2 lo + kk - 2][ci]
//
// Given dact = dL/d(out) in FP32, each layer's backward is
//
//   dz  = dact * GELU'(pre)                                  (FP32)
//   gb[co]             += sum_(b,lo) dz[b][lo][co]           (FP32)
//   gW[co][kk*cin+ci]  += sum_(b,lo) bf16(dz)[b][lo][co] * x[b][2 lo + kk - 2][ci]
//   dx[b][p][ci]        = sum_(kk,lo : 2 lo + kk - 2 = p) sum_co bf16(dz)[b][lo][co] * W[co][kk*cin + ci]
//
// with the weights' BF16 copies and the layer's BF16 inputs as operands,
// FP32 sums (the chain rule through Sec. 4.1's network; the rounding points
// are the ones the forward pass uses).
//
// The three 64-channel layers run conv_back_tc_kernel on the tcgen05 tensor
// cores.  A tile is 128 consecutive rows (b, lo), i.e. whole traces (lout is
// 128, 64 or 32), so no sum ever crosses a tile edge.  Per tile:
//   * dz from dact and pre (coalesced FP32 rows, loaded a tile ahead into
//     registers), its BF16 copy written three times into K-major
//     128-byte-swizzled operands S_j, S_j[q] = dz[q + 1 - j] (zero across a
//     trace edge);
//   * dx as two 128 x 64 sums in one N=128 accumulator: even positions
//     dx[2q] = S_0 W_0 + S_1 W_2 + S_2 W_4, odd dx[2q + 1] = S_0 W_1 + S_1 W_3,
//     with W_kk[co][ci] = W[co][kk*64 + ci] staged once per CTA as B operands
//     (row n < 64: tap 2j, n >= 64: tap 2j + 1);
//   * gW transposed, D[(kk, ci)][co] (320 rows in three M=128 tiles, N=64),
//     accumulated in TMEM over all of the CTA's tiles with K = the tile's 128
//     rows: both operands need the rows contiguous, so the layer's input
//     window (32 KB: the even and the odd positions of the tile's traces as
//     two TMA boxes, loaded a tile ahead) and dz are transposed in shared
//     memory by ldmatrix.trans (the stride-2 gather of the input rows is in
//     the ldmatrix row addresses) and stored K-major with the 128-byte swizzle.
// The third gW tile reads 64 rows past the 320 it needs (whatever lies beyond
// in shared memory): those accumulator rows are never read.  At the end each
// CTA adds its gW and gb partial sums to the gradient with FP32 atomics.
//
// The first layer (one input channel, K = 5) has no tensor-core shape and
// needs no dx: conv0_back_kernel does dz, gb and gW on CUDA cores.
//
// The forward of the 64-channel layers (conv_fwd_tc_kernel, with the
// pre-activations kept) and the FC and heads layers, forward and backward
// (tc_gemm_kernel), are further below.
//
// Completion waits on an mbarrier give up after 2 s of %globaltimer: the CTA
// then ORs PCHASE_DEV_TIMEOUT into *status, waits (again with a limit) for the
// MMAs and TMA loads it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "conv_tc.cuh"
#include "tc_common.cuh"
#include "tma_host.cuh"

namespace pchase {

namespace {

constexpr int kCh = 64;
constexpr int kTaps = 5;
constexpr int kRowsPerTile = 128;
constexpr int kBackThreads = 512;

// shared-memory layout (bytes from the 1024-aligned base)
constexpr uint32_t kOffS = 0;                       // S_0, S_1, S_2: 128 rows x 128 B each
constexpr uint32_t kOffWT = 3 * 16384;              // 3 B tiles of 128 rows (n) x 64 co
constexpr uint32_t kOffXT = kOffWT + 3 * 16384;     // 2 K atoms of 320 rows (kk, ci) x 64 rows
constexpr uint32_t kXTAtom = 320 * 128;
constexpr uint32_t kOffDZT = kOffXT + 2 * kXTAtom;  // 2 K atoms of 64 rows (co) x 64 rows
constexpr uint32_t kOffXS = kOffDZT + 2 * 8192;     // input window: 2 planes x 128 rows x 128 B
constexpr uint32_t kOffZero = kOffXS + 256 * 128;   // one zero row (padding source)
constexpr uint32_t kOffBar = kOffZero + 128;        // mbarriers (MMA, window), TMEM address
constexpr uint32_t kOffBias = kOffBar + 32;         // 64 FP32 bias partial sums
constexpr uint32_t kBackSmem = 1024 + kOffBias + 64 * 4;
static_assert(kOffXT + kXTAtom + 3 * 16384 <= kOffZero, "third gW tile reads past the window");
static_assert(kBackSmem <= 232448, "shared memory");

// tcgen05 instruction descriptors (FP32 accumulator, BF16 A and B, both
// K-major, M = 128): N = 128 for dx, N = 64 for gW
constexpr uint32_t idesc_n(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}
constexpr uint32_t kIdescDx = idesc_n(128);
constexpr uint32_t kIdescGw = idesc_n(64);
constexpr uint32_t kBackTmemCols = 512;  // dx 128 + gW 3 x 64, rounded to a power of two

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t &r0, uint32_t &r1,
                                              uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ void st_shared_b32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// byte offset of 16-byte chunk c of row r in a K-major operand whose rows are
// 128 bytes (64 BF16) with the 128-byte swizzle
__device__ __forceinline__ uint32_t sw_chunk(uint32_t r, uint32_t c) {
    return r * 128u + ((c ^ (r & 7u)) << 4);
}


template <int LOUT>
__global__ void __launch_bounds__(kBackThreads, 1)
    conv_back_tc_kernel(const float *__restrict__ dact, const float *__restrict__ pre,
                        const __grid_constant__ CUtensorMap xmap, const __nv_bfloat16 *__restrict__ W,
                        int nb, float *__restrict__ gW, float *__restrict__ gb,
                        float *__restrict__ dx, uint32_t *status) {
    constexpr int lout = LOUT;
    extern __shared__ uint8_t dsm[];
    const uint32_t raw = smem_u32(dsm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *const gbase = dsm + (base - raw);
    const uint32_t sS = base + kOffS, sWT = base + kOffWT, sXT = base + kOffXT;
    const uint32_t sDZT = base + kOffDZT, sXS = base + kOffXS, sZero = base + kOffZero;
    const uint32_t sBar = base + kOffBar;
    const uint32_t sXBar = sBar + 8;  // the window's TMA loads
    uint32_t *const tslot = reinterpret_cast<uint32_t *>(gbase + kOffBar + 16);
    float *const sbias = reinterpret_cast<float *>(gbase + kOffBias);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lin = 2 * lout;
    const int nrows = nb * lout;
    const int ntiles = (nrows + kRowsPerTile - 1) / kRowsPerTile;
    const int tpt = kRowsPerTile / lout;  // traces per tile

    // B operands of dx: tile j, row n = (tap 2j + n / 64, ci = n % 64), K = co
    for (int e = tid; e < 3 * 128 * 8; e += kBackThreads) {
        const int j = e >> 10, n = (e >> 3) & 127, c = e & 7;
        const int kk = 2 * j + (n >> 6), ci = n & 63;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (kk < kTaps) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int co = c * 8 + 2 * q;
                const __nv_bfloat16 a = W[(size_t)co * (kTaps * kCh) + kk * kCh + ci];
                const __nv_bfloat16 b = W[(size_t)(co + 1) * (kTaps * kCh) + kk * kCh + ci];
                w[q] = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
            }
        }
        st_shared_v4(sWT + (uint32_t)j * 16384u + sw_chunk((uint32_t)n, (uint32_t)c),
                     make_uint4(w[0], w[1], w[2], w[3]));
    }
    if (tid < 8) st_shared_v4(sZero + 16u * (uint32_t)tid, make_uint4(0u, 0u, 0u, 0u));
    if (tid < kCh) sbias[tid] = 0.0f;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sBar) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sXBar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(kBackTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    const int c = tid & 7;  // the 8 channels this thread takes in the dz phase
    float bacc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) bacc[e] = 0.0f;
    int it = 0;
    bool timed_out = false;
    // ---- the input window of tile t's traces as two TMA boxes, the even and
    // the odd positions: row tb * LOUT + pr of plane pl holds position
    // 2 pr + pl of trace t * tpt + tb (128-byte swizzle; traces past the batch
    // read as zeros).  One thread issues them; every thread waits on the
    // window's mbarrier before the transposes.
    int windows = 0;  // window loads issued
    auto fetch_window = [&](int t) {
        if (t < ntiles) {
            if (tid == 0) {
                mbar_expect_tx(sXBar, 2u * 16384u);
                tma_load_4d(sXS, &xmap, 0, 0, 0, t * tpt, sXBar);
                tma_load_4d(sXS + 16384u, &xmap, 0, 1, 0, t * tpt, sXBar);
            }
            ++windows;
        }
    };
    // ---- this thread's dact and pre of tile t (rows r0 + 32 i, channels
    // 8c .. 8c + 7), loaded a tile ahead
    float4 fa[2][2], fp[2][2];
    auto fetch_rows = [&](int t) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int grow = t * kRowsPerTile + (tid >> 3) + 64 * i;
            if (t < ntiles && grow < nrows) {
                const float4 *da = reinterpret_cast<const float4 *>(dact + (size_t)grow * kCh + c * 8);
                const float4 *pa = reinterpret_cast<const float4 *>(pre + (size_t)grow * kCh + c * 8);
                fa[i][0] = __ldg(da);
                fa[i][1] = __ldg(da + 1);
                fp[i][0] = __ldg(pa);
                fp[i][1] = __ldg(pa + 1);
            } else {
                fa[i][0] = fa[i][1] = fp[i][0] = fp[i][1] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
    fetch_window(blockIdx.x);
    fetch_rows(blockIdx.x);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int row0 = t * kRowsPerTile;
        // ---- dz into S_0, S_1, S_2 (rows past the end hold zeros)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = (tid >> 3) + 64 * i;
            const int grow = row0 + r;
            float d[8];
            if (grow < nrows) {
                const float4 a0 = fa[i][0], a1 = fa[i][1], p0 = fp[i][0], p1 = fp[i][1];
                d[0] = a0.x * gelu_grad_t(p0.x);
                d[1] = a0.y * gelu_grad_t(p0.y);
                d[2] = a0.z * gelu_grad_t(p0.z);
                d[3] = a0.w * gelu_grad_t(p0.w);
                d[4] = a1.x * gelu_grad_t(p1.x);
                d[5] = a1.y * gelu_grad_t(p1.y);
                d[6] = a1.z * gelu_grad_t(p1.z);
                d[7] = a1.w * gelu_grad_t(p1.w);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) d[e] = 0.0f;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) bacc[e] += d[e];
            const uint4 v = make_uint4(pack_bf16(d[0], d[1]), pack_bf16(d[2], d[3]),
                                       pack_bf16(d[4], d[5]), pack_bf16(d[6], d[7]));
            const uint4 z = make_uint4(0u, 0u, 0u, 0u);
            const int lo = r % lout;
            st_shared_v4(sS + 16384u + sw_chunk((uint32_t)r, (uint32_t)c), v);
            // S_0[q] = dz[q + 1]
            if (lo != 0) st_shared_v4(sS + sw_chunk((uint32_t)(r - 1), (uint32_t)c), v);
            if (lo == lout - 1) st_shared_v4(sS + sw_chunk((uint32_t)r, (uint32_t)c), z);
            // S_2[q] = dz[q - 1]
            if (lo != lout - 1) st_shared_v4(sS + 32768u + sw_chunk((uint32_t)(r + 1), (uint32_t)c), v);
            if (lo == 0) st_shared_v4(sS + 32768u + sw_chunk((uint32_t)r, (uint32_t)c), z);
        }
        const bool wok = mbar_wait(sXBar, (uint32_t)(windows - 1) & 1u);
        if (__syncthreads_or(!wok)) {
            timed_out = true;
            break;
        }
        // ---- transposes by ldmatrix.trans: 8 x 8 blocks of (8 channels) x
        // (8 rows), four per instruction (channel chunks 4g .. 4g + 3).  A
        // thread receives, per block, channel 8 cc + lane / 4 of rows
        // 8 rb + 2 (lane % 4) and the next, stored as one 32-bit word.
        {
            const int mi = lane >> 3, j = lane & 7;
            // input windows: XT[(kk, ci)][row], row = (b, lo) of the tile,
            // = x[b][2 lo + kk - 2][ci] (zero outside the trace)
            for (int u = warp; u < kTaps * 2 * 16; u += kBackThreads / 32) {
                const int kk = u / 32, g = (u >> 4) & 1, rb = u & 15;
                const int r = rb * 8 + j, tb = r / lout, lo = r % lout;
                // position 2 lo + kk - 2 = 2 pr + kk % 2
                const int pr = lo + (kk >> 1) - 1;
                const int cc = 4 * g + mi;
                uint32_t src = sZero;
                if (pr >= 0 && pr < lout)
                    src = sXS + (uint32_t)(kk & 1) * 16384u +
                          sw_chunk((uint32_t)(tb * lout + pr), (uint32_t)cc);
                uint32_t v[4];
                ldsm_x4_trans(src, v[0], v[1], v[2], v[3]);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t m = (uint32_t)(kk * kCh + (4 * g + q) * 8 + (lane >> 2));
                    st_shared_b32(sXT + (uint32_t)(rb >> 3) * kXTAtom + m * 128u +
                                      ((((uint32_t)rb & 7u) ^ (m & 7u)) << 4) + 4u * (lane & 3),
                                  v[q]);
                }
            }
            // dz: DZT[co][row] from S_1
            for (int u = warp; u < 2 * 16; u += kBackThreads / 32) {
                const int g = u >> 4, rb = u & 15;
                const uint32_t q0 = (uint32_t)(rb * 8 + j);
                uint32_t v[4];
                ldsm_x4_trans(sS + 16384u + sw_chunk(q0, (uint32_t)(4 * g + mi)), v[0], v[1], v[2],
                              v[3]);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t co = (uint32_t)((4 * g + q) * 8 + (lane >> 2));
                    st_shared_b32(sDZT + (uint32_t)(rb >> 3) * 8192u + co * 128u +
                                      ((((uint32_t)rb & 7u) ^ (co & 7u)) << 4) + 4u * (lane & 3),
                                  v[q]);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- MMAs (one thread): dx into columns 0..127, gW into 128 + 64 mt
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    mma_bf16_id(tmem, sw128_desc(sS + (uint32_t)j * 16384u + 32u * s),
                                sw128_desc(sWT + (uint32_t)j * 16384u + 32u * s), kIdescDx,
                                (j | s) != 0 ? 1u : 0u);
#pragma unroll
            for (int mt = 0; mt < 3; ++mt)
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int s = 0; s < 4; ++s)
                        mma_bf16_id(tmem + 128u + 64u * (uint32_t)mt,
                                    sw128_desc(sXT + (uint32_t)a * kXTAtom + (uint32_t)mt * 16384u + 32u * s),
                                    sw128_desc(sDZT + (uint32_t)a * 8192u + 32u * s), kIdescGw,
                                    (it | a | s) != 0 ? 1u : 0u);
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sBar)
                : "memory");
        }
        // the next tile's loads fly during the MMAs and the epilogue (the
        // window's buffer was last read by the transposes above)
        fetch_window(t + gridDim.x);
        fetch_rows(t + gridDim.x);
        const bool ok = mbar_wait(sBar, (uint32_t)it & 1u);
        tc_fence_after();
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            ++it;
            break;
        }
        // ---- dx epilogue: warp w reads lanes 32 (w % 4) .. (rows q) and
        // columns 32 (w / 4) .. +31: even positions for w / 4 < 2, odd after
        {
            const int lg = warp & 3, qq = warp >> 2, h = qq >> 1;
            const int q = 32 * lg + lane;
            uint32_t v[2][16];
#pragma unroll
            for (int k = 0; k < 2; ++k)
                tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(32 * qq + 16 * k), v[k]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int grow = row0 + q;
            if (grow < nrows) {
                const int b = grow / lout, lo = grow % lout;
                float4 *o = reinterpret_cast<float4 *>(dx + ((size_t)b * lin + 2 * lo + h) * kCh +
                                                       32 * (qq & 1));
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        o[4 * k + e] = make_float4(__uint_as_float(v[k][4 * e]),
                                                   __uint_as_float(v[k][4 * e + 1]),
                                                   __uint_as_float(v[k][4 * e + 2]),
                                                   __uint_as_float(v[k][4 * e + 3]));
            }
        }
        tc_fence_before();
    }
    // ---- partial sums into the gradient
#pragma unroll
    for (int e = 0; e < 8; ++e) atomicAdd(&sbias[c * 8 + e], bacc[e]);
    if (it > 0 && !timed_out) {
        const int lg = warp & 3;
        for (int u = warp >> 2; u < 6; u += kBackThreads / 128) {
            const int mt = u >> 1, hh = u & 1;
            uint32_t v[2][16];
            tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + 128u + 64u * (uint32_t)mt + 32u * hh, v[0]);
            tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + 128u + 64u * (uint32_t)mt + 32u * hh + 16u,
                      v[1]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int m = mt * 128 + 32 * lg + lane;
            if (m < kTaps * kCh) {
                const int kk = m >> 6, ci = m & 63;
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int co = 32 * hh + 16 * k + e;
                        atomicAdd(gW + (size_t)co * (kTaps * kCh) + kk * kCh + ci,
                                  __uint_as_float(v[k][e]));
                    }
            }
        }
    }
    if (timed_out && tid == 0) {
        // the last MMAs and window loads land before TMEM is freed and the CTA leaves
        if (it > 0) mbar_wait(sBar, (uint32_t)(it - 1) & 1u);
        if (windows > 0) mbar_wait(sXBar, (uint32_t)(windows - 1) & 1u);
        atomicOr(status, PCHASE_DEV_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < kCh) atomicAdd(gb + tid, sbias[tid]);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kBackTmemCols)
                     : "memory");
}

// First layer (one input channel): dact, pre [nb * 256][64] FP32, x [nb][512]
// BF16.  A CTA takes whole traces (a grid-stride loop): the trace's inputs
// are staged in shared memory and thread t takes channels 8 (t % 8) .. +7 at
// positions 8 (t / 8) .. +7, two positions' dact and pre (eight 16-byte
// loads) in flight at a time.  Partial sums stay in registers over all of the
// CTA's traces, then meet across the warp (shuffles), in shared memory, and
// in one atomic per value and CTA.
__global__ void __launch_bounds__(256) conv0_back_kernel(const float *__restrict__ dact,
                                                         const float *__restrict__ pre,
                                                         const __nv_bfloat16 *__restrict__ x,
                                                         int nb, float *__restrict__ gW,
                                                         float *__restrict__ gb) {
    constexpr int kLout = 256, kLin = 512;
    __shared__ float xs[kLin + 8];  // xs[q + 2] = x[q], zeros outside
    __shared__ float sw[kCh * kTaps], sb[kCh];
    const int t = threadIdx.x, c = t & 7, p0 = (t >> 3) * 8;
    for (int e = t; e < kCh * kTaps; e += blockDim.x) sw[e] = 0.0f;
    if (t < kCh) sb[t] = 0.0f;
    float aw[8][kTaps], ab[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        ab[e] = 0.0f;
#pragma unroll
        for (int k = 0; k < kTaps; ++k) aw[e][k] = 0.0f;
    }
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        __syncthreads();  // the previous trace's reads are done
        for (int q = t; q < kLin + 8; q += blockDim.x) {
            const int src = q - 2;
            xs[q] = (src >= 0 && src < kLin) ? __bfloat162float(x[(size_t)b * kLin + src]) : 0.0f;
        }
        __syncthreads();
#pragma unroll 1
        for (int i = 0; i < 8; i += 2) {
            float4 a[2][2], pr[2][2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const size_t row = (size_t)b * kLout + p0 + i + h;
                const float4 *da = reinterpret_cast<const float4 *>(dact + row * kCh + c * 8);
                const float4 *pa = reinterpret_cast<const float4 *>(pre + row * kCh + c * 8);
                a[h][0] = __ldg(da);
                a[h][1] = __ldg(da + 1);
                pr[h][0] = __ldg(pa);
                pr[h][1] = __ldg(pa + 1);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int p = p0 + i + h;
                float xv[kTaps];
#pragma unroll
                for (int k = 0; k < kTaps; ++k) xv[k] = xs[2 * p + k];  // x[2p + k - 2]
                const float av[8] = {a[h][0].x, a[h][0].y, a[h][0].z, a[h][0].w,
                                     a[h][1].x, a[h][1].y, a[h][1].z, a[h][1].w};
                const float pv[8] = {pr[h][0].x, pr[h][0].y, pr[h][0].z, pr[h][0].w,
                                     pr[h][1].x, pr[h][1].y, pr[h][1].z, pr[h][1].w};
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float d = av[e] * gelu_grad_t(pv[e]);
                    ab[e] += d;
                    const float db = __bfloat162float(__float2bfloat16(d));
#pragma unroll
                    for (int k = 0; k < kTaps; ++k) aw[e][k] = fmaf(db, xv[k], aw[e][k]);
                }
            }
        }
    }
    // lanes l, l ^ 8, l ^ 16, l ^ 24 hold the same channels
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        ab[e] += __shfl_xor_sync(0xffffffffu, ab[e], 8);
        ab[e] += __shfl_xor_sync(0xffffffffu, ab[e], 16);
#pragma unroll
        for (int k = 0; k < kTaps; ++k) {
            aw[e][k] += __shfl_xor_sync(0xffffffffu, aw[e][k], 8);
            aw[e][k] += __shfl_xor_sync(0xffffffffu, aw[e][k], 16);
        }
    }
    __syncthreads();
    if ((t & 31) < 8) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            atomicAdd(&sb[c * 8 + e], ab[e]);
#pragma unroll
            for (int k = 0; k < kTaps; ++k) atomicAdd(&sw[(c * 8 + e) * kTaps + k], aw[e][k]);
        }
    }
    __syncthreads();
    for (int e = t; e < kCh * kTaps; e += blockDim.x) atomicAdd(gW + e, sw[e]);
    if (t < kCh) atomicAdd(gb + t, sb[t]);
}

// ------------------------------------------------------- forward (training)
// One 64-channel layer with the pre-activations kept for the backward pass:
// pre[row][co] = bias[co] + sum_kk sum_ci W[co][kk*64 + ci] x[b][2 lo + kk - 2][ci]
// (FP32) and out[row][co] = BF16(GELU(pre)), row = (b, lo).  A tile is 128 rows
// (whole traces).  Its five tap operands A_kk[row][ci] = x[b][2 lo + kk - 2][ci]
// are TMA tile loads: x is described as a 4-D tensor (channel, parity, pair,
// trace) = x[trace][2 pair + parity][channel], and tap kk is the box
// (64 channels, parity kk % 2, pairs kk / 2 - 1 .. + LOUT - 1, the tile's
// traces), 128 rows of 128 bytes with the 128-byte swizzle, i.e. a K-major
// operand as the MMA reads it; pairs outside the trace (the zero padding)
// and traces past the batch are out of the tensor and read as zeros.  One
// thread issues the next tile's five loads (one mbarrier with the byte
// count) while this tile's MMAs and epilogue run.  The weights W_kk[co][ci] are
// five B tiles loaded once.  20 MMAs (M128 N64 K16) per tile.
constexpr int kFwdThreads = 512;
constexpr uint32_t kFwdW = 5 * 8192;             // B tiles: 64 rows x 128 B per tap
constexpr uint32_t kFwdA = 5 * 16384;            // A tiles of one tile: 128 rows x 128 B per tap
constexpr uint32_t kFwdSmem = 1024 + kFwdW + 2 * kFwdA + 64;
static_assert(kFwdSmem <= 232448, "shared memory");

template <int LOUT>
__global__ void __launch_bounds__(kFwdThreads, 1)
    conv_fwd_tc_kernel(const __grid_constant__ CUtensorMap xmap, int nb,
                       const __nv_bfloat16 *__restrict__ W, const float *__restrict__ bias,
                       float *__restrict__ pre, __nv_bfloat16 *__restrict__ out,
                       uint32_t *status) {
    constexpr int tpt = kRowsPerTile / LOUT;
    extern __shared__ uint8_t dsm[];
    const uint32_t raw = smem_u32(dsm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *const gbase = dsm + (base - raw);
    const uint32_t sW = base, sA = base + kFwdW;
    // mbarriers: MMA done [2] at sBar + 8s, operands loaded [2] at sBar + 16 + 8s
    const uint32_t sBar = base + kFwdW + 2 * kFwdA;
    uint32_t *const tslot = reinterpret_cast<uint32_t *>(gbase + kFwdW + 2 * kFwdA + 32);
    volatile uint32_t *const abort_flag = tslot + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nrows = nb * LOUT;
    const int ntiles = (nrows + kRowsPerTile - 1) / kRowsPerTile;
    const int lg = warp & 3, qq = warp >> 2;  // epilogue: TMEM lanes 32 lg.., channels 16 qq..
    float bq[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) bq[e] = __ldg(bias + 16 * qq + e);

    for (int e = tid; e < kTaps * kCh * 8; e += kFwdThreads) {
        const int kk = e >> 9, co = (e >> 3) & 63, c = e & 7;
        cp_async16(sW + (uint32_t)kk * 8192u + sw_chunk((uint32_t)co, (uint32_t)c),
                   W + (size_t)co * (kTaps * kCh) + kk * kCh + c * 8, true);
    }
    cp_async_commit();
    // the five tap boxes of tile t into buffer s (one thread)
    auto load = [&](int t, int s) {
        const uint32_t bar = sBar + 16u + 8u * (uint32_t)s;
        mbar_expect_tx(bar, kFwdA);
#pragma unroll
        for (int kk = 0; kk < kTaps; ++kk)
            tma_load_4d(sA + (uint32_t)s * kFwdA + (uint32_t)kk * 16384u, &xmap, 0, kk & 1,
                        (kk >> 1) - 1, t * tpt, bar);
    };
    if (tid == 0) {
        for (int q = 0; q < 4; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sBar + 8 * q) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
        if ((int)blockIdx.x < ntiles) load(blockIdx.x, 0);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    cp_async_wait_all();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    bool ok = true;
    int j = 0, last_load = (int)blockIdx.x < ntiles ? 0 : -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
        const int s = j & 1;
        if (j > 0) {
            // every thread is done with the previous tile's accumulator
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
        if (tid == 0) {
            // buffer s ^ 1 was last read by tile j - 1's MMAs, complete
            if (t + (int)gridDim.x < ntiles) {
                load(t + gridDim.x, s ^ 1);
                last_load = j + 1;
            }
            if (mbar_wait(sBar + 16u + 8u * (uint32_t)s, (uint32_t)(j >> 1) & 1u)) {
                tc_fence_after();
                const uint32_t a0 = sA + (uint32_t)s * kFwdA;
#pragma unroll
                for (int kk = 0; kk < kTaps; ++kk)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        mma_bf16_id(tmem + 64u * (uint32_t)s,
                                    sw128_desc(a0 + (uint32_t)kk * 16384u + 32u * q),
                                    sw128_desc(sW + (uint32_t)kk * 8192u + 32u * q), kIdescGw,
                                    (kk | q) != 0 ? 1u : 0u);
            } else {
                *abort_flag = 1;
            }
            // the commit arrives even without MMAs, so no thread waits in vain
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    sBar + 8u * (uint32_t)s)
                : "memory");
        }
        const bool got = mbar_wait(sBar + 8u * (uint32_t)s, (uint32_t)(j >> 1) & 1u);
        tc_fence_after();
        if (__syncthreads_or(!got || *abort_flag != 0)) {
            ok = false;
            break;
        }
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + 64u * (uint32_t)s + 16u * (uint32_t)qq, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int grow = t * kRowsPerTile + 32 * lg + lane;
        if (grow < nrows) {
            float4 *po = reinterpret_cast<float4 *>(pre + (size_t)grow * kCh + 16 * qq);
            uint4 *ao = reinterpret_cast<uint4 *>(out + (size_t)grow * kCh + 16 * qq);
            float y[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) y[e] = __uint_as_float(v[e]) + bq[e];
#pragma unroll
            for (int e = 0; e < 4; ++e)
                po[e] = make_float4(y[4 * e], y[4 * e + 1], y[4 * e + 2], y[4 * e + 3]);
            ao[0] = make_uint4(pack_bf16(gelu_t(y[0]), gelu_t(y[1])), pack_bf16(gelu_t(y[2]), gelu_t(y[3])),
                               pack_bf16(gelu_t(y[4]), gelu_t(y[5])), pack_bf16(gelu_t(y[6]), gelu_t(y[7])));
            ao[1] = make_uint4(pack_bf16(gelu_t(y[8]), gelu_t(y[9])), pack_bf16(gelu_t(y[10]), gelu_t(y[11])),
                               pack_bf16(gelu_t(y[12]), gelu_t(y[13])), pack_bf16(gelu_t(y[14]), gelu_t(y[15])));
        }
    }
    if (!ok && tid == 0) {
        atomicOr(status, PCHASE_DEV_TIMEOUT);
        // loads and MMAs still in flight land before the CTA leaves
        if (last_load >= j)
            mbar_wait(sBar + 16u + 8u * (uint32_t)(last_load & 1), (uint32_t)(last_load >> 1) & 1u);
        mbar_wait(sBar + 8u * (uint32_t)(j & 1), (uint32_t)(j >> 1) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u)
                     : "memory");
}

// ------------------------------------------------------------------ GEMM
// C = A B^T over K for the training step's dense layers: A [M][K] and B [N][K]
// BF16, both K-major (row strides lda, ldb elements, multiples of 8, 16-byte
// aligned bases), FP32 sums in TMEM.  A CTA takes a 128 x BN tile and a slice
// of the K blocks (gridDim.z slices of 64-element blocks).  One thread runs
// the main loop: both operands' 64-column blocks are TMA tile loads (2-D
// tensor maps, 128-byte swizzle; rows past M or N and columns past K are out
// of the tensor and read as zeros) into a 4-stage ring, three blocks ahead;
// a stage's mbarrier counts its bytes in, and a second one (tcgen05.commit)
// frees it once its MMAs are done.  Epilogues: kStore (C[m][n], or C[n][m] when transposed,
// + bias[n] if given; FP32 atomics when K is sliced) and kGelu (v = sum +
// bias[n]: pre[m][n] = v, Cb[m][n] = BF16(GELU(v)) with the exact tanh).
constexpr int kGemmStages = 4;
enum GemmEpi { kStore = 0, kGelu = 1 };

struct TcGemm {
    const __nv_bfloat16 *A, *B;
    int M, N, K, lda, ldb;
    int blocks_per_slice;  // K blocks of 64 per blockIdx.z
    const float *bias;
    float *C;              // kStore
    int ldc, atomic, transposed;
    float *pre;            // kGelu
    __nv_bfloat16 *Cb;
    uint32_t *status;
};

template <int BN>
struct GemmShape {
    static constexpr uint32_t kABytes = 128 * 128, kBBytes = BN * 128;
    static constexpr uint32_t kStageBytes = kABytes + kBBytes;
    static constexpr uint32_t kSmem = 1024 + kGemmStages * kStageBytes + 16 * kGemmStages + 16;
    static constexpr uint32_t kTmemCols = BN < 32 ? 32 : BN;
    static_assert(4 * 32 * (BN + 1) * 4 <= kGemmStages * kStageBytes, "epilogue staging");
    static constexpr uint32_t kIdesc = idesc_n(BN);
};

template <int BN, int EPI>
__global__ void __launch_bounds__(128)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
                   const TcGemm g) {
    using S = GemmShape<BN>;
    extern __shared__ uint8_t dsm[];
    const uint32_t raw = smem_u32(dsm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *const gbase = dsm + (base - raw);
    // mbarriers: stage loaded [S] at sBar + 8s, stage's MMAs done [S] at sBar + 8 (S + s)
    const uint32_t sBar = base + kGemmStages * S::kStageBytes;
    uint32_t *const tslot =
        reinterpret_cast<uint32_t *>(gbase + kGemmStages * S::kStageBytes + 16 * kGemmStages);
    volatile uint32_t *const abort_flag = tslot + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
    const int nkb = (g.K + 63) / 64;
    const int kb0 = blockIdx.z * g.blocks_per_slice;
    const int nblk = max(0, min(nkb, kb0 + g.blocks_per_slice) - kb0);
    const uint32_t full0 = sBar, done0 = sBar + 8u * kGemmStages;

    // block j's A and B tiles into stage j mod S (one thread)
    auto load = [&](int j) {
        const uint32_t q = (uint32_t)(j % kGemmStages);
        const uint32_t st = base + q * S::kStageBytes;
        const int k0 = (kb0 + j) * 64;
        mbar_expect_tx(full0 + 8u * q, S::kStageBytes);
        tma_load_2d(st, &amap, k0, m0, full0 + 8u * q);
        tma_load_2d(st + S::kABytes, &bmap, k0, n0, full0 + 8u * q);
    };
    if (tid == 0) {
        for (int q = 0; q < 2 * kGemmStages; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sBar + 8 * q) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(S::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    int loaded = 0;  // blocks whose loads went out (thread 0)
    if (tid == 0) {
        for (; loaded < min(nblk, kGemmStages - 1); ++loaded) load(loaded);
        for (int j = 0; j < nblk; ++j) {
            const uint32_t q = (uint32_t)(j % kGemmStages);
            if (!mbar_wait(full0 + 8u * q, (uint32_t)(j / kGemmStages) & 1u)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t st = base + q * S::kStageBytes;
#pragma unroll
            for (int s = 0; s < 4; ++s)
                mma_bf16_id(tmem, sw128_desc(st + 32u * s), sw128_desc(st + S::kABytes + 32u * s),
                            S::kIdesc, (j | s) != 0 ? 1u : 0u);
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    done0 + 8u * q)
                : "memory");
            // the stage of block j - 1 (its MMAs went out a step ago) takes block j + S - 1
            if (loaded < nblk) {
                const int pj = loaded - kGemmStages;  // the last block that used the stage
                if (pj >= 0 && !mbar_wait(done0 + 8u * (uint32_t)(pj % kGemmStages),
                                          (uint32_t)(pj / kGemmStages) & 1u)) {
                    *abort_flag = 1;
                    break;
                }
                load(loaded++);
            }
        }
    }
    __syncthreads();
    bool ok = *abort_flag == 0;
    if (ok && nblk > 0) {
        const int lb = nblk - 1;  // the last commit covers every earlier MMA
        const bool got = mbar_wait(done0 + 8u * (uint32_t)(lb % kGemmStages), (uint32_t)(lb / kGemmStages) & 1u);
        ok = __syncthreads_and(got);
        if (ok && g.transposed) {
            // C[n][m]: lanes hold consecutive m, so each store is coalesced
            tc_fence_after();
            const int m = m0 + warp * 32 + lane;  // TMEM lane = tile row
#pragma unroll 1
            for (int q = 0; q < BN / 16; ++q) {
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(16 * q), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (m >= g.M) continue;
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int n = n0 + 16 * q + e;
                    if (n >= g.N) break;
                    float val = __uint_as_float(v[e]);
                    if (g.bias) val += __ldg(g.bias + n);
                    float *dst = g.C + (size_t)n * g.ldc + m;
                    if (g.atomic) atomicAdd(dst, val);
                    else *dst = val;
                }
            }
        } else if (ok) {
            // row-major C: each warp stages its 32 rows in shared memory (the
            // ring, idle now; row stride BN + 1 words, no bank conflicts) and
            // writes them back a row at a time, 32 consecutive columns per
            // store
            tc_fence_after();
            float *stage = reinterpret_cast<float *>(gbase) + warp * 32 * (BN + 1);
#pragma unroll 1
            for (int q = 0; q < BN / 16; ++q) {
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(16 * q), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int e = 0; e < 16; ++e) stage[lane * (BN + 1) + 16 * q + e] = __uint_as_float(v[e]);
            }
            __syncwarp();
            for (int rr = 0; rr < 32; ++rr) {
                const int m = m0 + warp * 32 + rr;
                if (m >= g.M) break;
#pragma unroll
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    const int n = n0 + c0 + lane;
                    if (n >= g.N) continue;
                    float val = stage[rr * (BN + 1) + c0 + lane];
                    if (g.bias) val += __ldg(g.bias + n);
                    const size_t o = (size_t)m * g.ldc + n;
                    if (EPI == kGelu) {
                        g.pre[o] = val;
                        g.Cb[o] = __float2bfloat16(gelu_t(val));
                    } else if (g.atomic) {
                        atomicAdd(g.C + o, val);
                    } else {
                        g.C[o] = val;
                    }
                }
            }
        }
    }
    if (!ok && tid == 0) {
        atomicOr(g.status, PCHASE_DEV_TIMEOUT);
        // the loads and MMAs issued land before TMEM is freed and the CTA leaves
        for (int j = max(0, loaded - kGemmStages); j < loaded; ++j)
            mbar_wait(full0 + 8u * (uint32_t)(j % kGemmStages), (uint32_t)(j / kGemmStages) & 1u);
        if (loaded > 0)
            mbar_wait(done0 + 8u * (uint32_t)((loaded - 1) % kGemmStages),
                      (uint32_t)((loaded - 1) / kGemmStages) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(S::kTmemCols)
                     : "memory");
}

// out[c][r] = in[r][c] for r < R, c < C (out row stride ldo); columns R ..
// ldo - 1 of each out row and rows C .. Cpad - 1 are zero.  32 x 32 tiles
// through shared memory.
__global__ void transpose_bf16_kernel(const __nv_bfloat16 *__restrict__ in, int R, int C, int ldi,
                                      __nv_bfloat16 *__restrict__ out, int ldo, int Cpad) {
    __shared__ __nv_bfloat16 t[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    for (int i = ty; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + tx;
        t[i][tx] = (r < R && c < C) ? in[(size_t)r * ldi + c] : __float2bfloat16(0.0f);
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + tx;
        if (c < Cpad && r < ldo) out[(size_t)c * ldo + r] = t[tx][i];
    }
}

template <int BN, int EPI>
cudaError_t launch_tc_gemm(const TcGemm &g, int slices, cudaStream_t st) {
    using S = GemmShape<BN>;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(
            tc_gemm_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    alignas(64) CUtensorMap amap, bmap;
    if (!kmajor_map(g.A, g.M, g.K, g.lda, 128, &amap) || !kmajor_map(g.B, g.N, g.K, g.ldb, BN, &bmap))
        return cudaErrorInvalidValue;
    dim3 grid((g.M + 127) / 128, (g.N + BN - 1) / BN, slices);
    tc_gemm_kernel<BN, EPI><<<grid, 128, S::kSmem, st>>>(amap, bmap, g);
    return cudaGetLastError();
}

}  // namespace

// x [nb][2 lout][64] BF16 as the 4-D tensor (channel, parity, pair, trace)
// with boxes of 64 channels x 1 parity x lout pairs x (128 / lout) traces,
// 128-byte swizzle: the rows of one parity plane of a 128-row tile
static cudaError_t x_plane_map(const __nv_bfloat16 *x, int nb, int lout, CUtensorMap *map) {
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {(cuuint64_t)kCh, 2, (cuuint64_t)lout, (cuuint64_t)nb};
    const cuuint64_t strides[3] = {kCh * 2, 2 * kCh * 2, (cuuint64_t)lout * 2 * kCh * 2};
    const cuuint32_t box[4] = {(cuuint32_t)kCh, 1, (cuuint32_t)lout,
                               (cuuint32_t)(kRowsPerTile / lout)};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(x), dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t conv_back_tc(const float *dact, const float *pre, const __nv_bfloat16 *x, int nb,
                         int lout, const __nv_bfloat16 *W, float *gW, float *gb, float *dx,
                         uint32_t *status, int sms, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    if (lout != 128 && lout != 64 && lout != 32) return cudaErrorInvalidValue;
    if (reinterpret_cast<uintptr_t>(x) & 15) return cudaErrorInvalidValue;
    alignas(64) CUtensorMap map;
    const cudaError_t me = x_plane_map(x, nb, lout, &map);
    if (me != cudaSuccess) return me;
    static bool attr = false;
    if (!attr) {
        for (auto k : {conv_back_tc_kernel<128>, conv_back_tc_kernel<64>, conv_back_tc_kernel<32>}) {
            const cudaError_t e =
                cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBackSmem);
            if (e != cudaSuccess) return e;
        }
        attr = true;
    }
    const int ntiles = (nb * lout + kRowsPerTile - 1) / kRowsPerTile;
    const int grid = std::max(1, std::min(ntiles, sms));
    if (lout == 128)
        conv_back_tc_kernel<128><<<grid, kBackThreads, kBackSmem, st>>>(dact, pre, map, W, nb, gW, gb, dx, status);
    else if (lout == 64)
        conv_back_tc_kernel<64><<<grid, kBackThreads, kBackSmem, st>>>(dact, pre, map, W, nb, gW, gb, dx, status);
    else
        conv_back_tc_kernel<32><<<grid, kBackThreads, kBackSmem, st>>>(dact, pre, map, W, nb, gW, gb, dx, status);
    return cudaGetLastError();
}

cudaError_t conv0_back(const float *dact, const float *pre, const __nv_bfloat16 *x, int nb,
                       float *gW, float *gb, int sms, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    const int grid = std::max(1, std::min(nb, sms * 4));
    conv0_back_kernel<<<grid, 256, 0, st>>>(dact, pre, x, nb, gW, gb);
    return cudaGetLastError();
}

cudaError_t tc_gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N,
                    int K, int bn, int k_slices, const float *bias, float *C, int ldc, bool atomic,
                    bool transposed, float *pre, __nv_bfloat16 *Cb, uint32_t *status,
                    cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (lda % 8 || ldb % 8 || (reinterpret_cast<uintptr_t>(A) & 15) ||
        (reinterpret_cast<uintptr_t>(B) & 15))
        return cudaErrorInvalidValue;
    TcGemm g{A, B, M, N, K, lda, ldb, 0, bias, C, ldc, atomic ? 1 : 0, transposed ? 1 : 0,
             pre, Cb, status};
    const int nkb = (K + 63) / 64;
    const int slices = std::max(1, std::min(k_slices, nkb));
    g.blocks_per_slice = (nkb + slices - 1) / slices;
    if (slices > 1 && !atomic && !pre) return cudaErrorInvalidValue;
    if (pre) {
        if (slices > 1 || !Cb) return cudaErrorInvalidValue;
        if (bn == 64) return launch_tc_gemm<64, kGelu>(g, 1, st);
        return cudaErrorInvalidValue;
    }
    if (bn == 32) return launch_tc_gemm<32, kStore>(g, slices, st);
    if (bn == 128) return launch_tc_gemm<128, kStore>(g, slices, st);
    return cudaErrorInvalidValue;
}

cudaError_t transpose_bf16(const __nv_bfloat16 *in, int R, int C, int ldi, __nv_bfloat16 *out,
                           int ldo, int Cpad, cudaStream_t st) {
    if (R <= 0 || Cpad <= 0) return cudaSuccess;
    dim3 grid((std::max(R, ldo) + 31) / 32, (Cpad + 31) / 32);
    transpose_bf16_kernel<<<grid, 256, 0, st>>>(in, R, C, ldi, out, ldo, Cpad);
    return cudaGetLastError();
}

cudaError_t conv_fwd_tc(const __nv_bfloat16 *x, int nb, int lout, const __nv_bfloat16 *W,
                        const float *bias, float *pre, __nv_bfloat16 *out, uint32_t *status, int sms,
                        cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    if (lout != 128 && lout != 64 && lout != 32) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(W) & 15))
        return cudaErrorInvalidValue;
    alignas(64) CUtensorMap map;
    const cudaError_t me = x_plane_map(x, nb, lout, &map);
    if (me != cudaSuccess) return me;
    static bool attr = false;
    if (!attr) {
        for (auto k : {conv_fwd_tc_kernel<128>, conv_fwd_tc_kernel<64>, conv_fwd_tc_kernel<32>}) {
            const cudaError_t e =
                cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
            if (e != cudaSuccess) return e;
        }
        attr = true;
    }
    const int ntiles = (nb * lout + kRowsPerTile - 1) / kRowsPerTile;
    const int grid = std::max(1, std::min(ntiles, sms));
    if (lout == 128)
        conv_fwd_tc_kernel<128><<<grid, kFwdThreads, kFwdSmem, st>>>(map, nb, W, bias, pre, out, status);
    else if (lout == 64)
        conv_fwd_tc_kernel<64><<<grid, kFwdThreads, kFwdSmem, st>>>(map, nb, W, bias, pre, out, status);
    else
        conv_fwd_tc_kernel<32><<<grid, kFwdThreads, kFwdSmem, st>>>(map, nb, W, bias, pre, out, status);
    return cudaGetLastError();
}

}  // namespace pchase
