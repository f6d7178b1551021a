// The learned inverse's network at inference (S7) on sm_103a's fifth-
// generation tensor cores: tcgen05.mma with both operands in shared memory
// and the FP32 accumulator in tensor memory (TMEM).  Three kernels: layers 1
// and 2 (conv12_tc_kernel), layers 3 and 4 (conv34_tc_kernel), FC + heads
// (fc_heads_tc_kernel).  The 64-channel layers (kernel 5, stride 2, zero
// padding 2) use an implicit im2col:
//
// out[b][p][co] = GELU(bias[co] + sum_k sum_ci W[co][k*64 + ci] * x[b][2p + k - 2][ci])
//
// One tile is 128 consecutive output rows (b, p) x 64 output channels, i.e.
// one M=128, N=64 accumulator, computed as 5 taps x 4 K-slices of 16 channels
// (20 MMAs, issued by one thread).  The A operand of tap k would be the input
// rows 2p + k - 2: rows two apart, which no shared-memory matrix descriptor
// can address.  So the tile's rows are taken in a transposed order, TMEM lane
// r = 8g + i holding output row o = 16i + g of the tile, and the input slab is
// staged as two planes (even and odd input offsets) whose row 8G + i holds
// input position 2*p(16i) + 2(G - 1) + plane.  Tap k then reads plane k % 2 from
// row group k / 2 on: 128 consecutive rows of 128 bytes (64 BF16 channels), a
// canonical K-major operand with the 128-byte swizzle, every tap starting on
// a 1024-byte swizzle-atom boundary.  The weights are five such N=64 x K=64
// tiles, loaded once per CTA.  An epilogue warp w reads TMEM lanes
// 32 (w % 4) .. +31 (the lanes its quarter of the CTA may access).
// Completion waits on an mbarrier give up after 2 s of %globaltimer: the
// kernel then ORs PCHASE_DEV_TIMEOUT into *status, stops, waits for its own
// copies and MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "conv_tc.cuh"
#include "tc_common.cuh"
#include "tma_host.cuh"

namespace pchase {
namespace {

constexpr int kCh = 64;
constexpr int kTaps = 5;
constexpr int kTileRows = 128;
constexpr int kGroups = 18;                           // 8-row groups per slab plane
constexpr uint32_t kPlaneBytes = kGroups * 8 * 128;   // 18 KB
constexpr uint32_t kSlabBytes = 2 * kPlaneBytes;      // 36 KB
constexpr int kSlabs = 3;
constexpr uint32_t kWBytes = kTaps * kCh * 128;       // 40 KB
constexpr uint32_t kTmemCols = 128;                   // two 64-column accumulators

// Instruction descriptor of tcgen05.mma .kind::f16: FP32 accumulator (bits
// 4-5 = 1), BF16 A and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 =
// 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) |
                            ((uint32_t)(kTileRows >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
    mma_bf16_id(d_tmem, a, b, kIdesc, acc);
}

// ------------------------------------------- first two layers, fused
// Inference of layers 1 and 2 without the first layer's activations ever
// leaving the SM.  One tile is one trace: layer 2's 128 output positions are
// exactly an M=128 accumulator.  Its input slab (the two planes of 18 x 8
// rows of layer-1 outputs described above, 36 KB) is computed by eight
// producer warps straight from the trace's 512 FP32 inputs (rounded to BF16
// as the unfused path rounds them): row 8G + i of plane pl holds layer-1
// position q = 32i + 2G - 2 + pl, channels in 16-byte chunks with the
// 128-byte swizzle, zeros outside 0 <= q < 256.  The other eight warps issue
// the MMAs (one thread) and run the epilogue (bias, GELU, BF16 store).  The two
// roles meet on mbarriers: slab_full (the producers' 256 arrivals after a
// proxy fence), slab_empty (tcgen05.commit once the MMAs that read a slab
// are done; three slabs in flight) and acc_full (two TMEM accumulators).
// Every wait gives up after 2 s: the CTA then ORs PCHASE_DEV_TIMEOUT into
// *status, each role leaves its loop at its next group barrier, the MMAs
// already issued are waited for, and TMEM is freed.
constexpr int kFusedThreads = 512;
constexpr uint32_t kFusedXs = 520;  // staged inputs: xs[q + 2] = x[q], zeros around
// two buffers of staged inputs, a trace's and the next one's
constexpr uint32_t kFusedSmem = 1024 + kWBytes + kSlabs * kSlabBytes + 2 * 4 * kFusedXs + 128;

__global__ void __launch_bounds__(kFusedThreads, 1)
    conv12_tc_kernel(const float *__restrict__ x, int nb, const __nv_bfloat16 *__restrict__ W1,
                     const float *__restrict__ bias1, const __nv_bfloat16 *__restrict__ W2,
                     const float *__restrict__ bias2, __nv_bfloat16 *__restrict__ out,
                     uint32_t *__restrict__ status) {
    constexpr int kLin = 512, kL1 = 256, kL2 = 128;
    extern __shared__ uint8_t dsm[];
    const uint32_t raw = smem_u32(dsm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *const gbase = dsm + (base - raw);
    const uint32_t sW = base;
    const uint32_t sSlab = base + kWBytes;
    float *const xs = reinterpret_cast<float *>(gbase + kWBytes + kSlabs * kSlabBytes);
    const uint32_t sBar = base + kWBytes + kSlabs * kSlabBytes + 2 * 4 * kFusedXs;
    // barriers: slab_full[3] at sBar + 8b, slab_empty[3] at sBar + 24 + 8b,
    // acc_full[2] at sBar + 48 + 8a; then the TMEM address and the abort flag
    uint32_t *const tslot = reinterpret_cast<uint32_t *>(gbase + (sBar - base) + 64);
    volatile uint32_t *const abort_flag = tslot + 1;
    volatile uint32_t *const last_issued = tslot + 2;  // tiles whose MMAs were issued

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = nb;

    // layer 2's weights: tap k is W2[:, 64k .. 64k+63], 64 rows of 128 bytes, swizzled
    for (int e = tid; e < kTaps * kCh * 8; e += kFusedThreads) {
        const int k = e >> 9, co = (e >> 3) & 63, c = e & 7;
        cp_async16(sW + k * 8192 + co * 128 + ((c ^ (co & 7)) << 4),
                   W2 + (size_t)co * (kTaps * kCh) + k * kCh + c * 8, true);
    }
    cp_async_commit();
    if (tid == 0) {
        for (int q = 0; q < 3; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 256;" ::"r"(sBar + 8 * q) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sBar + 24 + 8 * q)
                         : "memory");
        }
        for (int a = 0; a < 2; ++a)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sBar + 48 + 8 * a)
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
        *last_issued = 0;
    }
    if (tid < 2) xs[tid] = xs[kFusedXs + tid] = 0.0f;
    if (tid < (int)kFusedXs - kLin - 2) xs[kLin + 2 + tid] = xs[kFusedXs + kLin + 2 + tid] = 0.0f;
    // slab rows of positions -2, -1 (row 0 of each plane) and 256, 257 (row
    // 8 * 17 + 7) are zero padding, written once: the producers never write them
    for (int e = tid; e < kSlabs * 2 * 2 * 8; e += kFusedThreads) {
        const int sb = e / 32, pl = (e / 16) & 1, which = (e / 8) & 1, c = e & 7;
        const int row = which ? 8 * 17 + 7 : 0;
        uint4 *d = reinterpret_cast<uint4 *>(gbase + kWBytes + (size_t)sb * kSlabBytes +
                                             (size_t)pl * kPlaneBytes + (size_t)row * 128 + c * 16);
        *d = make_uint4(0u, 0u, 0u, 0u);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    cp_async_wait_all();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp < 8) {
        // ---------------- producers: layer 1 into the slabs (barrier id 2)
        const int p = tid;             // 0..255
        const int c = p & 7;           // the 8 channels this thread computes
        const int r0 = p >> 3;         // rows r0, r0 + 32, ... of the 288 slab rows
        // the weights and biases of channels (2jj, 2jj + 1) of this thread's
        // 8, halved (exactly), so that the sums come out halved for gelu2h_bf16
        uint64_t w2[4][kTaps], b2[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int c0 = c * 8 + 2 * jj;
            b2[jj] = f2(0.5f * bias1[c0], 0.5f * bias1[c0 + 1]);
#pragma unroll
            for (int k = 0; k < kTaps; ++k)
                w2[jj][k] = f2(0.5f * __bfloat162float(W1[c0 * kTaps + k]),
                               0.5f * __bfloat162float(W1[(c0 + 1) * kTaps + k]));
        }
        // the next trace's inputs are loaded while this one's slab is computed
        float xa = 0.0f, xb = 0.0f;
        if ((int)blockIdx.x < ntiles) {
            xa = x[(size_t)blockIdx.x * kLin + p];
            xb = x[(size_t)blockIdx.x * kLin + 256 + p];
        }
        for (int j = 0;; ++j) {
            const int t = blockIdx.x + j * (int)gridDim.x;
            if (t >= ntiles) break;
            const int b = j % kSlabs;
            bool ok = true;
            if (j >= kSlabs) ok = mbar_wait(sBar + 24 + 8 * b, (uint32_t)(j / kSlabs - 1) & 1u);
            // this trace's inputs into buffer j mod 2 (every producer finished
            // trace j - 2, the last user of that buffer, before the barrier of
            // trace j - 1), then one barrier: the inputs are in, and no wait
            // gave up
            float *const xb_ = xs + (j & 1) * kFusedXs;
            xb_[p + 2] = __bfloat162float(__float2bfloat16(xa));
            xb_[p + 258] = __bfloat162float(__float2bfloat16(xb));
            if (group_any(2, !ok || *abort_flag != 0)) {
                if (p == 0) *abort_flag = 1;
                break;
            }
            const int tn = t + (int)gridDim.x;
            if (tn < ntiles) {
                xa = x[(size_t)tn * kLin + p];
                xb = x[(size_t)tn * kLin + 256 + p];
            }
            const uint32_t slab = sSlab + (uint32_t)b * kSlabBytes;
            // each layer-1 position once (a warp takes 4 consecutive ones, so
            // its input reads fall in different banks), stored to the slab row
            // that holds it and, for the positions two row groups repeat, to
            // the second one too; the rows outside 0..255 stay zero
#pragma unroll 2
            for (int q = r0; q < kL1; q += 32) {
                uint64_t xin[kTaps];
#pragma unroll
                for (int k = 0; k < kTaps; ++k) {
                    const float xv = xb_[2 * q + k];  // x[2q + k - 2]
                    xin[k] = f2(xv, xv);
                }
                uint32_t pk[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    // channels 2jj and 2jj + 1 side by side: the bias, then the
                    // taps in order from 0, as one FMA chain (all halved)
                    uint64_t acc = fma2(w2[jj][0], xin[0], b2[jj]);
#pragma unroll
                    for (int k = 1; k < kTaps; ++k) acc = fma2(w2[jj][k], xin[k], acc);
                    pk[jj] = gelu2h_bf16(acc);
                }
                // q = 32i + 2G - 2 + pl: row 8G + i of plane pl (i < 8), and
                // row 8(G + 16) + (i - 1) when G < 2 and i > 0
                const int pl = q & 1, u = (q + 2 - pl) >> 1;
                const int i = u >> 4, G = u & 15;
                const uint32_t pbase = slab + (uint32_t)pl * kPlaneBytes;
                uint32_t dst;
                if (i < 8) {
                    dst = pbase + (uint32_t)(8 * G + i) * 128u + ((uint32_t)(c ^ i) << 4);
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst),
                                 "r"(pk[0]), "r"(pk[1]), "r"(pk[2]), "r"(pk[3])
                                 : "memory");
                }
                if (G < 2 && i > 0) {
                    dst = pbase + (uint32_t)(8 * (G + 16) + i - 1) * 128u +
                          ((uint32_t)(c ^ (i - 1)) << 4);
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst),
                                 "r"(pk[0]), "r"(pk[1]), "r"(pk[2]), "r"(pk[3])
                                 : "memory");
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(sBar + 8 * b)
                         : "memory");
        }
    } else {
        // ---------------- MMA issue and epilogue (barrier id 1)
        const int g = tid - 256, gw = warp - 8;
        bool bad = false;  // an accumulator wait of this thread gave up
        for (int j = 0;; ++j) {
            const int t = blockIdx.x + j * (int)gridDim.x;
            const bool have = t < ntiles;
            tc_fence_before();
            const bool stop = group_any(1, bad || *abort_flag != 0);
            tc_fence_after();
            if (stop) {
                if (bad) *abort_flag = 1;
                break;
            }
            if (have && g == 0) {
                const int b = j % kSlabs;
                if (!mbar_wait(sBar + 8 * b, (uint32_t)(j / kSlabs) & 1u)) {
                    *abort_flag = 1;
                } else {
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(j & 1) * 64u;
                    const uint32_t slab = sSlab + (uint32_t)b * kSlabBytes;
#pragma unroll
                    for (int k = 0; k < kTaps; ++k) {
                        const uint32_t a0 = slab + (uint32_t)(k & 1) * kPlaneBytes + (uint32_t)(k >> 1) * 1024u;
                        const uint32_t b0 = sW + (uint32_t)k * 8192u;
#pragma unroll
                        for (int s = 0; s < 4; ++s)
                            mma_bf16(d, sw128_desc(a0 + 32u * s), sw128_desc(b0 + 32u * s),
                                     (k | s) != 0 ? 1u : 0u);
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            sBar + 48u + 8u * (uint32_t)(j & 1))
                        : "memory");
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            sBar + 24u + 8u * (uint32_t)b)
                        : "memory");
                    *last_issued = (uint32_t)(j + 1);
                }
            }
            if (j > 0) {
                // epilogue of tile j - 1 (issued: tile j - 1 had its MMAs unless aborted)
                const int jp = j - 1;
                if (!mbar_wait(sBar + 48 + 8 * (jp & 1), (uint32_t)(jp >> 1) & 1u)) bad = true;
                tc_fence_after();
                const int tp = t - (int)gridDim.x;
                const int quarter = gw & 3, half = gw >> 2;
                const uint32_t taddr = tmem + (uint32_t)(jp & 1) * 64u + (uint32_t)half * 32u +
                                       ((uint32_t)(quarter * 32) << 16);
                uint32_t v[2][16];
#pragma unroll
                for (int qq = 0; qq < 2; ++qq) tmem_ld16(taddr + qq * 16, v[qq]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const int r = quarter * 32 + lane;
                const int m = 16 * (r & 7) + (r >> 3);  // output position of TMEM lane r
                uint4 *o4 = reinterpret_cast<uint4 *>(out + ((size_t)tp * kL2 + m) * kCh + half * 32);
#pragma unroll
                for (int qq = 0; qq < 2; ++qq) {
                    uint32_t pk[8];
#pragma unroll
                    for (int e = 0; e < 16; e += 2) {
                        const int n = half * 32 + qq * 16 + e;
                        pk[e >> 1] = gelu2_bf16(add2(f2(__uint_as_float(v[qq][e]),
                                                        __uint_as_float(v[qq][e + 1])),
                                                     f2(__ldg(bias2 + n), __ldg(bias2 + n + 1))));
                    }
                    o4[2 * qq] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    o4[2 * qq + 1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                }
            }
            if (!have) break;
        }
        if (bad) *abort_flag = 1;
        // every commit's arrival lands before the CTA leaves (the last tiles'
        // slab_empty arrivals have no producer waiting for them; after a
        // timeout, MMAs issued but never waited for must also finish before
        // TMEM is freed)
        if (g == 0) {
            const uint32_t li = *last_issued;
            if (li && *abort_flag)
                mbar_wait(sBar + 48 + 8 * ((li - 1) & 1), (uint32_t)((li - 1) >> 1) & 1u);
            for (uint32_t jj = li > (uint32_t)kSlabs ? li - kSlabs : 0u; jj < li; ++jj)
                mbar_wait(sBar + 24 + 8 * (jj % kSlabs), (jj / kSlabs) & 1u);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && *abort_flag) atomicOr(status, PCHASE_DEV_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
}

// ------------------------------------------------------------ FC + heads
// logits[m][h] = bias5[h] + sum_n bf16(GELU(bias4[n] + sum_k act[m][k] W4[n][k])) W5[h][n]
// act [B][2048] BF16, W4 [256][2048] BF16, W5 [31][256] BF16.  CTA t takes
// rows 128t .. 128t+127 and all 256 hidden units, so each activation row is
// read once:
//   * FC on the tensor cores: M128 N256, K = 2048 in 32 blocks of 64; a block
//     is two TMA tile loads (the activation tile and W4's, 2-D tensor maps with
//     the 128-byte swizzle; rows past the batch read as zeros) into a 4-stage
//     ring three blocks ahead, one thread issuing loads and MMAs; a stage's
//     mbarrier counts its bytes in, a second one frees it once its MMAs are done;
//   * epilogue: bias, GELU, BF16 rounding of the 128 x 256 hidden tile into
//     four swizzled 64-column K blocks in shared memory (the ring's space),
//     then the heads as a second MMA (M128 N32 K256, W5 padded to 32 rows)
//     into 32 more TMEM columns, read back and stored with bias5 (no atomics:
//     each CTA owns its rows).
constexpr int kFcK = 2048, kFcN = 256, kHeads = 31, kHeadsPad = 32;
constexpr int kFcStages = 4;   // ring stages, loaded kFcStages - 1 blocks ahead
constexpr uint32_t kFcABytes = kTileRows * 128, kFcBBytes = kFcN * 128;
constexpr uint32_t kFcStageBytes = kFcABytes + kFcBBytes;  // 48 KB
constexpr uint32_t kW5Bytes = 4 * kHeadsPad * 128;         // 4 K blocks of 32 rows x 64 BF16
constexpr uint32_t kFcSmemBytes =
    1024 + kFcStages * kFcStageBytes + kW5Bytes + 8 * (2 * kFcStages + 1) + 16;
constexpr uint32_t kFcTmemCols = 512;  // 256 FC + 32 heads, rounded to a power of two
constexpr uint32_t kIdescFc = (1u << 4) | (1u << 7) | (1u << 10) |
                              ((uint32_t)(kFcN >> 3) << 17) | ((uint32_t)(kTileRows >> 4) << 24);
constexpr uint32_t kIdescHeads = (1u << 4) | (1u << 7) | (1u << 10) |
                                 ((uint32_t)(kHeadsPad >> 3) << 17) |
                                 ((uint32_t)(kTileRows >> 4) << 24);

__global__ void __launch_bounds__(128, 1)
    fc_heads_tc_kernel(const __grid_constant__ CUtensorMap amap,
                       const __grid_constant__ CUtensorMap wmap, int nb, const float *__restrict__ bias4,
                       const __nv_bfloat16 *__restrict__ W5, const float *__restrict__ bias5,
                       float *__restrict__ logits, uint32_t *__restrict__ status) {
    extern __shared__ uint8_t dsm[];
    const uint32_t raw = smem_u32(dsm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *const gbase = dsm + (base - raw);
    const uint32_t sStage = base;
    const uint32_t sW5 = base + kFcStages * kFcStageBytes;  // 1024-aligned
    // mbarriers: stage loaded [S] at sBar + 8s, stage's MMAs done [S] at
    // sBar + 8 (S + s), the heads MMAs at sBar + 16 S
    const uint32_t sBar = sW5 + kW5Bytes;
    const uint32_t full0 = sBar, done0 = sBar + 8u * kFcStages, hbar = sBar + 16u * kFcStages;
    uint32_t *const tslot = reinterpret_cast<uint32_t *>(
        gbase + kFcStages * kFcStageBytes + kW5Bytes + 8 * (2 * kFcStages + 1));
    volatile uint32_t *const abort_flag = tslot + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTileRows;
    constexpr int kBlocks = kFcK / 64;

    // W5 as the heads' B operand: K block kb holds hidden units 64kb .. +63 of
    // its 32 rows (row 31 zero), 128-byte swizzle
    for (int e = tid; e < 4 * kHeadsPad * 8; e += 128) {
        const int kb = e >> 8, h = (e >> 3) & 31, c = e & 7;
        const bool ok = h < kHeads;
        cp_async16(sW5 + kb * (kHeadsPad * 128) + h * 128 + ((c ^ (h & 7)) << 4),
                   ok ? W5 + (size_t)h * kFcN + kb * 64 + c * 8 : W5, ok);
    }
    // block kb's activation and W4 tiles into stage kb mod S (one thread)
    auto load = [&](int kb) {
        const uint32_t q = (uint32_t)(kb % kFcStages);
        const uint32_t st = sStage + q * kFcStageBytes;
        mbar_expect_tx(full0 + 8u * q, kFcStageBytes);
        tma_load_2d(st, &amap, kb * 64, m0, full0 + 8u * q);
        tma_load_2d(st + kFcABytes, &wmap, kb * 64, 0, full0 + 8u * q);
    };
    cp_async_commit();
    if (tid == 0) {
        for (int q = 0; q <= 2 * kFcStages; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sBar + 8 * q) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(kFcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;  // columns 0..255: FC; 256..287: heads

    int loaded = 0;  // blocks whose loads went out (thread 0)
    if (tid == 0) {
        for (; loaded < kFcStages - 1; ++loaded) load(loaded);
        for (int kb = 0; kb < kBlocks; ++kb) {
            const uint32_t q = (uint32_t)(kb % kFcStages);
            if (!mbar_wait(full0 + 8u * q, (uint32_t)(kb / kFcStages) & 1u)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t st = sStage + q * kFcStageBytes;
#pragma unroll
            for (int s = 0; s < 4; ++s)
                mma_bf16_id(tmem, sw128_desc(st + 32u * s), sw128_desc(st + kFcABytes + 32u * s),
                            kIdescFc, (kb | s) != 0 ? 1u : 0u);
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    done0 + 8u * q)
                : "memory");
            // the stage of block kb - 1 (its MMAs went out a step ago) takes block kb + S - 1
            if (loaded < kBlocks) {
                const int pj = loaded - kFcStages;
                if (pj >= 0 && !mbar_wait(done0 + 8u * (uint32_t)(pj % kFcStages),
                                          (uint32_t)(pj / kFcStages) & 1u)) {
                    *abort_flag = 1;
                    break;
                }
                load(loaded++);
            }
        }
    }
    cp_async_wait_all();  // W5
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    bool ok = *abort_flag == 0;
    if (ok) {
        const int lb = kBlocks - 1;  // the last commit covers every earlier MMA
        const bool got = mbar_wait(done0 + 8u * (uint32_t)(lb % kFcStages), (uint32_t)(lb / kFcStages) & 1u);
        ok = __syncthreads_and(got);
    }
    const int r = warp * 32 + lane;  // TMEM lane = tile row
    if (ok) {
        // hidden tile -> BF16 A operand of the heads MMA: K block kb (hidden
        // units 64kb .. +63) at sStage + kb * 16 KB, rows of 128 bytes swizzled
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int q = 0; q < 16; ++q) {
            uint32_t v[16];
            tmem_ld16(taddr + q * 16, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            uint32_t pk[8];
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const int n = q * 16 + e;
                pk[e >> 1] = gelu2_bf16(add2(f2(__uint_as_float(v[e]), __uint_as_float(v[e + 1])),
                                             f2(__ldg(bias4 + n), __ldg(bias4 + n + 1))));
            }
            // 16 columns = chunks 2(q % 4), +1 of row r in K block q / 4
            uint4 *row = reinterpret_cast<uint4 *>(gbase + (q >> 2) * kFcABytes + r * 128);
            const int c0 = 2 * (q & 3);
            row[c0 ^ (r & 7)] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            row[(c0 + 1) ^ (r & 7)] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
#pragma unroll
            for (int kb = 0; kb < 4; ++kb)
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    mma_bf16_id(tmem + 256u, sw128_desc(sStage + kb * kFcABytes + 32u * s),
                                sw128_desc(sW5 + kb * (kHeadsPad * 128) + 32u * s), kIdescHeads,
                                (kb | s) != 0 ? 1u : 0u);
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    hbar)
                : "memory");
        }
        const bool got = mbar_wait(hbar, 0u);
        ok = __syncthreads_and(got);
        if (ok) {
            tc_fence_after();
            uint32_t v[2][16];
            tmem_ld16(taddr + 256, v[0]);
            tmem_ld16(taddr + 272, v[1]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int m = m0 + r;
            if (m < nb) {
#pragma unroll
                for (int h = 0; h < kHeads; ++h)
                    logits[(size_t)m * kHeads + h] = __uint_as_float(v[h >> 4][h & 15]) + __ldg(bias5 + h);
            }
        }
    }
    if (!ok && tid == 0) {
        atomicOr(status, PCHASE_DEV_TIMEOUT);
        // the loads and MMAs issued land before TMEM is freed and the CTA leaves
        for (int j = loaded > kFcStages ? loaded - kFcStages : 0; j < loaded; ++j)
            mbar_wait(full0 + 8u * (uint32_t)(j % kFcStages), (uint32_t)(j / kFcStages) & 1u);
        if (loaded > 0)
            mbar_wait(done0 + 8u * (uint32_t)((loaded - 1) % kFcStages),
                      (uint32_t)((loaded - 1) / kFcStages) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kFcTmemCols)
                     : "memory");
}

// ------------------------------------------------------------ layers 3 + 4
// Inference of layers 3 and 4 in one kernel.  An iteration takes 4 traces
// (one 128-row tile of layer 4): the layer-3 outputs of its two 128-row tiles
// (2 traces each) go from TMEM through bias and GELU straight into layer 4's
// input slab in shared memory, laid out as the implicit im2col above wants
// (row 8g + i of plane pl holds position 32 (i & 1) + 2 (g - 1) + pl of the
// tile's trace i / 2), and layer 4's MMAs run from there; only layer 4's
// outputs go to global memory.  A layer-3 position q of trace b lands in row
// 8 ((q >> 1) + 1) + 2b when q <= 33 and in row 8 ((q >> 1) - 15) + 2b + 1
// when q >= 30 (plane q & 1); rows 2b of group 0 and 2b + 1 of group 17 are
// the zero padding, written once.  Layer-3 input slabs stream in by cp.async
// (three buffers).
constexpr int kL34Threads = 512;  // the first 256 load slabs; all run the epilogues
constexpr uint32_t kL34TmemCols = 256;  // accumulators: layer-3 tiles A, B and layer 4
constexpr uint32_t kL34Smem = 1024 + 2 * kWBytes + kSlabs * kSlabBytes + kSlabBytes + 64;

__global__ void __launch_bounds__(kL34Threads, 1)
    conv34_tc_kernel(const __nv_bfloat16 *__restrict__ x, int nb,
                     const __nv_bfloat16 *__restrict__ W3, const float *__restrict__ bias3,
                     const __nv_bfloat16 *__restrict__ W4, const float *__restrict__ bias4,
                     __nv_bfloat16 *__restrict__ out, uint32_t *__restrict__ status) {
    constexpr int kLin3 = 128, kL3 = 64, kL4 = 32;
    extern __shared__ uint8_t dsm[];
    const uint32_t raw = smem_u32(dsm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *const gbase = dsm + (base - raw);
    const uint32_t sW3 = base, sW4 = base + kWBytes;
    const uint32_t sSlab = base + 2 * kWBytes;         // layer-3 input slabs
    const uint32_t sL4 = sSlab + kSlabs * kSlabBytes;  // layer-4 input slab
    const uint32_t sBar = sL4 + kSlabBytes;            // mbarriers: tile A, tile B, layer 4
    uint32_t *const tslot = reinterpret_cast<uint32_t *>(gbase + (sBar - base) + 32);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int M3 = nb * kL3, M4 = nb * kL4;
    const int n4 = (M4 + kTileRows - 1) / kTileRows;  // iterations of 4 traces
    const int n3 = 2 * n4;                            // layer-3 tiles: 2 it and 2 it + 1

    for (int e = tid; e < kTaps * kCh * 8; e += kL34Threads) {
        const int k = e >> 9, co = (e >> 3) & 63, c = e & 7;
        const uint32_t off = k * 8192 + co * 128 + ((c ^ (co & 7)) << 4);
        const size_t src = (size_t)co * (kTaps * kCh) + k * kCh + c * 8;
        cp_async16(sW3 + off, W3 + src, true);
        cp_async16(sW4 + off, W4 + src, true);
    }
    cp_async_commit();

    const int ld_c = tid & 7, ld_i = (tid >> 3) & 7, ld_pl = (tid >> 6) & 1, ld_h = tid >> 7;
    const int ld_g0 = ld_h * (kGroups / 2);
    auto load_slab = [&](int buf, int u) {
        if (u < n3 && tid < 256) {
            const int mi = u * kTileRows + 16 * ld_i;
            const int b = mi / kL3, p0 = mi - b * kL3;
            const bool row_ok = mi < M3;
            const int q0 = 2 * p0 + 2 * (ld_g0 - 1) + ld_pl;
            const __nv_bfloat16 *src = x + ((size_t)(row_ok ? b : 0) * kLin3) * kCh + ld_c * 8;
            const uint32_t dst = sSlab + buf * kSlabBytes + ld_pl * kPlaneBytes +
                                 (8 * ld_g0 + ld_i) * 128 + ((ld_c ^ ld_i) << 4);
#pragma unroll
            for (int gg = 0; gg < kGroups / 2; ++gg) {
                const int q = q0 + 2 * gg;
                const bool ok = row_ok && q >= 0 && q < kLin3;
                cp_async16(dst + gg * 1024, ok ? src + (size_t)q * kCh : x, ok);
            }
        }
        cp_async_commit();  // one group per call, empty or not
    };

    // the layer-4 slab's padding rows (never written again)
    if (tid < 2 * 4 * 2 * 8) {
        const int pl = tid >> 6, b = (tid >> 4) & 3, which = (tid >> 3) & 1, c = tid & 7;
        const int row = which ? 8 * 17 + 2 * b + 1 : 2 * b;
        *reinterpret_cast<uint4 *>(gbase + (sL4 - base) + pl * kPlaneBytes + row * 128 +
                                   ((c ^ (row & 7)) << 4)) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int q = 0; q < 3; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sBar + 8 * q) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(kL34TmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    load_slab(0, 2 * (int)blockIdx.x);
    load_slab(1, 2 * (int)blockIdx.x + 1);
    load_slab(2, 2 * ((int)blockIdx.x + (int)gridDim.x));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // one thread: the 20 MMAs of a tile from slab a0 with weights sw into d
    auto mma_tile = [&](uint32_t d, uint32_t slab, uint32_t sw, uint32_t bar) {
#pragma unroll
        for (int k = 0; k < kTaps; ++k) {
            const uint32_t a0 = slab + (uint32_t)(k & 1) * kPlaneBytes + (uint32_t)(k >> 1) * 1024u;
            const uint32_t b0 = sw + (uint32_t)k * 8192u;
#pragma unroll
            for (int s = 0; s < 4; ++s)
                mma_bf16(d, sw128_desc(a0 + 32u * s), sw128_desc(b0 + 32u * s),
                         (k | s) != 0 ? 1u : 0u);
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
            : "memory");
    };
    // warp w reads TMEM lane quarter w mod 4 (its hardware quarter) and
    // columns 16 (w / 4) .. + 15: a thread holds 16 values of one tile row
    const int quarter = warp & 3, colq = warp >> 2;
    const int r = quarter * 32 + lane;          // this thread's TMEM lane
    const int mt = 16 * (r & 7) + (r >> 3);     // ... and the tile row it holds
    const uint32_t lane_off = ((uint32_t)(quarter * 32) << 16) + (uint32_t)colq * 16u;
    // bias + GELU of this thread's 16 columns of accumulator acc, as BF16 pairs
    auto finish = [&](uint32_t acc, const float *bias, uint32_t (&pk)[8]) {
        uint32_t v[16];
        tmem_ld16(tmem + acc + lane_off, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 16; e += 2) {
            const int n = colq * 16 + e;
            pk[e >> 1] = gelu2_bf16(add2(f2(__uint_as_float(v[e]), __uint_as_float(v[e + 1])),
                                         f2(__ldg(bias + n), __ldg(bias + n + 1))));
        }
    };
    // the two 16-byte chunks of a row written in an order that alternates
    // with the lane, so that a store instruction's lanes spread over more banks
    auto put_row = [&](uint32_t pbase, uint32_t row, const uint32_t (&pk)[8]) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int cc = k ^ (lane & 1);
            const uint32_t dst =
                pbase + row * 128u + ((uint32_t)((colq * 2 + cc) ^ (int)(row & 7)) << 4);
            const uint32_t w0 = cc ? pk[4] : pk[0], w1 = cc ? pk[5] : pk[1];
            const uint32_t w2 = cc ? pk[6] : pk[2], w3 = cc ? pk[7] : pk[3];
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(w0), "r"(w1),
                         "r"(w2), "r"(w3)
                         : "memory");
        }
    };

    // Software pipeline over iterations n (tiles 2n, 2n + 1 of layer 3; one
    // tile of layer 4): both layer-3 tiles' MMAs go out together, layer 4's
    // epilogue of iteration n - 1 runs while they execute, then the layer-3
    // epilogues fill the slab and layer 4's MMAs of iteration n go out, to
    // complete while the next iteration's loads are awaited.  Tile s sits in
    // buffer s mod 3, and tile s + 3 is loaded into it as soon as the
    // epilogue of tile s has seen s's MMAs complete.
    // layer 4's epilogue of the iteration at it (phase ph)
    // (a wait that gives up marks `bad`; the block learns of it at its next
    // barrier, so the waits themselves need none)
    bool bad = false;
    auto epilogue4 = [&](int it, uint32_t ph) {
        if (!mbar_wait(sBar + 16u, ph)) bad = true;
        tc_fence_after();
        uint32_t pk[8];
        finish(128u, bias4, pk);
        const int m = it * kTileRows + mt;
        if (m < M4) {
            uint4 *o4 = reinterpret_cast<uint4 *>(out + (size_t)m * kCh + colq * 16);
            o4[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            o4[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
        tc_fence_before();
    };
    int n = 0;
    bool ok = true;
    for (int it = blockIdx.x; it < n4; it += gridDim.x, ++n) {
        const uint32_t ph = (uint32_t)n & 1u;
        const int itn = it + (int)gridDim.x;
        // tiles 2n and 2n + 1 loaded (tile 2n + 2 may still be in flight)
        cp_async_wait1();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        if (__syncthreads_or(bad)) {
            ok = false;
            break;
        }
        tc_fence_after();
        if (tid == 0) {
            mma_tile(tmem, sSlab + (uint32_t)((2 * n) % kSlabs) * kSlabBytes, sW3, sBar);
            mma_tile(tmem + 64u, sSlab + (uint32_t)((2 * n + 1) % kSlabs) * kSlabBytes, sW3,
                     sBar + 8u);
        }
        if (n > 0) epilogue4(it - (int)gridDim.x, ph ^ 1u);
        // layer-3 epilogues into the layer-4 slab (layer 4's last MMAs
        // completed: its epilogue just waited for them)
        for (int X = 0; X < 2; ++X) {
            if (!mbar_wait(sBar + 8u * (uint32_t)X, ph)) bad = true;
            tc_fence_after();
            // this tile's buffer is free: tile 2n + X + 3 of the sequence goes
            // there (iteration n + 1's tile B, or iteration n + 2's tile A)
            load_slab((2 * n + X) % kSlabs, X == 0 ? 2 * itn + 1 : 2 * (itn + (int)gridDim.x));
            uint32_t pk[8];
            finish(64u * (uint32_t)X, bias3, pk);
            const int b = 2 * X + (mt >> 6), q = mt & 63;
            const uint32_t pbase = sL4 + (uint32_t)(q & 1) * kPlaneBytes;
            if (q <= 33) put_row(pbase, 8u * (uint32_t)((q >> 1) + 1) + 2u * (uint32_t)b, pk);
            if (q >= 30) put_row(pbase, 8u * (uint32_t)((q >> 1) - 15) + 2u * (uint32_t)b + 1u, pk);
            tc_fence_before();
        }
        // layer 4 from the slab just written
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        if (__syncthreads_or(bad)) {
            ok = false;
            break;
        }
        tc_fence_after();
        if (tid == 0) mma_tile(tmem + 128u, sL4, sW4, sBar + 16u);
    }
    if (ok && n > 0) epilogue4(blockIdx.x + (n - 1) * (int)gridDim.x, (uint32_t)(n - 1) & 1u);
    if (__syncthreads_or(bad) && tid == 0) atomicOr(status, PCHASE_DEV_TIMEOUT);
    cp_async_wait_all();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kL34TmemCols)
                     : "memory");
}

}  // namespace

cudaError_t conv34_tc(const __nv_bfloat16 *x, int nb, const __nv_bfloat16 *W3, const float *bias3,
                      const __nv_bfloat16 *W4, const float *bias4, __nv_bfloat16 *out,
                      uint32_t *status, int sms, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    if (!status) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(conv34_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kL34Smem);
    if (e != cudaSuccess) return e;
    const long long iters = ((long long)nb * 32 + kTileRows - 1) / kTileRows;
    const int grid = (int)std::min<long long>(iters, std::max(1, sms));
    conv34_tc_kernel<<<grid, kL34Threads, kL34Smem, st>>>(x, nb, W3, bias3, W4, bias4, out, status);
    return cudaGetLastError();
}

cudaError_t conv12_tc(const float *x, int nb, const __nv_bfloat16 *W1, const float *bias1,
                      const __nv_bfloat16 *W2, const float *bias2, __nv_bfloat16 *out,
                      uint32_t *status, int sms, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    if (!status) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(conv12_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFusedSmem);
    if (e != cudaSuccess) return e;
    const int grid = std::min(nb, std::max(1, sms));
    conv12_tc_kernel<<<grid, kFusedThreads, kFusedSmem, st>>>(x, nb, W1, bias1, W2, bias2, out,
                                                               status);
    return cudaGetLastError();
}

cudaError_t fc_heads_tc(const __nv_bfloat16 *act, int nb, const __nv_bfloat16 *W4,
                        const float *bias4, const __nv_bfloat16 *W5, const float *bias5,
                        float *logits, uint32_t *status, cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    if (!status) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fc_heads_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFcSmemBytes);
    if (e != cudaSuccess) return e;
    if ((reinterpret_cast<uintptr_t>(act) & 15) || (reinterpret_cast<uintptr_t>(W4) & 15))
        return cudaErrorInvalidValue;
    alignas(64) CUtensorMap amap, wmap;
    if (!kmajor_map(act, nb, kFcK, kFcK, kTileRows, &amap) ||
        !kmajor_map(W4, kFcN, kFcK, kFcK, kFcN, &wmap))
        return cudaErrorInvalidValue;
    const int grid = (nb + kTileRows - 1) / kTileRows;
    fc_heads_tc_kernel<<<grid, 128, kFcSmemBytes, st>>>(amap, wmap, nb, bias4, W5, bias5, logits,
                                                        status);
    return cudaGetLastError();
}

}  // namespace pchase
