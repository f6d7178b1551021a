// S8-S10: probes that produce traces on this GPU.
//
//   * fine-grained P-chase (Listing 3, Sec. 4.2): one thread, clock64 around
//     the load of j = A[j] followed by a store of j into shared memory, which
//     depends on the load and so holds back the second clock read until the
//     load has completed; latencies and indices are buffered in shared memory
//     (256 per round) and copied out between rounds;
//   * shared-memory stride latency (Listing 4, Sec. 6.2): one warp, lane t
//     starting at word t*stride of a self-pointing array, 64 dependent reads;
//   * global-memory read / write / copy throughput (Sec. 5.1) with 4- or
//     16-byte vectors, a grid-stride loop and `ilp` independent vectors per
//     thread per trip;
//   * shared-memory throughput (Sec. 6.1): every thread copies `ilp` 4-byte
//     words from one shared region to another, `iters` times; each CTA times
//     its loop with its SM's clock64 between two __syncthreads and records
//     its SM, so the host can sum bytes per SM over the SM's busy span.
// Every loop is bounded by its caller-given count.
#include <algorithm>
#include <vector>

#include "pchase_internal.cuh"

namespace pchase {

namespace {

constexpr int kRound = 256;

template <int MODE>
__device__ __forceinline__ uint32_t ld_chain(const uint32_t *p) {
    uint32_t v;
    if (MODE == 0)
        asm volatile("ld.global.ca.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    else if (MODE == 1)
        asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    else
        asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ long long clk() {
    long long c;
    asm volatile("mov.u64 %0, %%clock64;" : "=l"(c)::"memory");
    return c;
}

__device__ __forceinline__ void st_shared(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

template <int MODE>
__global__ void probe_latency_kernel(const uint32_t *A, uint32_t n, uint32_t start,
                                     uint32_t warmup, uint32_t iters, uint32_t *lat_out,
                                     uint32_t *idx_out, uint32_t *ovh_out, uint32_t *status) {
    __shared__ uint32_t s_t[kRound];
    __shared__ uint32_t s_i[kRound];
    __shared__ uint32_t s_sink[4];
    const uint32_t sa_i = (uint32_t)__cvta_generic_to_shared(s_i);
    const uint32_t sa_sink = (uint32_t)__cvta_generic_to_shared(s_sink);

    // calibration: back-to-back clock reads, and clock + dependent store + clock
    // around a value that is already in a register (the non-load part of one
    // timed access); the minimum over 64 tries
    uint32_t best_pair = 0xFFFFFFFFu, best_seg = 0xFFFFFFFFu;
    uint32_t v = start;
    for (int k = 0; k < 64; ++k) {
        long long a = clk();
        long long b = clk();
        best_pair = min(best_pair, (uint32_t)(b - a));
        a = clk();
        st_shared(sa_sink, v);
        b = clk();
        best_seg = min(best_seg, (uint32_t)(b - a));
        v += 1;
    }
    if (ovh_out) {
        ovh_out[0] = best_seg;
        ovh_out[1] = best_pair;
    }

    uint32_t j = start % n;
    for (uint32_t w = 0; w < warmup; ++w) {  // preheat
        j = ld_chain<MODE>(A + j);
        if (j >= n) {
            atomicOr(status, PCHASE_DEV_CHAIN_RANGE);
            return;
        }
    }
    for (uint32_t base = 0; base < iters; base += kRound) {
        const uint32_t m = min((uint32_t)kRound, iters - base);
        uint32_t visited0 = j;
        uint32_t k = 0;
        bool bad = false;
        for (; k < m; ++k) {
            const long long t0 = clk();
            const uint32_t nj = ld_chain<MODE>(A + j);
            st_shared(sa_i + 4 * k, nj);
            const long long t1 = clk();
            s_t[k] = (uint32_t)(t1 - t0);
            j = nj;
            if (j >= n) {
                bad = true;
                ++k;
                break;
            }
        }
        // copy out: idx_out[i] is the index visited by access i
        for (uint32_t q = 0; q < k; ++q) {
            const uint32_t raw = s_t[q];
            lat_out[base + q] = raw > best_seg ? raw - best_seg : 0;
            idx_out[base + q] = q == 0 ? visited0 : s_i[q - 1];
        }
        if (bad) {
            atomicOr(status, PCHASE_DEV_CHAIN_RANGE);
            return;
        }
    }
}

__global__ void probe_smem_kernel(uint32_t max_stride, uint32_t repeats, float *cycles,
                                  uint32_t *degree) {
    constexpr uint32_t kWords = 64 * 31 + 1;
    __shared__ uint32_t sdata[kWords];
    volatile uint32_t *vs = sdata;
    const uint32_t lane = threadIdx.x;
    for (uint32_t i = lane; i < kWords; i += 32) sdata[i] = i;  // each word points at itself
    __syncwarp();
    uint32_t sink = 0;
    for (uint32_t s = 1; s <= max_stride; ++s) {
        uint32_t times[64];
        for (uint32_t r = 0; r <= repeats; ++r) {  // round 0 is untimed (cold)
            uint32_t data = lane * s;
            __syncwarp();
            const long long t0 = clk();
#pragma unroll
            for (int k = 0; k < 64; ++k) data = vs[data];
            __syncwarp();
            const long long t1 = clk();
            sink += data;
            if (r > 0) times[r - 1] = (uint32_t)(t1 - t0);
        }
        if (lane == 0) {
            for (uint32_t a = 1; a < repeats; ++a)  // insertion sort, repeats <= 64
                for (uint32_t b = a; b > 0 && times[b - 1] > times[b]; --b) {
                    const uint32_t tmp = times[b];
                    times[b] = times[b - 1];
                    times[b - 1] = tmp;
                }
            cycles[s - 1] = (float)times[(repeats - 1) / 2] / 64.0f;
        }
        // bank model: word w in bank w mod 32, equal words broadcast
        const uint32_t word = lane * s;
        const uint32_t same_word = __match_any_sync(kFull, word);
        const bool leader = (same_word & ((1u << lane) - 1)) == 0;
        const uint32_t same_bank = __match_any_sync(kFull, word & 31u);
        const uint32_t leaders = __ballot_sync(kFull, leader);
        const uint32_t deg = __reduce_max_sync(kFull, (uint32_t)__popc(same_bank & leaders));
        if (lane == 0) degree[s - 1] = deg;
    }
    if (sink == 0xFFFFFFFFu) cycles[0] = -1.0f;  // keeps the chase alive; never true
}

template <typename V>
__device__ __forceinline__ V vzero();
template <>
__device__ __forceinline__ float vzero<float>() { return 0.0f; }
template <>
__device__ __forceinline__ int4 vzero<int4>() { return make_int4(0, 0, 0, 0); }

__device__ __forceinline__ uint32_t vfold(float v) { return __float_as_uint(v); }
__device__ __forceinline__ uint32_t vfold(int4 v) { return (uint32_t)(v.x ^ v.y ^ v.z ^ v.w); }

template <typename V>
__device__ __forceinline__ V vfill(uint64_t i);
template <>
__device__ __forceinline__ float vfill<float>(uint64_t i) { return (float)(i & 1023); }
template <>
__device__ __forceinline__ int4 vfill<int4>(uint64_t i) {
    return make_int4((int)i, (int)(i >> 1), (int)(i >> 2), (int)(i >> 3));
}

// kind 0 read, 1 write, 2 copy; n = vectors, a multiple of ILP
template <typename V, int ILP, int KIND>
__global__ void gmem_kernel(const V *__restrict__ src, V *__restrict__ dst, uint64_t n,
                            uint32_t *sink) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    uint32_t acc = 0;
    for (uint64_t base = tid; base < n; base += nt * ILP) {
        V r[ILP];
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
            const uint64_t i = base + (uint64_t)k * nt;
            if (KIND == 1) {
                r[k] = vfill<V>(i);
            } else {
                r[k] = i < n ? src[i] : vzero<V>();
            }
        }
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
            const uint64_t i = base + (uint64_t)k * nt;
            if (KIND == 0) acc ^= vfold(r[k]);
            else if (i < n) dst[i] = r[k];
        }
    }
    if (KIND == 0 && acc == 0x9E3779B9u) *sink = acc;  // keeps the loads alive
}

template <typename V, int KIND>
cudaError_t launch_gmem_ilp(uint32_t ilp, uint32_t ctas, uint32_t threads, const void *src,
                            void *dst, uint64_t n, cudaStream_t st) {
    const V *s = static_cast<const V *>(src);
    V *d = static_cast<V *>(dst);
    uint32_t *sink = static_cast<uint32_t *>(dst);
    switch (ilp) {
        case 1: gmem_kernel<V, 1, KIND><<<ctas, threads, 0, st>>>(s, d, n, sink); break;
        case 2: gmem_kernel<V, 2, KIND><<<ctas, threads, 0, st>>>(s, d, n, sink); break;
        case 4: gmem_kernel<V, 4, KIND><<<ctas, threads, 0, st>>>(s, d, n, sink); break;
        default: gmem_kernel<V, 8, KIND><<<ctas, threads, 0, st>>>(s, d, n, sink); break;
    }
    return cudaGetLastError();
}

template <typename V>
cudaError_t launch_gmem(int kind, uint32_t ilp, uint32_t ctas, uint32_t threads,
                        const void *src, void *dst, uint64_t n, cudaStream_t st) {
    if (kind == 0) return launch_gmem_ilp<V, 0>(ilp, ctas, threads, src, dst, n, st);
    if (kind == 1) return launch_gmem_ilp<V, 1>(ilp, ctas, threads, src, dst, n, st);
    return launch_gmem_ilp<V, 2>(ilp, ctas, threads, src, dst, n, st);
}

// Sec. 6.1's copy: per trip, `ILP` independent shared loads, then their
// stores into the second region (the words a thread copies are ILP x 4 bytes
// read and written).  Volatile keeps every trip's accesses.
template <int ILP>
__global__ void smem_copy_kernel(uint32_t iters, unsigned long long *t0_out,
                                 unsigned long long *t1_out, uint32_t *smid_out) {
    extern __shared__ uint32_t sm_words[];
    volatile uint32_t *src = sm_words;
    volatile uint32_t *dst = sm_words + ILP * blockDim.x;
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
#pragma unroll
    for (int k = 0; k < ILP; ++k) src[k * nt + tid] = tid * 7u + (uint32_t)k;
    __syncthreads();
    const long long t0 = clk();
    for (uint32_t it = 0; it < iters; ++it) {
        uint32_t v[ILP];
#pragma unroll
        for (int k = 0; k < ILP; ++k) v[k] = src[k * nt + tid];
#pragma unroll
        for (int k = 0; k < ILP; ++k) dst[k * nt + tid] = v[k] + it;
    }
    __syncthreads();
    const long long t1 = clk();
    if (tid == 0) {
        uint32_t smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        t0_out[blockIdx.x] = (unsigned long long)t0;
        t1_out[blockIdx.x] = (unsigned long long)t1;
        smid_out[blockIdx.x] = smid;
    }
}

}  // namespace

cudaError_t probe_smem_copy(uint32_t ctas, uint32_t threads, uint32_t ilp, uint32_t iters,
                            unsigned long long *t0, unsigned long long *t1, uint32_t *smid,
                            cudaStream_t st) {
    const size_t bytes = 8ull * ilp * threads;
    cudaError_t e = cudaSuccess;
    switch (ilp) {
#define PCHASE_SMEM_ILP(N)                                                                     \
    case N:                                                                                    \
        e = cudaFuncSetAttribute(smem_copy_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)bytes);                                                  \
        if (e != cudaSuccess) return e;                                                        \
        smem_copy_kernel<N><<<ctas, threads, bytes, st>>>(iters, t0, t1, smid);                \
        break;
        PCHASE_SMEM_ILP(1)
        PCHASE_SMEM_ILP(2)
        PCHASE_SMEM_ILP(4)
        PCHASE_SMEM_ILP(6)
        PCHASE_SMEM_ILP(8)
#undef PCHASE_SMEM_ILP
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t probe_latency(const uint32_t *A, uint32_t n, uint32_t start, uint32_t warmup,
                          uint32_t iters, int mode, uint32_t *lat, uint32_t *idx, uint32_t *ovh,
                          uint32_t *status, cudaStream_t st) {
    if (mode == 0)
        probe_latency_kernel<0><<<1, 1, 0, st>>>(A, n, start, warmup, iters, lat, idx, ovh, status);
    else if (mode == 1)
        probe_latency_kernel<1><<<1, 1, 0, st>>>(A, n, start, warmup, iters, lat, idx, ovh, status);
    else
        probe_latency_kernel<2><<<1, 1, 0, st>>>(A, n, start, warmup, iters, lat, idx, ovh, status);
    return cudaGetLastError();
}

cudaError_t probe_smem(uint32_t max_stride, uint32_t repeats, float *cycles, uint32_t *degree,
                       cudaStream_t st) {
    probe_smem_kernel<<<1, 32, 0, st>>>(max_stride, repeats, cycles, degree);
    return cudaGetLastError();
}

cudaError_t probe_gmem(int kind, uint32_t vec_bytes, uint32_t ctas, uint32_t threads,
                       uint32_t ilp, const void *src, void *dst, uint64_t bytes, uint32_t reps,
                       double *gbs, cudaStream_t st) {
    const uint64_t n = bytes / vec_bytes;
    cudaEvent_t e0, e1;
    cudaError_t err = cudaEventCreate(&e0);
    if (err != cudaSuccess) return err;
    err = cudaEventCreate(&e1);
    if (err != cudaSuccess) {
        cudaEventDestroy(e0);
        return err;
    }
    std::vector<float> ms;
    for (uint32_t r = 0; r <= reps && err == cudaSuccess; ++r) {
        err = cudaEventRecord(e0, st);
        if (err != cudaSuccess) break;
        err = vec_bytes == 16 ? launch_gmem<int4>(kind, ilp, ctas, threads, src, dst, n, st)
                              : launch_gmem<float>(kind, ilp, ctas, threads, src, dst, n, st);
        if (err != cudaSuccess) break;
        err = cudaEventRecord(e1, st);
        if (err != cudaSuccess) break;
        err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) break;
        float t = 0;
        err = cudaEventElapsedTime(&t, e0, e1);
        if (r > 0) ms.push_back(t);  // launch 0 warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return err;
    std::sort(ms.begin(), ms.end());
    const double med = ms[(ms.size() - 1) / 2];
    const double moved = (kind == 2 ? 2.0 : 1.0) * (double)(n * vec_bytes);
    *gbs = med > 0 ? moved / (med * 1e-3) / 1e9 : 0.0;
    return cudaSuccess;
}

}  // namespace pchase
