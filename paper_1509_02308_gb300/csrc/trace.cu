// S1: P-chase array and trace construction (Listing 1, Sec. 4.1; the chase
// j = A[j] of Listings 2-3; caller-built non-uniform chains of Fig. 10).
//
// A uniform chain A[i] = (i + s) mod N walked from j = 0 visits (t * s) mod N
// at access t, so the trace is written in parallel: each thread produces four
// consecutive indices per 16-byte store and advances by a precomputed
// (4 * threads * s) mod N with one conditional subtraction.
#include "pchase_internal.cuh"

namespace pchase {

namespace {

__device__ __forceinline__ uint32_t add_mod(uint32_t x, uint32_t d, uint32_t n) {
    // (x + d) mod n for x, d < n without 32-bit overflow
    return x >= n - d ? x - (n - d) : x + d;
}

// Writes trace[t] = (t * s) mod n for t in [0, len), with trace 4-byte aligned.
__device__ __forceinline__ void write_uniform(uint32_t *trace, uint32_t n, uint32_t s,
                                              uint64_t len, uint32_t tid, uint32_t nthr) {
    s %= n;
    // scalar head up to a 16-byte boundary
    const uint32_t mis = (uint32_t)((reinterpret_cast<uintptr_t>(trace) >> 2) & 3u);
    const uint64_t head = mis ? ((4 - mis) < len ? (uint64_t)(4 - mis) : len) : 0;
    if (tid < head) trace[tid] = (uint32_t)(((uint64_t)tid * s) % n);
    const uint64_t body = (len - head) & ~3ull;
    uint4 *out4 = reinterpret_cast<uint4 *>(trace + head);
    const uint64_t nq = body >> 2;
    uint64_t q = tid;
    if (q < nq) {
        uint32_t j = (uint32_t)(((head + 4 * q) % n * (uint64_t)s) % n);
        const uint32_t step = (uint32_t)(((4ull * nthr) % n) * (uint64_t)s % n);
        for (; q < nq; q += nthr) {
            uint4 v;
            v.x = j;
            v.y = add_mod(v.x, s, n);
            v.z = add_mod(v.y, s, n);
            v.w = add_mod(v.z, s, n);
            out4[q] = v;
            j = add_mod(j, step, n);
        }
    }
    const uint64_t tail0 = head + body;
    if (tail0 + tid < len) {
        const uint64_t t = tail0 + tid;
        trace[t] = (uint32_t)((t % n * (uint64_t)s) % n);
    }
}

__global__ void uniform_trace_kernel(uint32_t n, uint32_t s, uint64_t len, uint32_t *trace) {
    write_uniform(trace, n, s, len, blockIdx.x * blockDim.x + threadIdx.x,
                  gridDim.x * blockDim.x);
}

__global__ void uniform_array_kernel(uint32_t n, uint32_t s, uint32_t *A) {
    const uint32_t sm = s % n;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        A[i] = add_mod((uint32_t)i, sm, n);
}

// One thread follows a caller-built chain; a link outside the array stops it.
__global__ void chain_walk_kernel(const uint32_t *next, uint32_t n, uint64_t len,
                                  uint32_t *trace, uint32_t *status) {
    uint32_t j = 0;
    for (uint64_t t = 0; t < len; ++t) {
        trace[t] = j;
        j = next[j];
        if (j >= n) {
            if (t + 1 < len) atomicOr(status, PCHASE_DEV_CHAIN_RANGE);
            return;
        }
    }
}

constexpr int kBatchPerLaunch = 1024;

struct BatchEntry {
    uint32_t n, s;
    uint64_t len;
    uint64_t off;
};

struct BatchParams {
    BatchEntry e[kBatchPerLaunch];
};

__global__ void uniform_batch_kernel(const __grid_constant__ BatchParams p, uint32_t *out) {
    const BatchEntry &e = p.e[blockIdx.x];
    write_uniform(out + e.off, e.n, e.s, e.len, threadIdx.x, blockDim.x);
}

}  // namespace

cudaError_t build_uniform(uint32_t n, uint32_t s, uint64_t len, uint32_t *trace,
                          uint32_t *array_out, cudaStream_t st, int sms) {
    if (len) {
        const uint64_t quads = (len + 3) / 4;
        const int threads = 256;
        uint64_t blocks = (quads + threads - 1) / threads;
        const uint64_t cap = (uint64_t)sms * 8;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        uniform_trace_kernel<<<(unsigned)blocks, threads, 0, st>>>(n, s, len, trace);
    }
    if (array_out) {
        uint64_t blocks = ((uint64_t)n + 255) / 256;
        const uint64_t cap = (uint64_t)sms * 8;
        if (blocks > cap) blocks = cap;
        uniform_array_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, s, array_out);
    }
    return cudaGetLastError();
}

cudaError_t build_chain(const uint32_t *next, uint32_t n, uint64_t len, uint32_t *trace,
                        uint32_t *status, cudaStream_t st) {
    if (len) chain_walk_kernel<<<1, 1, 0, st>>>(next, n, len, trace, status);
    return cudaGetLastError();
}

cudaError_t build_uniform_batch(const pchase_trace *traces, uint32_t count, uint32_t *out,
                                const uint64_t *offsets, cudaStream_t st) {
    thread_local BatchParams p;  // host staging of the kernel's parameter block
    for (uint32_t base = 0; base < count; base += kBatchPerLaunch) {
        const uint32_t m = count - base < (uint32_t)kBatchPerLaunch ? count - base
                                                                    : (uint32_t)kBatchPerLaunch;
        for (uint32_t i = 0; i < m; ++i) {
            const pchase_trace &d = traces[base + i];
            p.e[i].n = d.n_elems;
            p.e[i].s = d.stride;
            p.e[i].len = d.len;
            p.e[i].off = offsets[base + i];
        }
        uniform_batch_kernel<<<m, 512, 0, st>>>(p, out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pchase
