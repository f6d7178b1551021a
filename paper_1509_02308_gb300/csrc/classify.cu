// S4: latency -> hit/miss, and the matcher's canonical pick.
//
// Sec. 4.1 models a P-chase latency as t0 (hit) or t0 + t_m (miss); the paper
// states no cut rule.  The rule implemented (the same one the CPU oracle
// states): over one observation of n latencies, set aside the floor(n/200)
// largest, take the largest gap between consecutive distinct kept values (the
// lowest on ties) and cut at (lo + hi) * 0.5f.
//
// GPU form, without a sort:
//   1. radix select (four 8-bit digit passes over order-preserving keys) finds
//      the cut value v[keep-1] exactly, and the minimum;
//   2. maximum gap by pigeonhole (Gonzalez's linear-time maximum-gap method):
//      the kept values go into 2*keep equal-width buckets keeping each
//      bucket's min and max; a gap inside one bucket is at most half the
//      average gap, so the largest gap lies between consecutive non-empty
//      buckets, and is computed from the same two floats as a sort would give;
//   3. a block scans the buckets in order (first maximum wins) and a grid
//      writes the miss bits with __ballot_sync.
#include <mutex>

#include <algorithm>

#include "pchase_internal.cuh"

namespace pchase {

namespace {

__device__ __forceinline__ uint32_t fkey(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fval(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

struct ObsMeta {
    uint32_t cut_key;
    uint32_t min_key;
    uint32_t nb;   // buckets (0: no gap possible)
    float thr;
};

// One CTA per observation: cut value by radix select, minimum, bucket init.
__global__ void __launch_bounds__(1024) select_cut_kernel(const float *lat,
                                                          const uint64_t *offsets,
                                                          uint64_t max_len, ObsMeta *meta,
                                                          uint2 *buckets) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_prefix, s_mask, s_k, s_min;
    const uint32_t o = blockIdx.x;
    const uint64_t b0 = offsets[o], n = offsets[o + 1] - b0;
    const float *x = lat + b0;
    const uint64_t keep = n - n / 200;
    if (threadIdx.x == 0) {
        s_prefix = 0;
        s_mask = 0;
        s_k = (uint32_t)keep;
        s_min = 0xFFFFFFFFu;
    }
    __syncthreads();
    if (n == 0) {
        if (threadIdx.x == 0) meta[o] = ObsMeta{0, 0, 0, 0.0f};
        return;
    }
    if (n > max_len) {
        // the observation's bucket slice holds 2 * max_len buckets: an
        // observation longer than the caller's max_len is refused (NaN cut, so
        // no latency is above it and every bit stays 0) instead of writing
        // into the next observation's slice or past the scratch
        if (threadIdx.x == 0) meta[o] = ObsMeta{0, 0, 0, __int_as_float(0x7FC00000)};
        return;
    }
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const uint32_t prefix = s_prefix, mask = s_mask;
        uint32_t mn = 0xFFFFFFFFu;
        // latencies crowd into a few digits, so lanes with the same digit add
        // their count with one atomic (warp-aggregated)
        for (uint64_t i0 = 0; i0 < n; i0 += blockDim.x) {
            const uint64_t i = i0 + threadIdx.x;
            uint32_t d = 0xFFFFFFFFu;
            if (i < n) {
                const uint32_t k = fkey(x[i]);
                if (pass == 0) mn = min(mn, k);
                if ((k & mask) == prefix) d = (k >> shift) & 255u;
            }
            const uint32_t peers = __match_any_sync(kFull, d);
            if (d != 0xFFFFFFFFu && (peers & ((1u << (threadIdx.x & 31)) - 1u)) == 0)
                atomicAdd(&hist[d], (uint32_t)__popc(peers));
        }
        if (pass == 0) {
            mn = __reduce_min_sync(kFull, mn);
            if ((threadIdx.x & 31) == 0) atomicMin(&s_min, mn);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t cum = 0, k = s_k;
            for (uint32_t d = 0; d < 256; ++d) {
                if (cum + hist[d] >= k) {
                    s_prefix = prefix | (d << shift);
                    s_mask = mask | (255u << shift);
                    s_k = k - cum;
                    break;
                }
                cum += hist[d];
            }
        }
        __syncthreads();
    }
    const uint32_t cut = s_prefix, mnk = s_min;
    const uint32_t nb = (cut == mnk) ? 0u : (uint32_t)(2 * keep);
    uint2 *bk = buckets + (uint64_t)o * 2 * max_len;
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) bk[i] = make_uint2(0xFFFFFFFFu, 0u);
    if (threadIdx.x == 0) meta[o] = ObsMeta{cut, mnk, nb, fval(cut)};
}

// Kept values into buckets (min / max key per bucket).
__global__ void bucket_kernel(const float *lat, const uint64_t *offsets, uint64_t max_len,
                              const ObsMeta *meta, uint2 *buckets) {
    const uint32_t o = blockIdx.y;
    const ObsMeta m = meta[o];
    if (m.nb == 0) return;
    const uint64_t b0 = offsets[o], n = offsets[o + 1] - b0;
    const float lo = fval(m.min_key), hi = fval(m.cut_key);
    const float scale = (float)m.nb / (hi - lo);
    uint2 *bk = buckets + (uint64_t)o * 2 * max_len;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const float v = lat[b0 + i];
        const uint32_t k = fkey(v);
        if (k > m.cut_key) continue;
        uint32_t bi = (uint32_t)((v - lo) * scale);
        if (bi >= m.nb) bi = m.nb - 1;
        atomicMin(&bk[bi].x, k);
        atomicMax(&bk[bi].y, k);
    }
}

struct GapPart {
    uint32_t first_min, last_max;  // keys; first_min = 0xFFFFFFFF when empty
    float gap, lo, hi;
};

// One CTA per observation: the largest gap between consecutive non-empty
// buckets, first one on ties; each thread scans a contiguous range, then one
// warp-serial pass joins the ranges in order.
__global__ void __launch_bounds__(1024) gap_kernel(uint64_t max_len, ObsMeta *meta,
                                                   const uint2 *buckets, float *thresh_out) {
    __shared__ GapPart part[1024];
    const uint32_t o = blockIdx.x;
    ObsMeta m = meta[o];
    if (m.nb == 0) {
        if (threadIdx.x == 0 && thresh_out) thresh_out[o] = m.thr;
        return;
    }
    const uint2 *bk = buckets + (uint64_t)o * 2 * max_len;
    const uint32_t per = (m.nb + blockDim.x - 1) / blockDim.x;
    const uint32_t beg = threadIdx.x * per;
    const uint32_t end = min(m.nb, beg + per);
    GapPart p{0xFFFFFFFFu, 0u, -1.0f, 0.0f, 0.0f};
    for (uint32_t i = beg; i < end; ++i) {
        const uint2 b = bk[i];
        if (b.x == 0xFFFFFFFFu) continue;
        if (p.first_min == 0xFFFFFFFFu) {
            p.first_min = b.x;
        } else {
            const float a = fval(p.last_max), c = fval(b.x);
            const float g = c - a;
            if (g > p.gap) { p.gap = g; p.lo = a; p.hi = c; }
        }
        p.last_max = b.y;
    }
    part[threadIdx.x] = p;
    __syncthreads();
    if (threadIdx.x == 0) {
        float best = 0.0f, lo = 0.0f, hi = 0.0f;
        bool found = false, have_prev = false;
        uint32_t prev_max = 0;
        for (uint32_t t = 0; t < blockDim.x; ++t) {
            const GapPart q = part[t];
            if (q.first_min == 0xFFFFFFFFu) continue;
            if (have_prev) {
                const float a = fval(prev_max), c = fval(q.first_min);
                const float g = c - a;
                if (g > best) { best = g; lo = a; hi = c; found = true; }
            }
            if (q.gap > best) { best = q.gap; lo = q.lo; hi = q.hi; found = true; }
            prev_max = q.last_max;
            have_prev = true;
        }
        m.thr = found ? (lo + hi) * 0.5f : fval(m.cut_key);
        meta[o].thr = m.thr;
        if (thresh_out) thresh_out[o] = m.thr;
    }
}

// Miss bits of segment s against the threshold of observation s / per_seg
// (per_seg segments per observation; 0: one pooled threshold)
// or of observation 0 (every segment pooled into one observation).
__global__ void bits_kernel(const float *lat, const uint64_t *seg_offsets, int per_seg,
                            uint32_t n_seg, const ObsMeta *meta, uint32_t *bits,
                            const uint64_t *word_offsets) {
    const uint32_t s = blockIdx.y;
    const float thr = meta[per_seg ? s / (uint32_t)per_seg : 0].thr;
    const uint64_t b0 = seg_offsets[s], n = seg_offsets[s + 1] - b0;
    const uint64_t words = (n + 31) / 32;
    const uint64_t wo = word_offsets[s];
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t w = warp; w < words; w += nwarps) {
        const uint64_t i = w * 32 + lane;
        const bool miss = i < n && lat[b0 + i] > thr;
        const uint32_t v = __ballot_sync(kFull, miss);
        if (lane == 0) bits[wo + w] = v;
    }
}

// Canonical pick: one block.
__device__ __forceinline__ bool better(const pchase_geom *g, const uint64_t *d, uint32_t x,
                                       uint32_t y) {
    if (d[x] != d[y]) return d[x] < d[y];
    const pchase_geom &a = g[x], &b = g[y];
    if (a.policy != b.policy) return a.policy < b.policy;
    if (a.line_bytes != b.line_bytes) return a.line_bytes > b.line_bytes;
    if (a.ways != b.ways) return a.ways < b.ways;
    if (a.C_bytes != b.C_bytes) return a.C_bytes < b.C_bytes;
    return x < y;
}

__global__ void __launch_bounds__(1024) pick_kernel(const pchase_geom *geoms, const uint64_t *dist,
                                                    uint32_t n, uint32_t *pick) {
    // block o picks for observation o: distances dist + o * n
    dist += (size_t)blockIdx.x * n;
    pick += 2ull * blockIdx.x;
    __shared__ uint32_t best[1024];
    __shared__ uint32_t count;
    uint32_t b = 0xFFFFFFFFu;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x)
        if (b == 0xFFFFFFFFu || better(geoms, dist, i, b)) b = i;
    best[threadIdx.x] = b;
    if (threadIdx.x == 0) count = 0;
    __syncthreads();
    for (uint32_t s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const uint32_t x = best[threadIdx.x], y = best[threadIdx.x + s];
            if (y != 0xFFFFFFFFu && (x == 0xFFFFFFFFu || better(geoms, dist, y, x)))
                best[threadIdx.x] = y;
        }
        __syncthreads();
    }
    const uint32_t w = best[0];
    uint32_t c = 0;
    if (w != 0xFFFFFFFFu)
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) c += dist[i] == dist[w];
    atomicAdd(&count, c);
    __syncthreads();
    if (threadIdx.x == 0) {
        pick[0] = w == 0xFFFFFFFFu ? n : w;
        pick[1] = count;
    }
}

}  // namespace

size_t classify_meta_bytes(uint32_t n_obs) { return ((size_t)n_obs * sizeof(ObsMeta) + 255) & ~size_t(255); }

size_t classify_bucket_bytes(uint32_t n_obs, uint64_t max_len) {
    return (size_t)n_obs * 2 * (max_len ? max_len : 1) * sizeof(uint2);
}

// Thresholds for n_obs observations (lat + offsets), buckets in `work`.
cudaError_t classify_thresholds(const float *lat, const uint64_t *offsets, uint32_t n_obs,
                                uint64_t max_len, void *meta_mem, void *bucket_mem,
                                float *thresh_out, cudaStream_t st, int sms) {
    ObsMeta *meta = static_cast<ObsMeta *>(meta_mem);
    uint2 *bk = static_cast<uint2 *>(bucket_mem);
    select_cut_kernel<<<n_obs, 1024, 0, st>>>(lat, offsets, max_len, meta, bk);
    uint32_t gx = (uint32_t)((max_len + 255) / 256);
    const uint32_t cap = (uint32_t)(sms > 0 ? sms : 1) * 8;
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    bucket_kernel<<<dim3(gx, n_obs), 256, 0, st>>>(lat, offsets, max_len, meta, bk);
    gap_kernel<<<n_obs, 1024, 0, st>>>(max_len, meta, bk, thresh_out);
    return cudaGetLastError();
}

cudaError_t classify_bits(const float *lat, const uint64_t *seg_offsets, int per_seg,
                          uint32_t n_seg, uint64_t max_seg_len, const void *meta_mem,
                          uint32_t *bits, const uint64_t *word_offsets, cudaStream_t st,
                          int sms) {
    uint32_t gx = (uint32_t)((max_seg_len + 255) / 256);
    const uint32_t cap = (uint32_t)(sms > 0 ? sms : 1) * 8;
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    bits_kernel<<<dim3(gx, n_seg), 256, 0, st>>>(lat, seg_offsets, per_seg, n_seg,
                                                  static_cast<const ObsMeta *>(meta_mem), bits,
                                                  word_offsets);
    return cudaGetLastError();
}

cudaError_t canonical_pick(const pchase_geom *geoms, const uint64_t *dist, uint32_t n,
                           uint32_t *pick, cudaStream_t st, uint32_t n_obs) {
    pick_kernel<<<n_obs ? n_obs : 1, 1024, 0, st>>>(geoms, dist, n, pick);
    return cudaGetLastError();
}

// Segment and word offsets of n_obs observations laid out back to back, each
// L latencies in plan-trace order (T traces, seg[T + 1], owo[T]).
__global__ void batch_offsets_kernel(const uint64_t *seg, const uint64_t *owo, uint32_t T,
                                     uint32_t n_obs, uint64_t L, uint64_t obs_words,
                                     uint64_t *obs_off, uint64_t *seg_out, uint64_t *wo_out) {
    const uint64_t n = (uint64_t)n_obs * T;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t o = i / T, t = i % T;
        if (i == n) {
            seg_out[n] = n_obs * L;
        } else {
            seg_out[i] = o * L + seg[t];
            wo_out[i] = o * obs_words + owo[t];
        }
        if (i <= n_obs) obs_off[i] = i * L;
    }
}

cudaError_t batch_offsets(const uint64_t *seg, const uint64_t *owo, uint32_t T, uint32_t n_obs,
                          uint64_t L, uint64_t obs_words, uint64_t *obs_off, uint64_t *seg_out,
                          uint64_t *wo_out, cudaStream_t st) {
    const uint64_t n = (uint64_t)n_obs * T + 1;
    const unsigned blocks = (unsigned)std::min<uint64_t>((n + 255) / 256, 1024);
    batch_offsets_kernel<<<blocks, 256, 0, st>>>(seg, owo, T, n_obs, L, obs_words, obs_off,
                                                 seg_out, wo_out);
    return cudaGetLastError();
}

// ------------------------------------------------ classification without allocation
// Scratch of pchase_classify_noalloc: a fixed array in the library's own
// device memory, shared by every call on a device and kept until the process
// exits.  Host code cannot use the name g_noalloc_scratch as an address: it
// names a host-side stand-in, so the device address is looked up once per
// device with cudaGetSymbolAddress.
constexpr size_t kNoallocScratchBytes = 8u << 20;
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices];

// Device address of the scratch array for the current device (set up on the
// first call per device).
cudaError_t noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}
}  // namespace

}  // namespace pchase

extern "C" size_t pchase_classify_noalloc_limit_bytes(void) {
    return pchase::kNoallocScratchBytes;
}

extern "C" int pchase_classify_noalloc(const float *lat, const uint64_t *offsets, uint32_t n_obs,
                                       uint64_t max_len, uint32_t *bits_out,
                                       const uint64_t *bit_word_offsets, float *thresh_out,
                                       pchase_stream_t stream) {
    using namespace pchase;
    if (n_obs == 0) return PCHASE_OK;
    if (!lat || !offsets || !bits_out || !bit_word_offsets)
        return set_last_error(PCHASE_EINVAL, "pchase_classify_noalloc: NULL argument");
    const size_t meta = classify_meta_bytes(n_obs);
    const size_t bk = (classify_bucket_bytes(n_obs, max_len) + 255) & ~size_t(255);
    if (max_len > (kNoallocScratchBytes >> 4) || n_obs > (kNoallocScratchBytes >> 4) ||
        meta + bk > kNoallocScratchBytes)
        return set_last_error(PCHASE_ERANGE,
                              "pchase_classify_noalloc: n_obs * max_len too large for the "
                              "8 MiB static scratch (need 16 * n_obs * (max_len + 1) bytes, "
                              "rounded up); use pchase_classify with a workspace");
    void *scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess)
        return set_last_error(PCHASE_ECUDA, "pchase_classify_noalloc: cudaGetSymbolAddress failed");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint8_t *w = static_cast<uint8_t *>(scratch);
    // the kernels write every metadata entry and initialise every bucket they
    // read, so nothing left by an earlier call is consumed
    e = classify_thresholds(lat, offsets, n_obs, max_len, w, w + meta, thresh_out, st, sms);
    if (e == cudaSuccess)
        e = classify_bits(lat, offsets, 1, n_obs, max_len, w, bits_out, bit_word_offsets, st, sms);
    if (e != cudaSuccess) return set_last_error(PCHASE_ECUDA, cudaGetErrorString(e));
    return PCHASE_OK;
}
