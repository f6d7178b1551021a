// Batched set-associative cache simulator (S2 decode, S3 set simulation) and
// its Hamming-compare form for the exhaustive matcher (S5).
//
// Model (Assumptions 1-3 and Fig. 2, Sec. 4.1): line = (4 * index) / b,
// set = line mod T; an access hits when its line is held by its set; a miss
// fills the lowest invalid way, else evicts by LRU (oldest use), FIFO (oldest
// fill) or RANDOM (SplitMix64-keyed way).
//
// Mapping onto the GPU:
//   * one warp per item (geometry x trace), pulled from a per-class atomic
//     queue by persistent CTAs; the item's whole cache state lives in the
//     warp's slice of shared memory;
//   * the warp streams the trace 32 consecutive accesses at a time (one
//     coalesced 128-byte load; analytic uniform chains are generated in
//     registers instead), decodes set and line in registers, and marks the
//     accesses that repeat the previous access's line: such an access is a hit
//     under every policy and changes no recency order, so only run heads touch
//     set state;
//   * heads in different sets are independent, heads in the same set must go
//     in trace order: __match_any_sync groups the heads by set, and a head of
//     rank r inside its group acts in round r;
//   * one access is resolved by one lane: "scan" sets (few ways) keep
//     {line, stamp} per way and scan them; "table" sets (many ways) find the
//     way through a per-item line table (line -> way + 1) and keep LRU order
//     as a doubly linked list, FIFO order as a ring pointer;
//   * miss bits come from __ballot_sync, 32 steps are buffered one word per
//     lane and stored as one coalesced 128-byte write.
#include "pchase_internal.cuh"

namespace pchase {

namespace {

// Dynamic shared memory of the simulator kernel: one arena per warp.
extern __shared__ __align__(16) uint8_t g_smem[];

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

constexpr uint16_t kNil = 0xFFFF;

// ----------------------------------------------------------- scan sets
// Arena: uint2 slot[T*a] = {line, stamp}; RANDOM adds uint32 evictions[T].
// Stamps: an invalid way w holds stamp w (< a), a filled way t + a, where t
// is the access time of its last use (LRU) or of its fill (FIFO, RANDOM), so
// the smallest stamp is the lowest invalid way if any, else the victim.
template <int POLICY, int A>
struct ScanSets {
    uint2 *slot;
    uint32_t *evict;
    uint32_t ways;
    uint64_t seed;

    __device__ __forceinline__ void init(uint8_t *arena, const SimItem &it, int lane) {
        ways = A ? A : it.ways;
        seed = it.seed;
        slot = reinterpret_cast<uint2 *>(arena);
        const uint32_t n = it.sets * ways;
        evict = reinterpret_cast<uint32_t *>(arena + 8ull * n);
        for (uint32_t i = lane; i < n; i += 32) slot[i] = make_uint2(kInvalidLine, i % ways);
        if (POLICY == PCHASE_RANDOM)
            for (uint32_t i = lane; i < it.sets; i += 32) evict[i] = 0;
    }

    __device__ __forceinline__ bool access(uint32_t set, uint32_t line, uint32_t t) {
        const uint32_t a = A ? A : ways;
        uint2 *s = slot + set * a;
        int hit = -1;
        uint32_t best = 0xFFFFFFFFu;
        uint32_t bw = 0;
#pragma unroll
        for (uint32_t w = 0; w < (A ? A : 32); ++w) {
            if (!A && w >= a) break;
            const uint2 e = s[w];
            if (e.x == line) hit = (int)w;
            if (e.y < best) { best = e.y; bw = w; }
        }
        if (hit >= 0) {
            if (POLICY == PCHASE_LRU) s[hit].y = t + a;
            return false;
        }
        uint32_t v = bw;
        if (POLICY == PCHASE_RANDOM && best >= a) {
            const uint32_t k = evict[set];
            evict[set] = k + 1;
            v = random_way(seed, set, k, a);
        }
        s[v] = make_uint2(line, t + a);
        return true;
    }
};

// ---------------------------------------------------------- table sets
// Arena: uint2 meta[T]; uint32 sline[T*a]; (LRU) uint16 prev[T*a], next[T*a];
// uint16 table[table_n] (line -> way + 1, 0 = absent).
//   LRU meta = {head | tail << 16, filled}; FIFO meta.x = ring pointer;
//   RANDOM meta = {filled, evictions}.
template <int POLICY>
struct TableSets {
    uint2 *meta;
    uint32_t *sline;
    uint16_t *prv, *nxt, *tab;
    uint32_t ways;
    uint64_t seed;

    __device__ __forceinline__ void init(uint8_t *arena, const SimItem &it, int lane) {
        ways = it.ways;
        seed = it.seed;
        const uint32_t n = it.sets * ways;
        size_t off = 0;
        meta = reinterpret_cast<uint2 *>(arena);
        off += 8ull * it.sets;
        sline = reinterpret_cast<uint32_t *>(arena + off);
        off += 4ull * n;
        if (POLICY == PCHASE_LRU) {
            prv = reinterpret_cast<uint16_t *>(arena + off);
            off += 2ull * n;
            nxt = reinterpret_cast<uint16_t *>(arena + off);
            off += 2ull * n;
        }
        tab = reinterpret_cast<uint16_t *>(arena + off);
        const uint2 m0 = POLICY == PCHASE_LRU ? make_uint2(0xFFFFFFFFu, 0) : make_uint2(0, 0);
        for (uint32_t i = lane; i < it.sets; i += 32) meta[i] = m0;
        for (uint32_t i = lane; i < n; i += 32) sline[i] = kInvalidLine;
        uint32_t *t32 = reinterpret_cast<uint32_t *>(tab);
        for (uint32_t i = lane; i < (it.table_n + 1) / 2; i += 32) t32[i] = 0;
    }

    __device__ __forceinline__ bool access(uint32_t set, uint32_t line, uint32_t) {
        const uint32_t a = ways;
        const uint32_t base = set * a;
        const uint32_t w1 = tab[line];
        if (POLICY == PCHASE_LRU) {
            uint2 m = meta[set];
            uint32_t head = m.x & 0xFFFFu, tail = m.x >> 16;
            uint32_t v;
            if (w1) {
                v = w1 - 1;
                if (v == head) return false;
            } else if (m.y < a) {
                // fill the lowest invalid way and push it in front
                v = m.y;
                m.y += 1;
                prv[base + v] = kNil;
                nxt[base + v] = (uint16_t)head;
                if (head != kNil) prv[base + head] = (uint16_t)v; else tail = v;
                head = v;
                sline[base + v] = line;
                tab[line] = (uint16_t)(v + 1);
                meta[set] = make_uint2(head | (tail << 16), m.y);
                return true;
            } else {
                v = tail;
                tab[sline[base + v]] = 0;
                sline[base + v] = line;
                tab[line] = (uint16_t)(v + 1);
                if (v == head) return true;  // a == 1
            }
            // move v (not the head) to the front
            const uint32_t p = prv[base + v], q = nxt[base + v];
            nxt[base + p] = (uint16_t)q;
            if (q != kNil) prv[base + q] = (uint16_t)p; else tail = p;
            prv[base + v] = kNil;
            nxt[base + v] = (uint16_t)head;
            prv[base + head] = (uint16_t)v;
            head = v;
            meta[set] = make_uint2(head | (tail << 16), m.y);
            return w1 == 0;
        } else if (POLICY == PCHASE_FIFO) {
            if (w1) return false;
            const uint32_t v = meta[set].x;
            meta[set].x = (v + 1 == a) ? 0 : v + 1;
            const uint32_t old = sline[base + v];
            if (old != kInvalidLine) tab[old] = 0;
            sline[base + v] = line;
            tab[line] = (uint16_t)(v + 1);
            return true;
        } else {
            if (w1) return false;
            uint2 m = meta[set];
            uint32_t v;
            if (m.x < a) {
                v = m.x;
                m.x += 1;
            } else {
                v = random_way(seed, set, m.y, a);
                m.y += 1;
                tab[sline[base + v]] = 0;
            }
            meta[set] = m;
            sline[base + v] = line;
            tab[line] = (uint16_t)(v + 1);
            return true;
        }
    }
};

// --------------------------------------------------------------- item loop
template <typename Sets>
__device__ __forceinline__ void run_item(const SimItem &it, Sets &S, const SimOut &out,
                                         int lane) {
    const uint32_t len = it.len;
    const uint32_t *__restrict__ idxp = it.idx;
    const uint32_t N = it.n_elems;
    const uint32_t lt = lanemask_lt();
    const bool ham = out.dist != nullptr;
    const uint64_t wbase = out.word_offsets ? out.word_offsets[it.out_item] : it.word_off;
    const uint64_t obase = ham ? out.obs_word_offsets[it.obs] : 0;

    uint32_t carry = kInvalidLine;
    uint32_t myword = 0;
    uint32_t tot = 0, aft = 0;
    uint64_t dsum = 0;  // Hamming distance so far (warp-uniform)

    // analytic chain: access t visits (t * stride) mod N
    uint32_t aj = 0, ainc = 0;
    if (!idxp && N) {
        aj = (uint32_t)(((uint64_t)lane * it.stride) % N);
        ainc = (uint32_t)((32ull * it.stride) % N);
    }
    const uint32_t nsteps = (len + 31) >> 5;
    uint32_t nxt = (idxp && (uint32_t)lane < len) ? idxp[lane] : 0;

    for (uint32_t st = 0; st < nsteps; ++st) {
        const uint32_t t = (st << 5) + lane;
        bool active = t < len;
        uint32_t j;
        if (idxp) {
            j = nxt;
            const uint32_t t2 = t + 32;
            nxt = (t2 < len) ? idxp[t2] : 0;
        } else {
            j = aj;
            aj = (aj >= N - ainc) ? aj - (N - ainc) : aj + ainc;
        }
        if (active && j >= N) {
            atomicOr(out.status, PCHASE_DEV_INDEX_RANGE);
            active = false;
        }
        const uint32_t line = j >> it.lsh;
        const uint32_t set = line - div_q(line, it.magic_m, it.s1, it.s2) * it.sets;
        uint32_t prev = __shfl_up_sync(kFull, line, 1);
        if (lane == 0) prev = carry;
        carry = __shfl_sync(kFull, line, 31);
        const bool head = active && line != prev;

        const uint32_t key = head ? set : (0x80000000u | (uint32_t)lane);
        const uint32_t peers = __match_any_sync(kFull, key);
        const uint32_t rank = __popc(peers & lt);
        const uint32_t rounds = __reduce_max_sync(kFull, head ? rank + 1 : 0u);
        bool miss = false;
        for (uint32_t r = 0; r < rounds; ++r) {
            if (head && rank == r) miss = S.access(set, line, t);
            __syncwarp();
        }
        const uint32_t bits = __ballot_sync(kFull, miss);
        const uint32_t after = __ballot_sync(kFull, active && t >= it.warmup);
        tot += __popc(bits);
        aft += __popc(bits & after);
        const uint32_t slot = st & 31;
        if ((uint32_t)lane == slot) myword = bits;
        if (slot == 31 || st + 1 == nsteps) {
            const uint64_t w0 = (uint64_t)(st & ~31u);
            uint32_t dl = 0;
            if ((uint32_t)lane <= slot) {
                if (ham) {
                    dl = __popc(out.observed[obase + w0 + lane] ^ myword);
                } else if (out.bitmaps) {
                    out.bitmaps[wbase + w0 + lane] = myword;
                }
            }
            myword = 0;
            if (ham) {
                dsum += __reduce_add_sync(kFull, dl);
                if (dsum > out.stop_above) break;
            }
        }
    }
    if (ham) {
        if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long *>(out.dist + it.cand),
                                 (unsigned long long)dsum);
    } else if (lane == 0 && out.miss_counts) {
        out.miss_counts[2ull * it.out_item] = tot;
        out.miss_counts[2ull * it.out_item + 1] = aft;
    }
}

template <int POLICY, int A>
__device__ __forceinline__ void run_scan(const SimItem &it, uint32_t arena_off, const SimOut &out,
                                         int lane) {
    ScanSets<POLICY, A> S;
    S.init(g_smem + arena_off, it, lane);
    __syncwarp();
    run_item(it, S, out, lane);
}

template <int POLICY>
__device__ __noinline__ void run_scan_any(const SimItem &it, uint32_t arena, const SimOut &out,
                                          int lane) {
    switch (it.ways) {
        case 1: run_scan<POLICY, 1>(it, arena, out, lane); break;
        case 2: run_scan<POLICY, 2>(it, arena, out, lane); break;
        case 4: run_scan<POLICY, 4>(it, arena, out, lane); break;
        case 8: run_scan<POLICY, 8>(it, arena, out, lane); break;
        case 16: run_scan<POLICY, 16>(it, arena, out, lane); break;
        case 32: run_scan<POLICY, 32>(it, arena, out, lane); break;
        default: run_scan<POLICY, 0>(it, arena, out, lane); break;
    }
}

template <int POLICY>
__device__ __noinline__ void run_table(const SimItem &it, uint32_t arena, const SimOut &out,
                                       int lane) {
    TableSets<POLICY> S;
    S.init(g_smem + arena, it, lane);
    __syncwarp();
    run_item(it, S, out, lane);
}

__global__ void __launch_bounds__(512) sim_kernel(const SimItem *__restrict__ items,
                                                  ClassLaunch cls, uint32_t *queue,
                                                  SimOut out) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t arena = (uint32_t)warp * cls.arena_bytes;
    for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = atomicAdd(queue, 1u);
        k = __shfl_sync(kFull, k, 0);
        if (k >= cls.count) break;
        const SimItem it = items[cls.first + k];
        if (it.mode == kModeScan) {
            if (it.policy == PCHASE_LRU) run_scan_any<PCHASE_LRU>(it, arena, out, lane);
            else if (it.policy == PCHASE_FIFO) run_scan_any<PCHASE_FIFO>(it, arena, out, lane);
            else run_scan_any<PCHASE_RANDOM>(it, arena, out, lane);
        } else {
            if (it.policy == PCHASE_LRU) run_table<PCHASE_LRU>(it, arena, out, lane);
            else if (it.policy == PCHASE_FIFO) run_table<PCHASE_FIFO>(it, arena, out, lane);
            else run_table<PCHASE_RANDOM>(it, arena, out, lane);
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_sim_class(const SimItem *items, const ClassLaunch &cls, uint32_t *queue,
                             int grid, const SimOut &out, bool, cudaStream_t st) {
    const size_t smem = (size_t)cls.arena_bytes * cls.warps;
    cudaError_t e = cudaFuncSetAttribute(sim_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    sim_kernel<<<grid, cls.warps * 32, smem, st>>>(items, cls, queue, out);
    return cudaGetLastError();
}

int sim_max_ctas_per_sm(const ClassLaunch &cls, bool) {
    const size_t smem = (size_t)cls.arena_bytes * cls.warps;
    if (cudaFuncSetAttribute(sim_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sim_kernel, cls.warps * 32, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

}  // namespace pchase
