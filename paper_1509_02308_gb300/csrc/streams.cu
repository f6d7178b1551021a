// Head streams of the items a plan splits by sets (S3, S6).
//
// A part of an item split into K parts by sets simulates only the accesses
// that fall in its own sets, but it has to find them: gathering them itself
// means reading and decoding the whole trace once per part, K times per item,
// on the part's own dependent chain.  Here the batch's split items are
// partitioned once, in parallel, before the simulator runs: each part gets
// the stream of its run heads (an access whose line differs from the
// previous access's line, the accesses every policy resolves; the others hit
// and change nothing, Assumptions 1-3, Sec. 4.1) as entries {local line,
// position}, in trace order.  These are exactly the heads the part would
// queue by gathering, so the simulation that follows is unchanged.
//
// Three launches: count (one warp per segment of kSegAccesses accesses, a
// count per part), offsets (one warp per item: lane k scans part k's counts
// over the item's segments, then the parts' totals are laid out one after
// another), write (the segments' warps again, each head to its part's
// stream at its segment's offset plus its rank).
//
// The same launches take a census of each LRU item cut in time: the count
// launch marks the line ids its segments use (a bitmap per warp in shared
// memory, OR-ed into the item's bitmap), and the offsets launch counts each
// set's distinct lines from the bitmap.  A time part that rebuilds its sets'
// recency order from the accesses before it needs, per set, min(a, that
// count) lines: once every set has them it can stop reading back, instead of
// reading to the trace's start whenever some set is never visited or holds
// fewer than a lines (LRU state is the a most recent distinct lines of each
// set, Sec. 4.1's model).
#include "pchase_internal.cuh"

namespace pchase {
namespace {

constexpr int kStreamWarps = 8;  // warps per CTA of the count and write launches

__device__ __forceinline__ uint32_t lanemask_lt_() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Decoded access t of a job's trace: its line as the simulator numbers it
// (line shift, then the set-mapping renumbering) and whether the index is in
// range.
struct Decoder {
    const uint32_t *idx;
    uint32_t N, stride, lsh, mk, gT, gm, gs1, gs2;
    __device__ __forceinline__ explicit Decoder(const SimItem &it)
        : idx(it.idx), N(it.n_elems), stride(it.stride), lsh(it.lsh & 255u),
          mk((it.lsh >> 8) & 255u), gT(it.gsets), gm(it.gmagic), gs1(it.gs1), gs2(it.gs2) {}
    __device__ __forceinline__ uint32_t index(uint32_t t) const {
        return idx ? idx[t] : (N ? (uint32_t)(((uint64_t)t * stride) % N) : 0u);
    }
    __device__ __forceinline__ uint32_t line(uint32_t j) const {
        const uint32_t ln = j >> lsh;
        return mk ? remap_line(ln, mk, gT, gm, gs1, gs2) : ln;
    }
};

// Which part access t's head belongs to, and its local line; take: it is a
// head (in range, line unlike the previous access's).
struct Split {
    uint32_t psh, pmask, K, km, ks1, ks2, sets, gT, gm, gs1, gs2;
    __device__ __forceinline__ explicit Split(const SimItem &it)
        : psh(it.psh), pmask((1u << it.psh) - 1u), K(it.kcnt), km(it.kmagic), ks1(it.ks1),
          ks2(it.ks2), sets(it.sets), gT(it.gsets), gm(it.gmagic), gs1(it.gs1), gs2(it.gs2) {}
    // part of line ln, and its line within the part
    __device__ __forceinline__ uint32_t part(uint32_t ln, uint32_t &lp) const {
        const uint32_t q = div_q(ln, gm, gs1, gs2);
        const uint32_t set = ln - q * gT;
        const uint32_t sg = set >> psh;
        const uint32_t kq = div_q(sg, km, ks1, ks2);
        lp = ((kq << psh) | (set & pmask)) + q * sets;
        return sg - kq * K;
    }
};

// Walks segment `seg` of its job 32 accesses at a time; f(t, take, part, lp)
// is called by every lane for every chunk (take false past the end).
template <typename F>
__device__ __forceinline__ void walk_segment(const SimItem &it, uint32_t seg, int lane,
                                             uint32_t *status, F &&f) {
    const Decoder D(it);
    const Split S(it);
    const uint32_t len = it.len;
    const uint32_t t0 = seg * kSegAccesses;
    const uint32_t t1 = min(len, t0 + kSegAccesses);
    // line of the access before the segment (none before the trace)
    uint32_t carry = kInvalidLine;
    if (t0 > 0) carry = D.line(D.index(t0 - 1));
    bool bad = false;
    uint32_t jn = t0 + (uint32_t)lane < t1 ? D.index(t0 + (uint32_t)lane) : 0u;
    for (uint32_t c = t0; c < t1; c += 32) {
        const uint32_t t = c + (uint32_t)lane;
        bool valid = t < t1;
        const uint32_t j = jn;
        jn = t + 32 < t1 ? D.index(t + 32) : 0u;
        if (valid && j >= D.N) {
            bad = true;
            valid = false;
        }
        const uint32_t ln = D.line(j);
        const uint32_t rot = __shfl_sync(kFull, ln, (lane + 31) & 31);
        const uint32_t prev = lane == 0 ? carry : rot;
        carry = __shfl_sync(kFull, ln, 31);
        uint32_t lp = 0;
        const uint32_t k = S.part(ln, lp);
        f(t, valid && ln != prev, k, lp);
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(status, PCHASE_DEV_INDEX_RANGE);
}

// Line id of index j as a time part keys it (compact lines: the id of
// line * lstep), and its set (BatchLRU::set_of's numbering).
struct CensusKey {
    uint32_t lsh, mk, gT, gm, gs1, gs2, lcomp, lstep, sets, sm, ss1, ss2;
    __device__ __forceinline__ explicit CensusKey(const SimItem &it)
        : lsh(it.lsh & 255u), mk((it.lsh >> 8) & 255u), gT(it.gsets), gm(it.gmagic), gs1(it.gs1),
          gs2(it.gs2), lcomp((it.lsh >> 18) & 1u), lstep(((it.lsh >> 18) & 1u) ? it.gsets : 1u),
          sets(it.sets), sm(it.magic_m), ss1(it.s1), ss2(it.s2) {}
    __device__ __forceinline__ uint32_t id(uint32_t j) const {
        const uint32_t ln = j >> lsh;
        if (lcomp) return div_q(ln, gm, gs1, gs2);
        return mk ? remap_line(ln, mk, gT, gm, gs1, gs2) : ln;
    }
    __device__ __forceinline__ uint32_t set(uint32_t id) const {
        const uint32_t l = id * lstep;
        return l - div_q(l, sm, ss1, ss2) * sets;
    }
};

// Census: the segment's line ids into this warp's bitmap, then into the item's.
__device__ __forceinline__ void census_segment(const SimItem &it, const StreamJob &J, uint32_t seg,
                                               int lane, uint32_t *sbm, uint32_t *gbm) {
    const Decoder D(it);
    const CensusKey C(it);
    constexpr uint32_t kWords = kCensusMaxLines / 32;
    for (uint32_t k = (uint32_t)lane; k < kWords; k += 32) sbm[k] = 0;
    __syncwarp();
    const uint32_t t0 = seg * kSegAccesses;
    const uint32_t t1 = min(it.len, t0 + kSegAccesses);
    for (uint32_t c = t0; c < t1; c += 32) {
        const uint32_t t = c + (uint32_t)lane;
        if (t < t1) {
            const uint32_t j = D.index(t);
            if (j < D.N) {
                const uint32_t id = C.id(j);
                if (id < kCensusMaxLines) atomicOr(sbm + (id >> 5), 1u << (id & 31));
            }
        }
    }
    __syncwarp();
    for (uint32_t k = (uint32_t)lane; k < kWords; k += 32)
        if (sbm[k]) atomicOr(gbm + k, sbm[k]);
}

__global__ void __launch_bounds__(kStreamWarps * 32)
    head_count_kernel(const SimItem *__restrict__ items, const StreamJob *__restrict__ jobs,
                      const uint32_t *__restrict__ seg_job, uint32_t n_seg, uint32_t *cnt,
                      uint32_t *status) {
    __shared__ uint32_t counts[kStreamWarps][32];
    __shared__ uint32_t census[kStreamWarps][kCensusMaxLines / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t g = blockIdx.x * kStreamWarps + (uint32_t)w;
    if (g >= n_seg) return;
    const StreamJob J = jobs[seg_job[g]];
    const SimItem it = items[J.unit];
    if (J.kind == kJobCensus) {
        census_segment(it, J, g - J.seg_first, lane, census[w], cnt + J.cnt_off);
        return;
    }
    uint32_t *const cs = counts[w];
    cs[lane] = 0;
    __syncwarp();
    walk_segment(it, g - J.seg_first, lane, status, [&](uint32_t, bool take, uint32_t k, uint32_t) {
        const uint32_t m = __match_any_sync(kFull, take ? k : 0x80000000u | (uint32_t)lane);
        if (take && (m & lanemask_lt_()) == 0) cs[k] += (uint32_t)__popc(m);
        __syncwarp();
    });
    if ((uint32_t)lane < J.K) cnt[J.cnt_off + (uint64_t)(g - J.seg_first) * J.K + lane] = cs[lane];
}

// One warp per job: lane k turns part k's counts into offsets within the
// part's stream and takes its total; the parts' streams follow one another.
__global__ void __launch_bounds__(256)
    head_offsets_kernel(const SimItem *__restrict__ items, const StreamJob *__restrict__ jobs,
                        uint32_t n_jobs, uint32_t *cnt, PartInfo *parts, uint32_t *targets) {
    __shared__ uint32_t per_set[8][kCensusMaxSets];
    const int lane = threadIdx.x & 31;
    const uint32_t j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= n_jobs) return;
    const StreamJob J = jobs[j];
    if (J.kind == kJobCensus) {
        // each set's distinct lines, at most a of them
        const SimItem it = items[J.unit];
        const CensusKey C(it);
        uint32_t *const ps = per_set[threadIdx.x >> 5];
        for (uint32_t s = (uint32_t)lane; s < C.sets; s += 32) ps[s] = 0;
        __syncwarp();
        const uint32_t *bm = cnt + J.cnt_off;
        for (uint32_t k = (uint32_t)lane; k < kCensusMaxLines / 32; k += 32) {
            for (uint32_t bits = bm[k]; bits; bits &= bits - 1)
                atomicAdd(ps + C.set(k * 32u + (uint32_t)(__ffs(bits) - 1)), 1u);
        }
        __syncwarp();
        for (uint32_t s = (uint32_t)lane; s < C.sets; s += 32)
            targets[J.ent_base + s] = min(ps[s], it.ways);
        if (lane == 0) {
            PartInfo p;
            p.start = J.ent_base;
            p.len = C.sets;
            p.pad = 0;
            parts[J.slot_first] = p;
        }
        return;
    }
    const bool on = (uint32_t)lane < J.K;
    uint32_t run = 0;
    for (uint32_t s = 0; s < J.nseg; ++s) {
        if (on) {
            uint32_t *c = cnt + J.cnt_off + (uint64_t)s * J.K + lane;
            const uint32_t v = *c;
            *c = run;
            run += v;
        }
    }
    uint32_t inc = on ? run : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += v;
    }
    if (on) {
        PartInfo p;
        p.start = J.ent_base + (inc - run);
        p.len = run;
        p.pad = 0;
        parts[J.slot_first + lane] = p;
    }
}

__global__ void __launch_bounds__(kStreamWarps * 32)
    head_write_kernel(const SimItem *__restrict__ items, const StreamJob *__restrict__ jobs,
                      const uint32_t *__restrict__ seg_job, uint32_t n_seg,
                      const uint32_t *__restrict__ cnt, const PartInfo *__restrict__ parts,
                      uint2 *ents, uint32_t *status) {
    __shared__ uint64_t cursor[kStreamWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t g = blockIdx.x * kStreamWarps + (uint32_t)w;
    if (g >= n_seg) return;
    const StreamJob J = jobs[seg_job[g]];
    if (J.kind == kJobCensus) return;
    const SimItem it = items[J.unit];
    uint64_t *const cur = cursor[w];
    if ((uint32_t)lane < J.K)
        cur[lane] = parts[J.slot_first + lane].start +
                    cnt[J.cnt_off + (uint64_t)(g - J.seg_first) * J.K + lane];
    __syncwarp();
    walk_segment(it, g - J.seg_first, lane, status, [&](uint32_t t, bool take, uint32_t k, uint32_t lp) {
        const uint32_t m = __match_any_sync(kFull, take ? k : 0x80000000u | (uint32_t)lane);
        const uint32_t lt = lanemask_lt_();
        if (take) ents[cur[k] + (uint32_t)__popc(m & lt)] = make_uint2(lp, t);
        __syncwarp();
        if (take && (m & lt) == 0) cur[k] += (uint32_t)__popc(m);
        __syncwarp();
    });
}

}  // namespace

cudaError_t launch_streams(const SimItem *items, const StreamJob *jobs, uint32_t n_jobs,
                           const uint32_t *seg_job, uint32_t n_seg, uint32_t *cnt,
                           PartInfo *parts, uint2 *ents, uint32_t *targets, uint32_t *status,
                           cudaStream_t st) {
    if (!n_jobs) return cudaSuccess;
    // (items with empty traces still get their parts' {start, 0})
    const unsigned blocks = (n_seg + kStreamWarps - 1) / kStreamWarps;
    if (n_seg)
        head_count_kernel<<<blocks, kStreamWarps * 32, 0, st>>>(items, jobs, seg_job, n_seg, cnt,
                                                                status);
    head_offsets_kernel<<<(n_jobs + 7) / 8, 256, 0, st>>>(items, jobs, n_jobs, cnt, parts, targets);
    if (n_seg)
        head_write_kernel<<<blocks, kStreamWarps * 32, 0, st>>>(items, jobs, seg_job, n_seg, cnt,
                                                                parts, ents, status);
    return cudaGetLastError();
}

}  // namespace pchase
