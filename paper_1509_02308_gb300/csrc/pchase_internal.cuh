// Internal declarations shared by the library's translation units.
// Device code targets sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pchase.h"

namespace pchase {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kInvalidLine = 0xFFFFFFFFu;

// ---------------------------------------------------------------- division
// Unsigned division of 32-bit n by an invariant d >= 1 with one multiply-high,
// after Granlund & Montgomery, "Division by invariant integers using
// multiplication" (PLDI 1994), Fig. 4.1: with l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n),
// q = (t + ((n - t) >> min(l,1))) >> max(l-1, 0).  Exact for every 32-bit n.
struct DivMagic {
    uint32_t d;
    uint32_t m;
    uint32_t s1;
    uint32_t s2;
};

__host__ inline DivMagic make_div_magic(uint32_t d) {
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    DivMagic r;
    r.d = d;
    r.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
    r.s1 = l < 1 ? l : 1;
    r.s2 = l > 1 ? l - 1 : 0;
    return r;
}

__device__ __forceinline__ uint32_t div_q(uint32_t n, uint32_t m, uint32_t s1, uint32_t s2) {
    uint32_t t = __umulhi(m, n);
    return (t + ((n - t) >> s1)) >> s2;
}

// ------------------------------------------------------------ SplitMix64
// First output of the SplitMix64 generator (Steele, Lea & Flood, OOPSLA 2014)
// whose state is x: advance by the golden-ratio increment, then two
// xor-shift-multiply rounds and a final xor-shift.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Victim way of the k-th eviction of set `set` under the RANDOM policy, or
// under WEIGHTED (the Fermi L1 data cache, Sec. 4.5): evictions 0, 2, 4, ...
// take way 2, the others one of the remaining ways, seeded-uniform.
__device__ __forceinline__ uint32_t random_way(uint64_t seed, uint32_t set, uint32_t k,
                                               uint32_t ways, bool weighted) {
    if (weighted && (k & 1u) == 0) return 2;
    uint64_t h = splitmix64(seed ^ ((uint64_t)set << 40) ^ (uint64_t)k);
    const uint32_t n = weighted ? ways - 1 : ways;
    const uint32_t r = (uint32_t)(((h >> 32) * (uint64_t)n) >> 32);
    return weighted && r >= 2 ? r + 1 : r;
}

// Line id under a mapping that takes the set from m line bits higher
// (set = (line >> m) mod T): line = ((hi * T + set) << m) | lo becomes
// ((hi << m) | lo) * T + set, a one-to-one renumbering under which
// set = id mod T, so every set mode, table and split sees the usual form.
__device__ __forceinline__ uint32_t remap_line(uint32_t ln, uint32_t m, uint32_t T, uint32_t tm,
                                               uint32_t ts1, uint32_t ts2) {
    const uint32_t u = ln >> m;
    const uint32_t hi = div_q(u, tm, ts1, ts2);
    return (((hi << m) | (ln & ((1u << m) - 1u))) * T) + (u - hi * T);
}

// ------------------------------------------------------------ plan items
enum SetMode : uint8_t { kModeScan = 0, kModeTable = 1, kModeBatch = 2 };

// One simulation unit as the kernels read it (64-bit aligned, 112 bytes).
// A caller's item is one unit, or K (a power of two or three times one) when
// its sets are split: unit r owns the sets s with (s >> psh) mod K == r,
// renumbered locally as (((s >> psh) div K) << psh) | (s & (2^psh - 1)), and
// sees each line as the local line  local set + T' * (line div T), T' = T / K.
// A whole LRU item that steps directly over its accesses may instead be cut in
// time: a unit with kcnt = 1 and ks1 = 1 covers steps [kres, kmagic) (32
// accesses a step, bounds multiples of 32 steps so that every bitmap word has
// one writer) and first rebuilds the sets' recency order from the accesses
// before its first one.
struct SimItem {
    const uint32_t *idx;  // NULL: analytic uniform chain
    uint32_t len;
    uint32_t warmup;
    uint32_t n_elems;
    uint32_t stride;      // analytic chains, already reduced mod n_elems
    uint32_t ways;
    uint32_t sets;        // local sets T' = T / K
    uint32_t magic_m;     // local set = local line mod T', by DivMagic of T'
    uint8_t s1, s2, policy, mode;
    uint32_t lsh;         // line = index >> (lsh & 255) (b = 4 << that); bits 8-15: mapping m;
                          // bit 16: unequal sets (gsets/gmagic: M = T*a + extra, kmagic: a,
                          // ways: a + extra, the ways of set 0); bit 17: way scans with the
                          // set state in global memory at 16 * kres bytes (whole units);
                          // bit 18: compact lines (whole units of analytic chains whose
                          // visited lines are the multiples of gsets: the unit keys its
                          // state by line / gsets, gmagic/gs1/gs2 its DivMagic, and takes
                          // the set from the line itself)
    uint32_t table_n;     // line-table entries (local lines)
    uint64_t seed;
    uint64_t word_off;    // plan-owned bitmap layout
    uint32_t out_item;    // caller's item number
    uint32_t cand;        // matcher: candidate
    uint32_t obs;         // matcher: observed trace
    uint32_t arena_bytes; // shared memory this unit needs (queue + set state)
    uint32_t ring;        // batch-mode LRU: recency ring entries per set (power of two)
    uint32_t gsets;       // the geometry's T
    uint32_t gmagic;      // DivMagic of T
    uint8_t gs1, gs2, psh, ks1;
    uint32_t kres;        // this unit's residue (0 when not split)
    uint8_t lead;         // 1 on exactly one unit of each caller item
    uint8_t direct;       // 1: step over consecutive accesses (dense, unsplit), no queue;
                          // 2: a part of a split that reads its head stream (when the
                          // run has streams; else it gathers like 0)
    uint8_t kcnt;         // K: parts of the split (1: whole)
    uint8_t ks2;
    float cost;           // planner's estimate of the unit's warp time (ns)
    uint32_t kmagic;      // DivMagic of K (with ks1, ks2)
};

static_assert(sizeof(SimItem) == 112, "SimItem layout");

// Global set index of local set `local` of a unit (see SimItem).
__host__ __device__ __forceinline__ uint32_t global_set(uint32_t local, uint32_t psh, uint32_t K,
                                                        uint32_t kres) {
    return (((local >> psh) * K + kres) << psh) | (local & ((1u << psh) - 1u));
}

// Staging at the start of a queued unit's arena: the compaction queue (run
// heads of the unit's sets wait here, in trace order, until a full step of 32
// is ready), then the ring the trace streams into ahead of use.
constexpr uint32_t kQueueEntries = 64;   // uint2 {local line, position | observed bit << 31}
constexpr uint32_t kQueueBytes = kQueueEntries * 8;
constexpr uint32_t kRing = 16;           // chunks of 32 accesses (+ observed words)
constexpr uint32_t kStageBytes = kQueueBytes + kRing * 32 * 4 + kRing * 4;

// One launch serves every unit.  Each CTA holds the same mix of per-warp
// shared-memory arenas ("slots"); a free warp takes, among the classes its
// slot can hold (pad .. warp_class[w]), the next unit of the class whose next
// unit has the highest estimated cost (each class queue is costliest first).
//
// Units are also grouped by kind (set mode x policy, WEIGHTED with RANDOM,
// whose code it runs), one queue per group and class.  With affinity on, CTA
// b starts on the group whose site range [home_end[g - 1], home_end[g]) holds
// b mod home_mod (the SM it sits on, for CTAs placed round-robin) and keeps
// to it while its classes have units, so the warps sharing an SM's
// instruction cache mostly run one kind's code; a warp whose group is out of
// units takes the costliest next unit of any group and keeps to that group.
// Without affinity every pop looks at all groups.
constexpr int kMaxWarpsPerCta = 16;
constexpr int kMaxClasses = 25;  // size classes + the global-state pool's
constexpr int kUnitGroups = 9;
constexpr uint32_t kQueueStride = 32;  // queue counter of (group g, class c): g * 32 + c
constexpr size_t kQueueHeader = 2048;  // workspace head: the queue counters, then the status word
constexpr size_t kStatusOffset = 1536;
__host__ __device__ __forceinline__ uint32_t unit_group(uint32_t mode, uint32_t policy) {
    return mode * 3u + (policy < 2u ? policy : 2u);
}
struct SlotLayout {
    uint32_t nwarps;                          // warps per CTA
    uint32_t nclasses;
    uint32_t smem_bytes;                      // dynamic shared memory per CTA
    uint32_t pad;                             // lowest class a warp may take
    uint32_t stagger_ns;                      // first pop of warp w waits w * this
    uint32_t pool16;                          // global-state pool: warp g = CTA * nwarps + w
                                              // keeps its units' state at g * 16 * pool16
                                              // bytes of the state area (0: no pool)
    uint32_t spec;                            // 1: per-mode unit loops (units alone on an SM)
    uint32_t affinity;                        // 1: CTAs start on a home group
    uint32_t home_mod;                        // CTA b sits on site b mod home_mod
    uint32_t home_end[kUnitGroups];               // sites [home_end[g-1], home_end[g]) start on g
    uint32_t warp_class[kMaxWarpsPerCta];     // class served first by warp w
    uint32_t warp_off[kMaxWarpsPerCta];       // byte offset of warp w's arena
    uint32_t cls_first[kUnitGroups][kMaxClasses]; // first item of (group, class) (sorted table)
    uint32_t cls_count[kUnitGroups][kMaxClasses];
};

// Simulation output sinks.
struct SimOut {
    uint32_t *bitmaps;
    const uint64_t *word_offsets;  // NULL: item.word_off
    uint64_t *miss_counts;
    uint32_t *status;
    // matcher
    const uint32_t *observed;
    const uint64_t *obs_word_offsets;
    uint64_t stop_above;
    uint64_t *dist;
    // optional per-item timeline (4 uint64 per item)
    uint64_t *timeline;
    // matcher over several observations: every unit runs once per
    // observation r < n_rep (0 = 1), with dist + r * rep_dist_stride and
    // observed + r * rep_obs_stride
    uint32_t n_rep;
    uint64_t rep_dist_stride;
    uint64_t rep_obs_stride;
    // a lower level of a hierarchy: item i's unit sees only the accesses set
    // in filter + filter_word_offsets[i] (queued units only; not with the matcher)
    const uint32_t *filter;
    const uint64_t *filter_word_offsets;
    // set state of the units that keep it in global memory (SimItem lsh bit
    // 17), each at 16 * kres bytes from here
    uint8_t *gstate;
    // head streams of the parts of items split by sets (SimItem direct = 2):
    // part k of caller item i reads parts[item_slot[i] + k].len entries
    // {local line, position} from ents + parts[...].start, in trace order.
    // NULL: such units gather their heads from the trace themselves.
    const uint32_t *item_slot;
    const struct PartInfo *parts;
    const uint2 *ents;
    // LRU items cut in time: parts[item_slot[i]].start indexes targets, one
    // per set: min(a, the set's distinct lines over the whole trace), the
    // lines a time part's read-back needs before the set is complete
    const uint32_t *targets;
};

// Head streams (streams.cu).  Every item split by sets into K parts is one
// job: its trace is cut into segments of kSegAccesses accesses, one warp per
// segment counts each part's run heads (an access whose line differs from the
// previous access's line, falling in the part's sets), a warp per job turns
// the counts into offsets, and the segments' warps write the heads out, so
// each part's stream holds exactly the heads the part would gather itself.
// A census job (an LRU item cut in time, at most kCensusMaxLines line ids and
// kCensusMaxSets sets) marks the lines its trace uses in a bitmap instead, and
// its warp counts each set's distinct lines into the targets.
constexpr uint32_t kSegAccesses = 8192;
constexpr uint32_t kCensusMaxLines = 4096;
constexpr uint32_t kCensusMaxSets = 256;
enum : uint32_t { kJobHeads = 0, kJobCensus = 1 };
struct PartInfo {
    uint64_t start;  // first entry of the part's stream
    uint32_t len;    // entries
    uint32_t pad;
};
struct StreamJob {
    uint64_t ent_base;    // first entry of the item's K streams (census: first target)
    uint64_t cnt_off;     // counts: cnt_off + segment * K + part (census: the line bitmap)
    uint32_t unit;        // one of the item's units (any part: they share trace and split)
    uint32_t K;
    uint32_t nseg;
    uint32_t seg_first;   // its first segment in the plan's segment list
    uint32_t slot_first;  // parts[slot_first + k]
    uint32_t kind;        // kJobHeads or kJobCensus
};

// Records the text pchase_last_error_string() returns on this thread and
// passes `code` through (capi.cu).
int set_last_error(int code, const char *msg);

// Kernel launchers (sim.cu)
cudaError_t launch_sim(const SimItem *items, const SlotLayout &layout, uint32_t *queues, int grid,
                       const SimOut &out, cudaStream_t st);
// Zeroes the outputs the units accumulate into (bitmap words, miss counts,
// timeline) for every caller item of the plan.
cudaError_t launch_sim_zero(const SimItem *items, uint64_t n_units, int sms, const SimOut &out,
                            cudaStream_t st);
int sim_max_ctas_per_sm(const SlotLayout &layout);
// The head streams of a plan's split items (three launches on `st`).
cudaError_t launch_streams(const SimItem *items, const StreamJob *jobs, uint32_t n_jobs,
                           const uint32_t *seg_job, uint32_t n_seg, uint32_t *cnt,
                           PartInfo *parts, uint2 *ents, uint32_t *targets, uint32_t *status,
                           cudaStream_t st);

}  // namespace pchase
