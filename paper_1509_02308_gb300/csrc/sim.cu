// Batched set-associative cache simulator (S2 decode, S3 set simulation) and
// its Hamming-compare form for the exhaustive matcher (S5).
//
// Model (Assumptions 1-3 and Fig. 2, Sec. 4.1): line = (4 * index) / b,
// set = line mod T; an access hits when its line is held by its set; a miss
// fills the lowest invalid way, else evicts by LRU (oldest use), FIFO (oldest
// fill) or RANDOM (SplitMix64-keyed way).
//
// Mapping onto the GPU:
//   * one warp per unit, pulled from a per-class atomic queue by persistent
//     CTAs; a unit is an item (geometry x trace) or, for long items, one part
//     of a split of its sets (sets never interact, so each part replays the
//     whole trace but keeps only its own sets' accesses); the unit's cache
//     state lives in the warp's slice of shared memory;
//   * the warp reads the trace 32 accesses at a time (coalesced loads issued
//     128 accesses ahead; analytic uniform chains are generated in registers)
//     and drops every access that repeats the previous access's line: it hits
//     under every policy and changes no replacement order.  The remaining run
//     heads of the unit's sets are compacted, in trace order, into a queue in
//     shared memory, and the cache steps over full groups of 32 of them;
//   * heads in different sets are independent; heads in one set must act in
//     trace order.  Three set modes:
//       scan  (few ways, many sets): a head of rank r among the step's heads
//             of its set acts in round r (__match_any_sync groups them); the
//             lane scans the set's {line, stamp} ways;
//       table (many ways, many sets): the same rounds, with a per-item line
//             table (line -> way + 1), LRU order as a doubly linked list and
//             FIFO order as a ring pointer;
//       batch (few sets): all heads of a set are resolved together, one lane
//             each, without rounds (see the batch section below);
//   * miss bits are OR-ed into bitmap words zeroed beforehand (one reduction
//     per word touched by a step), counts are added atomically, so the units
//     of a split item need no coordination.
#include <algorithm>

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
constexpr int32_t kBig = 0x3FFFFFFF;
constexpr uint32_t kStale = 0xFFFFFFFFu;

// ----------------------------------------------------------- scan sets
// Arena: uint2 slot[T*a] = {line, stamp}; RANDOM adds uint32 evictions[T].
// Stamps: an invalid way w holds stamp w (< a), a filled way t + a, where t
// is the access time of its last use (LRU) or of its fill (FIFO, RANDOM), so
// the smallest stamp is the lowest invalid way if any, else the victim.
template <int POLICY>
struct ScanSets {
    static constexpr bool kStaticHits = false;  // residency needs a scan
    uint2 *slot;
    uint32_t *evict;
    uint32_t ways;
    uint32_t ways_rest;        // unequal sets: ways of sets 1.. (set 0 has `ways`)
    uint64_t seed;
    bool wtd;                  // WEIGHTED victims (RANDOM code path)
    uint32_t psh, kcnt, kres;  // local -> global set (RANDOM's key)

    __device__ __forceinline__ void bind(uint8_t *arena, const SimItem &it) {
        ways = it.ways;
        ways_rest = (it.lsh >> 16) & 1u ? it.kmagic : it.ways;
        seed = it.seed;
        wtd = it.policy == PCHASE_WEIGHTED;
        psh = it.psh;
        kcnt = it.kcnt;
        kres = (it.lsh >> 17) & 1u ? 0u : it.kres;  // global state: kres is its offset
        slot = reinterpret_cast<uint2 *>(arena);
        evict = reinterpret_cast<uint32_t *>(arena + 8ull * it.sets * ways);
    }

    __device__ __forceinline__ void clear(const SimItem &it, int lane) {
        const uint32_t n = it.sets * ways;
        for (uint32_t i = lane; i < n; i += 32) slot[i] = make_uint2(kInvalidLine, i % ways);
        if (POLICY == PCHASE_RANDOM)
            for (uint32_t i = lane; i < it.sets; i += 32) evict[i] = 0;
    }

    __device__ __forceinline__ bool access(uint32_t set, uint32_t line, uint32_t t) {
        const uint32_t a = ways;
        const uint32_t na = set ? ways_rest : a;  // ways this set has
        uint2 *s = slot + set * a;
        int hit = -1;
        uint32_t best = 0xFFFFFFFFu;
        uint32_t bw = 0;
        for (uint32_t w = 0; w < na; ++w) {
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
            v = random_way(seed, global_set(set, psh, kcnt, kres), k, a, wtd);
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
    // FIFO and RANDOM hits change nothing, and residency is one table read
    static constexpr bool kStaticHits = POLICY != PCHASE_LRU;
    __device__ __forceinline__ bool held(uint32_t line) const { return tab[line] != 0; }
    uint2 *meta;
    uint32_t *sline;
    uint16_t *prv, *nxt, *tab;
    uint32_t ways;
    uint64_t seed;
    bool wtd;
    uint32_t psh, kcnt, kres;

    __device__ __forceinline__ void bind(uint8_t *arena, const SimItem &it) {
        ways = it.ways;
        seed = it.seed;
        wtd = it.policy == PCHASE_WEIGHTED;
        psh = it.psh;
        kcnt = it.kcnt;
        kres = it.kres;
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
    }

    __device__ __forceinline__ void clear(const SimItem &it, int lane) {
        const uint32_t n = it.sets * ways;
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
                v = random_way(seed, global_set(set, psh, kcnt, kres), m.y, a, wtd);
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

// Rounds driver for scan and table sets: a head of rank r inside its set's
// group of heads acts in round r.
template <typename Sets>
struct RoundResolver {
    Sets S;
    __device__ __forceinline__ void bind(uint8_t *arena, const SimItem &it) { S.bind(arena, it); }
    __device__ __forceinline__ bool resolve(uint32_t line, uint32_t set, bool head, uint32_t t,
                                            int lane, uint32_t lt, uint32_t) {
        // only a miss evicts: when every head's line is held at the start of
        // the step, all of them hit, and under FIFO / RANDOM nothing changes
        if constexpr (Sets::kStaticHits) {
            if (__all_sync(kFull, !head || S.held(line))) return false;
        }
        const uint32_t key = head ? set : (0x80000000u | (uint32_t)lane);
        const uint32_t peers = __match_any_sync(kFull, key);
        const uint32_t rank = __popc(peers & lt);
        bool miss = false, pending = head;
        for (uint32_t r = 0; __any_sync(kFull, pending); ++r) {
            if (pending && rank == r) {
                miss = S.access(set, line, t);
                pending = false;
            }
            __syncwarp();
        }
        return miss;
    }
};

// ------------------------------------------------------------ batch sets
// For items with few sets each step has many heads per set.  The step's heads
// are first regrouped so every set's heads sit on consecutive lanes in trace
// order; then each set's group is resolved at once.
//
// FIFO and RANDOM: the k-th miss of a group (k = 0, 1, ...) goes to a way
// fixed in advance (FIFO: (p + L + k) mod a; RANDOM: the lowest invalid way
// while the set fills, then the SplitMix64 way of its eviction number).  A
// line held in way w is evicted by the first miss k whose way is w (its
// eviction index e); an access misses exactly when the number of misses
// before it in its group exceeds the eviction index of its line, and a line
// inserted by miss k next leaves at the next k' > k with the same way.  The
// outcome vector is the fixed point of that rule; any fixed point equals the
// sequential answer (a lane depends only on earlier lanes), and 32 rounds of
// the rule reach it from any start, usually 1-2 from the start used here.
//
// LRU: by the stack property an access hits exactly when fewer than a
// distinct lines were used since the previous use of its line.  Recency is a
// per-set ring of lines in use order (an entry goes stale when its line is
// used again); the 32 oldest live entries (the tail window) give the exact
// depth of every line that could fall out within one step, every other
// resident line is a sure hit.  After the decisions the step's lines are
// appended in last-use order and the oldest non-step lines are evicted so
// that a lines stay live; the ring is compacted when it nears full.
struct Grouped {
    uint32_t x, set;   // line and set of the head now on this lane
    bool act;          // lane holds a head
    bool same;         // no head moved (every lane holds its own)
    uint32_t gmask;    // lanes of this head's set group
    uint32_t gb;       // first lane of the group
    uint32_t dest;     // where this lane's own head went
};

__device__ __forceinline__ Grouped group_heads(uint32_t line, uint32_t set, bool head, int lane,
                                               uint32_t lt, uint32_t *perm) {
    // common case (compacted steps, single-set units): the heads fill lanes
    // 0..n-1 and share one set, so they already form one group in order
    const uint32_t hb = __ballot_sync(kFull, head);
    const uint32_t s0 = __shfl_sync(kFull, set, 0);
    if ((hb & (hb + 1u)) == 0 && __all_sync(kFull, !head || set == s0)) {
        Grouped g;
        g.x = line;
        g.set = set;
        g.act = head;
        g.gmask = hb;
        g.gb = 0;
        g.dest = (uint32_t)lane;
        g.same = true;
        return g;
    }
    const uint32_t key = head ? set : (0x80000000u | (uint32_t)lane);
    const uint32_t gm = __match_any_sync(kFull, key);
    const bool leader = head && (gm & lt) == 0;
    const uint32_t size = leader ? (uint32_t)__popc(gm) : 0u;
    uint32_t inc = size;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += v;
    }
    const uint32_t base = __shfl_sync(kFull, inc - size, __ffs(gm) - 1);
    const uint32_t dest = base + __popc(gm & lt);
    const uint32_t nh = __popc(hb);
    if (head) perm[dest] = (uint32_t)lane;
    __syncwarp();
    const bool act = (uint32_t)lane < nh;
    const uint32_t src = act ? perm[lane] : (uint32_t)lane;
    __syncwarp();
    Grouped g;
    g.x = __shfl_sync(kFull, line, src);
    g.set = __shfl_sync(kFull, set, src);
    g.act = act;
    g.gmask = __match_any_sync(kFull, act ? g.set : (0x80000000u | (uint32_t)lane));
    g.gb = __ffs(g.gmask) - 1;
    g.dest = dest;
    g.same = false;
    return g;
}

// x mod a for x < 4a (else the division)
__device__ __forceinline__ uint32_t mod_ways(uint32_t x, uint32_t a) {
    if (x < 4u * a) {
        if (x >= 2u * a) x -= 2u * a;
        if (x >= a) x -= a;
        return x;
    }
    return x % a;
}

// mask of lanes whose key is below this lane's threshold (keys, thresholds < 64)
__device__ __forceinline__ uint32_t lanes_below(uint32_t key, uint32_t thr) {
    uint32_t less = 0, eq = kFull;
#pragma unroll
    for (int b = 5; b >= 0; --b) {
        const uint32_t plane = __ballot_sync(kFull, (key >> b) & 1u);
        if ((thr >> b) & 1u) {
            less |= eq & ~plane;
            eq &= plane;
        } else {
            eq &= ~plane;
        }
    }
    return less;
}

// FIFO / RANDOM.  Arena: uint4 meta[T] ({p, L} or {filled, evictions});
// uint32 sline[T*a]; (RANDOM) uint2 scr[T*a]; uint16 tab[table_n] (way + 1).
// A FIFO / RANDOM step of one set goes miss by miss (BatchFR::seq_step) when
// at most this many of its heads start out not held.
constexpr int kSeqMaxFirst = 4;

template <int POLICY>
struct BatchFR {
    uint4 *meta;
    uint32_t *sline;
    uint2 *scr;
    uint16_t *tab;
    uint32_t *perm;
    uint32_t ways;
    uint64_t seed;
    bool wtd;
    uint32_t psh, kcnt, kres;
    // steps left before the pure-set test is tried again: a unit whose steps
    // are not pure (hits and misses in one set) skips it for a while (bound
    // once per unit, the count lives across its steps)
    uint32_t pure_skip = 0;

    __device__ __forceinline__ void bind(uint8_t *arena, const SimItem &it) {
        ways = it.ways;
        seed = it.seed;
        wtd = it.policy == PCHASE_WEIGHTED;
        psh = it.psh;
        kcnt = it.kcnt;
        kres = it.kres;
        const uint32_t n = it.sets * ways;
        size_t off = 0;
        perm = reinterpret_cast<uint32_t *>(arena);
        off += 256;
        meta = reinterpret_cast<uint4 *>(arena + off);
        off += 16ull * it.sets;
        sline = reinterpret_cast<uint32_t *>(arena + off);
        off += (4ull * n + 15) & ~15ull;
        if (POLICY == PCHASE_RANDOM) {
            scr = reinterpret_cast<uint2 *>(arena + off);
            off += 8ull * n;
        }
        tab = reinterpret_cast<uint16_t *>(arena + off);
    }

    __device__ __forceinline__ void clear(const SimItem &it, int lane) {
        const uint32_t n = it.sets * ways;
        for (uint32_t i = lane; i < it.sets; i += 32) meta[i] = make_uint4(0, 0, 0, 0);
        for (uint32_t i = lane; i < n; i += 32) sline[i] = kInvalidLine;
        if (POLICY == PCHASE_RANDOM)
            for (uint32_t i = lane; i < n; i += 32) scr[i] = make_uint2(0, 0);
        uint32_t *t32 = reinterpret_cast<uint32_t *>(tab);
        for (uint32_t i = lane; i < (it.table_n + 1) / 2; i += 32) t32[i] = 0;
    }

    // The way the group's r-th miss of this step fills, given the set's
    // counters m at the step's start, and whether that miss evicts.
    __device__ __forceinline__ uint32_t rank_way(uint4 m, uint32_t set, uint32_t r,
                                                 bool &evicts) const {
        const uint32_t a = ways;
        if (POLICY == PCHASE_FIFO) {
            evicts = m.y + r >= a;
            return mod_ways(m.x + m.y + r, a);
        }
        const uint32_t k = m.x + r;
        evicts = k >= a;
        return evicts ? random_way(seed, global_set(set, psh, kcnt, kres), m.y + (k - a), a, wtd) : k;
    }

    // The set's counters after M more misses (FIFO: {ring pointer, lines
    // held}; RANDOM: {lines held, evictions}).
    __device__ __forceinline__ uint4 after_misses(uint4 m, uint32_t M) const {
        const uint32_t a = ways;
        uint4 n = m;
        if (POLICY == PCHASE_FIFO) {
            const uint32_t tot = m.y + M;
            n.y = tot < a ? tot : a;
            n.x = mod_ways(m.x + (tot > a ? tot - a : 0u), a);
        } else {
            const uint32_t tot = m.x + M;
            n.x = tot < a ? tot : a;
            n.y = m.y + (tot > a ? tot - a : 0u);
        }
        return n;
    }

    // One set's heads (in lane order), resolved miss by miss, for a <= 32
    // ways.  A hit changes nothing, so between misses every head whose line
    // is held hits; the first head whose line is not held misses, fills the
    // way of the step's next miss (rank_way), and from there on the line it
    // evicted is not held and its own line is.  The set's ways sit one per
    // lane in a register for the step (lane w: way w), so a miss costs a few
    // votes and shuffles; the line table is brought up to date at the end
    // (lines that left first, then the ways' final lines).  res: the lane's
    // line is held as of the misses handled so far.
    __device__ __forceinline__ bool seq_step(uint32_t line, uint32_t set, bool head, bool res,
                                             uint32_t cand, int lane) {
        const uint32_t a = ways;
        const uint4 m = meta[set];
        bool ev;
        const uint32_t vw = rank_way(m, set, (uint32_t)lane, ev);  // the way of miss `lane`
        uint32_t *const sl = sline + (size_t)set * a;
        const uint32_t orig = (uint32_t)lane < a ? sl[lane] : kInvalidLine;
        uint32_t cur = orig;
        uint32_t bits = 0, nm = 0;
        while (cand) {
            const int j = __ffs(cand) - 1;
            const uint32_t v = __shfl_sync(kFull, vw, nm);
            const uint32_t xj = __shfl_sync(kFull, line, j);
            const uint32_t old = __shfl_sync(kFull, cur, v);
            if ((uint32_t)lane == v) cur = xj;
            if (lane > j) res = line == xj || (res && line != old);
            bits |= 1u << j;
            ++nm;
            cand = __ballot_sync(kFull, head && !res && lane > j);
        }
        if (cur != orig) {
            if (orig != kInvalidLine) tab[orig] = 0;
            sl[lane] = cur;
        }
        __syncwarp();
        if (cur != orig) tab[cur] = (uint16_t)(lane + 1);
        if (lane == 0) meta[set] = after_misses(m, nm);
        __syncwarp();
        return head && ((bits >> lane) & 1u);
    }

    // A step whose heads are all new lines, none held at its start: every
    // head misses, the r-th miss of a set's group takes that group's r-th
    // way, and the last writer of each way is what stays.
    __device__ __forceinline__ bool fresh_step(uint32_t line, uint32_t set, bool head, int lane,
                                               uint32_t lt, uint32_t sm) {
        const uint32_t a = ways;
        const uint32_t r = __popc(sm & lt);
        const uint32_t M = __popc(sm);
        const uint4 m = head ? meta[set] : make_uint4(0, 0, 0, 0);
        uint32_t insw;
        bool evicts;
        if (POLICY == PCHASE_FIFO) {
            evicts = m.y + r >= a;
            insw = mod_ways(m.x + m.y + r, a);
        } else {
            const uint32_t k = m.x + r;
            evicts = k >= a;
            insw = evicts ? random_way(seed, global_set(set, psh, kcnt, kres), m.y + (k - a), a, wtd)
                          : k;
        }
        // FIFO groups of at most a misses write distinct ways (p + L + r mod a)
        const uint32_t sw =
            (POLICY == PCHASE_FIFO && __all_sync(kFull, !head || M <= a))
                ? (1u << lane)
                : __match_any_sync(kFull, head ? set * a + insw : (0x80000000u | (uint32_t)lane));
        // the first writer of a way that was in use evicts the line it held
        // (a line of the step is written again only after its earlier way
        // was taken over, so only last writers stay)
        if (head && evicts && (sw & lt) == 0) tab[sline[set * a + insw]] = 0;
        __syncwarp();
        if (head && (sw & ~(lt | (1u << lane))) == 0) {
            sline[set * a + insw] = line;
            tab[line] = (uint16_t)(insw + 1);
        }
        if (head && r == 0) {
            uint4 n = m;
            if (POLICY == PCHASE_FIFO) {
                const uint32_t tot = m.y + M;
                n.y = tot < a ? tot : a;
                n.x = mod_ways(m.x + (tot > a ? tot - a : 0u), a);
            } else {
                const uint32_t tot = m.x + M;
                n.x = tot < a ? tot : a;
                n.y = m.y + (tot > a ? tot - a : 0u);
            }
            meta[set] = n;
        }
        __syncwarp();
        return head;
    }

    __device__ __forceinline__ bool resolve(uint32_t line, uint32_t set, bool head, uint32_t,
                                            int lane, uint32_t lt, uint32_t stamp) {
        const uint32_t hb = __ballot_sync(kFull, head);
        if (hb == 0) return false;
        // Only a miss evicts: when every head's line is held at the start of
        // the step, all of them hit and nothing changes.
        const uint32_t w0 = head ? tab[line] : 1u;
        if (__all_sync(kFull, w0 != 0u)) return false;
        const uint32_t lm0 = __match_any_sync(kFull, head ? line : (0x80000000u | (uint32_t)lane));
        if (pure_skip) {
            --pure_skip;
        } else {
            // Pure sets: in a group where no head can hit all miss; a group
            // whose heads all hold their lines all hits.  If every earlier
            // head of its group misses, a first use misses when its line is
            // not held or (FIFO) is pushed out by those misses, and a repeat
            // (FIFO) when at least a misses of its set came since its previous
            // use.  RANDOM takes only groups of new lines not held.
            const uint32_t sm0 =
                __match_any_sync(kFull, head ? set : (0x80000000u | (uint32_t)lane));
            const uint32_t pm0 = lm0 & lt;
            const int fh = __ffs(hb) - 1;
            const bool one_set = POLICY == PCHASE_FIFO && __shfl_sync(kFull, sm0, fh) == hb;
            if (one_set) {
                // every head in one set s0: its counters are one broadcast
                // load, a head's miss rank is its head rank r, and when all
                // miss, the first a ranks find the ways in use (evicting
                // their lines when the set is full) and the last a ranks are
                // what stays (consecutive ranks fill consecutive ways)
                const uint32_t s0 = __shfl_sync(kFull, set, fh);
                const uint4 m = meta[s0];
                const uint32_t a = ways;
                const uint32_t r = __popc(hb & lt);
                bool nh = w0 == 0u && pm0 == 0u;
                if (pm0) {
                    const uint32_t below = (2u << (31 - __clz(pm0))) - 1u;
                    nh = (uint32_t)__popc(hb & lt & ~below) >= a;
                } else if (w0) {
                    const uint32_t rho = mod_ways(w0 - 1u + a - m.x, a);
                    nh = r >= a - m.y + rho + 1u;
                }
                if (__all_sync(kFull, !head || nh)) {
                    const uint32_t M = __popc(hb);
                    const uint32_t insw = mod_ways(m.x + m.y + r, a);
                    uint32_t *const sl = sline + (size_t)s0 * a;
                    if (head && r < a && m.y + r >= a) tab[sl[insw]] = 0;
                    __syncwarp();
                    if (head && r + a >= M) {
                        sl[insw] = line;
                        tab[line] = (uint16_t)(insw + 1);
                    }
                    if (lane == fh) meta[s0] = after_misses(m, M);
                    __syncwarp();
                    return head;
                }
                pure_skip = 7;  // (the test below would fail the same way)
            } else {
                bool nohit = w0 == 0u && pm0 == 0u;
                if (POLICY == PCHASE_FIFO) {
                    if (pm0) {
                        const uint32_t below = (2u << (31 - __clz(pm0))) - 1u;
                        nohit = (uint32_t)__popc(sm0 & lt & ~below) >= ways;
                    } else if (w0) {
                        // held in way w, rho lines inserted before it: it leaves at
                        // the (a - L + rho + 1)-th miss of its set
                        const uint4 mf = head ? meta[set] : make_uint4(0, 0, 0, 0);
                        const uint32_t rho = mod_ways(w0 - 1u + ways - mf.x, ways);
                        nohit = (uint32_t)__popc(sm0 & lt) >= ways - mf.y + rho + 1u;
                    }
                }
                // held groups hit and change nothing; the others all miss
                const uint32_t hbal = __ballot_sync(kFull, head && w0 != 0u);
                const uint32_t nbal = __ballot_sync(kFull, head && nohit);
                const bool gheld = head && (hbal & sm0) == sm0;
                if (__all_sync(kFull, !head || gheld || (nbal & sm0) == sm0))
                    return fresh_step(line, set, head && !gheld, lane, lt, sm0);
                pure_skip = 7;
            }
        }
        {
            // one set with few lines not held: miss by miss
            const uint32_t s0 = __shfl_sync(kFull, set, __ffs(hb) - 1);
            const uint32_t cand = __ballot_sync(kFull, head && w0 == 0u);
            if (ways <= 32u && __popc(cand) <= kSeqMaxFirst &&
                __all_sync(kFull, !head || set == s0))
                return seq_step(line, s0, head, w0 != 0u, cand, lane);
        }
        const Grouped g = group_heads(line, set, head, lane, lt, perm);
        const uint32_t a = ways;
        const uint32_t ltg = g.gmask & lt;
        const uint32_t r = (uint32_t)lane - g.gb;
        const uint4 m = g.act ? meta[g.set] : make_uint4(0, 0, 0, 0);
        const uint32_t w1 = !g.act ? 0u : g.same ? w0 : tab[g.x];
        const uint32_t lm =
            g.same ? lm0 : __match_any_sync(kFull, g.act ? g.x : (0x80000000u | (uint32_t)lane));
        const uint32_t pm = lm & lt;
        const int prev = pm ? 31 - __clz(pm) : -1;
        // way of the group's r-th miss, and whether it evicts
        bool evicts;
        const uint32_t insw = rank_way(m, g.set, r, evicts);
        // next group rank with the same way
        const uint32_t sw = __match_any_sync(kFull, g.act ? g.set * a + insw
                                                           : (0x80000000u | (uint32_t)lane));
        const uint32_t above = sw & ~(lt | (1u << lane));
        const int32_t nx = above ? (int32_t)(__ffs(above) - 1 - g.gb) : kBig;
        // eviction index of this line's way (first group rank targeting it)
        int32_t e0 = -1;
        if (POLICY == PCHASE_FIFO) {
            if (w1) e0 = (int32_t)(mod_ways(w1 - 1 + a - m.x, a) + (a - m.y));
        } else {
            if (g.act && (sw & lt) == 0) scr[g.set * a + insw] = make_uint2(stamp, r);
            __syncwarp();
            if (w1) {
                const uint2 q = scr[g.set * a + w1 - 1];
                e0 = q.x == stamp ? (int32_t)q.y : kBig;
            }
        }
        // Fixed point over the miss vector.  Before access i its line's way
        // is next evicted at the group rank nx(rho) if an earlier access of
        // the line missed, rho the miss rank of the last such one (a hit
        // moves nothing), else at e0; i misses when more misses precede it
        // in its group than that rank.  Every lane reads its line's last
        // earlier miss from the current vector, so a run of repeats settles
        // in one round.
        // (from the sure misses: first uses of lines not held)
        bool miss = g.act && w1 == 0 && prev < 0;
        const uint32_t lme = lm & lt;  // earlier lanes of this lane's line
        for (int it = 0; it < 33; ++it) {
            const uint32_t bal = __ballot_sync(kFull, miss);
            const int32_t mi = __popc(bal & ltg);
            // where a line this lane inserted would be evicted next
            const int32_t nxm = __shfl_sync(kFull, nx, (g.gb + (uint32_t)mi) & 31u);
            const uint32_t pmiss = lme & bal;
            const int32_t pe = __shfl_sync(kFull, nxm, pmiss ? 31 - __clz(pmiss) : lane);
            const bool nm = g.act && mi > (pmiss ? pe : e0);
            if (__all_sync(kFull, nm == miss)) break;
            miss = nm;
        }
        // state update
        const uint32_t bal = __ballot_sync(kFull, miss);
        const uint32_t mi = __popc(bal & ltg);
        const uint32_t M = __popc(bal & g.gmask);
        // the way this lane's miss fills (bit 31: it evicts; ways < 2^24)
        const uint32_t wv = __shfl_sync(kFull, insw | (evicts ? 0x80000000u : 0u),
                                        (g.gb + mi) & 31u);
        const uint32_t myw = wv & 0x7FFFFFFFu;
        const bool myev = (wv >> 31) != 0;
        const uint32_t smw = __match_any_sync(kFull, miss ? g.set * a + myw
                                                         : (0x80000000u | (uint32_t)lane));
        const uint32_t below = smw & lt;
        const bool last = miss && (smw & ~(lt | (1u << lane))) == 0;
        const uint32_t prev_line = __shfl_sync(kFull, g.x, below ? 31 - __clz(below) : lane);
        if (miss && (below || myev)) {
            const uint32_t old = below ? prev_line : sline[g.set * a + myw];
            tab[old] = 0;
        }
        __syncwarp();
        if (last) {
            sline[g.set * a + myw] = g.x;
            tab[g.x] = (uint16_t)(myw + 1);
        }
        if (g.act && (uint32_t)lane == g.gb) {
            uint4 n = m;
            if (POLICY == PCHASE_FIFO) {
                const uint32_t tot = m.y + M;
                n.y = tot < a ? tot : a;
                n.x = mod_ways(m.x + (tot > a ? tot - a : 0u), a);
            } else {
                const uint32_t tot = m.x + M;
                n.x = tot < a ? tot : a;
                n.y = m.y + (tot > a ? tot - a : 0u);
            }
            meta[g.set] = n;
        }
        __syncwarp();
        if (g.same) return miss && head;
        return __shfl_sync(kFull, miss ? 1u : 0u, head ? g.dest : (uint32_t)lane) != 0 && head;
    }
};

// LRU.  Arena: uint32 perm[32] (+ pad to 256 B); uint4 meta[T] =
// {tail, head, live, compact} (monotone ring positions; compact = 1 when no
// stale entry lies between tail and head); uint32 ring[T*R];
// uint16 tab[table_n] (ring index + 1).
struct BatchLRU {
    uint4 *meta;
    uint32_t *ring;
    uint16_t *tab;
    uint32_t *perm;
    uint32_t ways, R, rmask;

    __device__ __forceinline__ void bind(uint8_t *arena, const SimItem &it) {
        ways = it.ways;
        R = it.ring;
        rmask = R - 1;
        sets_m = it.magic_m;
        sets_s1 = it.s1;
        sets_s2 = it.s2;
        nsets = it.sets;
        lstep = ((it.lsh >> 18) & 1u) ? it.gsets : 1u;  // compact lines: id * lstep is the line
        size_t off = 0;
        perm = reinterpret_cast<uint32_t *>(arena);
        off += 256;
        meta = reinterpret_cast<uint4 *>(arena + off);
        off += 16ull * it.sets;
        ring = reinterpret_cast<uint32_t *>(arena + off);
        off += 4ull * it.sets * R;
        tab = reinterpret_cast<uint16_t *>(arena + off);
    }

    __device__ __forceinline__ void clear(const SimItem &it, int lane) {
        for (uint32_t i = lane; i < it.sets; i += 32) meta[i] = make_uint4(0, 0, 0, 1);
        uint32_t *t32 = reinterpret_cast<uint32_t *>(tab);
        for (uint32_t i = lane; i < (it.table_n + 1) / 2; i += 32) t32[i] = 0;
    }

    // Moves the live entries of [tail, head) down to start at tail.
    __device__ __forceinline__ uint4 compact(uint32_t set, uint4 m, int lane, uint32_t lt) {
        uint32_t *rg = ring + (size_t)set * R;
        uint32_t done = 0;
        for (uint32_t p0 = m.x; p0 < m.y; p0 += 32) {
            const uint32_t p = p0 + (uint32_t)lane;
            const uint32_t e = p < m.y ? rg[p & rmask] : kStale;
            const bool live = e != kStale;
            const uint32_t bal = __ballot_sync(kFull, live);
            __syncwarp();
            if (live) {
                const uint32_t d = (m.x + done + __popc(bal & lt)) & rmask;
                rg[d] = e;
                tab[e] = (uint16_t)(d + 1);
            }
            __syncwarp();
            done += __popc(bal);
        }
        m.y = m.x + done;
        m.w = 1;
        if (lane == 0) meta[set] = m;
        __syncwarp();
        return m;
    }

    // Every head of set s in the step misses (`last` marks the last use of
    // each of its lines): the D distinct lines go on top in last-use order
    // (only the last a of them stay when D > a) and the oldest held lines
    // leave until a lines are held.
    __device__ __forceinline__ void nohit_step(uint32_t s, uint32_t line, bool last, int lane,
                                               uint32_t lt) {
        const uint32_t a = ways;
        uint32_t *rg = ring + (size_t)s * R;
        uint4 m = meta[s];
        if (m.y - m.x > R - 64) m = compact(s, m, lane, lt);
        const uint32_t lb = __ballot_sync(kFull, last);
        const uint32_t D = __popc(lb);
        const uint32_t keep_old = D <= a ? a - D : 0u;
        const uint32_t E = m.z > keep_old ? m.z - keep_old : 0u;
        // evict the E oldest held lines; the tail moves to the first kept one,
        // or past the step's own lines that do not stay
        uint32_t new_tail = m.y + (D > a ? D - a : 0u), evd = 0;
        bool found = false;
        if (m.w) {
            // compact ring: the E oldest held lines are positions tail .. tail+E-1
            for (uint32_t q = (uint32_t)lane; q < E; q += 32) {
                const uint32_t pq = (m.x + q) & rmask;
                tab[rg[pq]] = 0;
                rg[pq] = kStale;
            }
            found = E < m.z;
            if (found) new_tail = m.x + E;
            evd = E;
        }
        for (uint32_t p0 = m.x; !m.w && p0 < m.y && (evd < E || !found); p0 += 32) {
            const uint32_t p = p0 + (uint32_t)lane;
            const uint32_t e = p < m.y ? rg[p & rmask] : kStale;
            const bool live = e != kStale;
            const uint32_t bal = __ballot_sync(kFull, live);
            const bool ev = live && evd + __popc(bal & lt) < E;
            if (ev) {
                tab[e] = 0;
                rg[p & rmask] = kStale;
            }
            const uint32_t keep = __ballot_sync(kFull, live && !ev);
            if (!found && keep) {
                new_tail = p0 + (uint32_t)(__ffs(keep) - 1);
                found = true;
            }
            evd += __popc(bal);
        }
        __syncwarp();
        if (last) {
            const uint32_t q = __popc(lb & lt);
            const uint32_t p = (m.y + q) & rmask;
            if (D > a && q < D - a) {
                rg[p] = kStale;
            } else {
                rg[p] = line;
                tab[line] = (uint16_t)(p + 1);
            }
        }
        // a prefix of the held lines left: a compact ring stays compact, and
        // one whose held lines all left becomes compact
        const uint32_t cpt = (m.w || !found) ? 1u : 0u;
        if (lane == 0) meta[s] = make_uint4(new_tail, m.y + D, D <= a ? m.z - E + D : a, cpt);
        __syncwarp();
    }

    // The state at access c0 of a time part: every set's a most recent
    // distinct lines before c0, newest last (by the stack property that is
    // the whole of an LRU set's state).  The trace is read backwards 32
    // accesses at a time; the newest occurrence of a line not yet taken goes
    // below the set's lines taken so far, until every set holds a lines or
    // the trace's start is reached.  load(t) gives the line of access t, or
    // kInvalidLine for an access the simulation skips.
    //
    // tgt (may be NULL): per set, the lines it needs before it is complete,
    // min(a, its distinct lines over the whole trace); sets that need none
    // are complete from the start, and the read stops once every set is.
    template <typename Load>
    __device__ __forceinline__ void rebuild(uint32_t c0, uint32_t T, int lane, uint32_t lt,
                                            Load load, const uint32_t *tgt) {
        const uint32_t a = ways;
        uint32_t full = 0;
        if (tgt) {
            for (uint32_t s0 = 0; s0 < T; s0 += 32) {
                const uint32_t s = s0 + (uint32_t)lane;
                full += (uint32_t)__popc(__ballot_sync(kFull, s < T && tgt[s] == 0));
            }
        }
        auto need_of = [&](uint32_t set) -> uint32_t { return tgt ? tgt[set] : a; };
        auto chunk = [&](uint32_t ln) {
            const bool valid = ln != kInvalidLine;
            const uint32_t set = valid ? set_of(ln) : 0u;
            // a chunk whose lines are all taken or in complete sets changes nothing
            const bool need = valid && tab[ln] == 0 && meta[set].y < need_of(set);
            if (!__any_sync(kFull, need)) return;
            const uint32_t lm = __match_any_sync(kFull, valid ? ln : (0x80000000u | (uint32_t)lane));
            const bool cand = need && (lm & ~(lt | (1u << lane))) == 0;  // newest in the chunk
            const uint32_t sm = __match_any_sync(kFull, cand ? set : (0x80000000u | (uint32_t)lane));
            const uint32_t k = cand ? meta[set].y : 0u;
            const uint32_t q = k + (uint32_t)__popc(sm & ~(lt | (1u << lane)));  // newer ones first
            const bool lead_s = cand && (sm & lt) == 0;
            full += (uint32_t)__popc(
                __ballot_sync(kFull, lead_s && k + (uint32_t)__popc(sm) >= need_of(set)));
            __syncwarp();
            if (cand && q < a) {
                ring[(size_t)set * R + (a - 1 - q)] = ln;
                tab[ln] = (uint16_t)(a - q);
            }
            if (lead_s) meta[set].y = min(a, k + (uint32_t)__popc(sm));
            __syncwarp();
        };
        // chunks of 32 accesses, newest first; the lines of the next kAhead
        // chunks back are loaded while these are taken
        constexpr int kAhead = 4;
        uint32_t v[kAhead];
#pragma unroll
        for (int k = 0; k < kAhead; ++k) {
            const int64_t t = (int64_t)c0 - 32 * (k + 1) + lane;
            v[k] = t >= 0 ? load((uint32_t)t) : kInvalidLine;
        }
        for (int64_t b = c0; b > 0 && full < T; b -= 32 * kAhead) {
#pragma unroll
            for (int k = 0; k < kAhead; ++k) {
                const uint32_t ln = v[k];
                const int64_t t = b - 32 * (kAhead + k + 1) + lane;
                v[k] = t >= 0 ? load((uint32_t)t) : kInvalidLine;
                if (b - 32 * k > 0 && full < T) chunk(ln);
            }
        }
        for (uint32_t s = (uint32_t)lane; s < T; s += 32) {
            const uint32_t k = meta[s].y;
            meta[s] = make_uint4(a - k, a, k, 1u);
        }
        __syncwarp();
    }
    uint32_t sets_m, sets_s1, sets_s2, nsets, lstep;
    // set of a line as the unit keys it (a compact id stands for id * lstep)
    __device__ __forceinline__ uint32_t set_of(uint32_t ln) const {
        const uint32_t l = ln * lstep;
        return l - div_q(l, sets_m, sets_s1, sets_s2) * nsets;
    }

    // All set groups at once.  A group of g heads can push out at most g
    // resident lines, so a line whose rank (live entries older than it) is g
    // or more is a sure hit, and the g oldest live entries of the set (its
    // window) are all that is needed: the group's own lanes read the ring g
    // positions at a time until g live entries are seen or the ring ends.
    __device__ __forceinline__ bool resolve(uint32_t line, uint32_t set, bool head, uint32_t,
                                            int lane, uint32_t lt, uint32_t) {
        // Pure sets.  Only a miss evicts, so when every head of a set's group
        // holds its line at the start of the step (a held group), all of them
        // hit: their old entries go stale and the lines are appended in
        // last-use order, the held count and the tail stay.  A group in which
        // no head can hit (each first use of a line not held, each repeat
        // after at least a other distinct lines of its set since its previous
        // use, each of them a miss inserted above it) all misses.  Steps made
        // of such groups (at most 8 of the second kind) skip the general path.
        const uint32_t hb = __ballot_sync(kFull, head);
        if (hb == 0) return false;
        uint32_t w0 = head ? tab[line] : 1u;
        const uint32_t sm0 = __match_any_sync(kFull, head ? set : (0x80000000u | (uint32_t)lane));
        const uint32_t lm0 = __match_any_sync(kFull, head ? line : (0x80000000u | (uint32_t)lane));
        uint4 m0 = head ? meta[set] : make_uint4(0, 0, 0, 0);
        const uint32_t pm0 = lm0 & lt;
        const bool last = head && (lm0 & ~(lt | (1u << lane))) == 0;
        const uint32_t hbal = __ballot_sync(kFull, head && w0 != 0u);
        const bool gheld = head && (hbal & sm0) == sm0;
        bool pure = hbal == hb;
        uint32_t nlead = 0;
        if (!pure) {
            const int prev = pm0 ? 31 - __clz(pm0) : -1;
            const uint32_t pkey = head ? (uint32_t)(prev + 1) : 63u;
            const uint32_t pthr = prev < 0 ? 0u : (uint32_t)prev + 1;
            // distinct lines between a repeat and its previous use (none
            // needed when no line repeats inside the step)
            uint32_t between = 0;
            if (__any_sync(kFull, prev >= 0))
                between = lanes_below(pkey, pthr) & sm0 & lt &
                          ~((prev < 0) ? 0u : ((2u << prev) - 1u));
            // a held first use at depth d leaves once d plus the distinct
            // lines before it in the step reach a (exact depth needs a
            // compact ring)
            const uint32_t fbal = __ballot_sync(kFull, head && prev < 0);
            bool nohit;
            if (prev >= 0) nohit = (uint32_t)__popc(between) >= ways;
            else if (w0 == 0u) nohit = true;
            else nohit = m0.w && ((m0.y - w0) & rmask) + __popc(fbal & sm0 & lt) >= ways;
            nohit = nohit && head;
            const uint32_t nbal = __ballot_sync(kFull, nohit);
            const bool gnohit = head && !gheld && (nbal & sm0) == sm0;
            nlead = __ballot_sync(kFull, gnohit && (sm0 & lt) == 0);
            pure = __all_sync(kFull, !head || gheld || gnohit) && __popc(nlead) <= 8;
        }
        if (pure && __any_sync(kFull, gheld)) {
            // room for 32 entries in every held group's ring: compact the ones
            // nearly full (the lines keep their order; positions move)
            const uint32_t full =
                __ballot_sync(kFull, gheld && (sm0 & lt) == 0 && m0.y - m0.x > R - 64);
            if (full) {
                for (uint32_t todo = full; todo; todo &= todo - 1) {
                    const uint32_t s0 = __shfl_sync(kFull, set, __ffs(todo) - 1);
                    compact(s0, meta[s0], lane, lt);
                }
                w0 = head ? tab[line] : 1u;
                m0 = head ? meta[set] : make_uint4(0, 0, 0, 0);
            }
            const uint32_t lb = __ballot_sync(kFull, last && gheld);
            // a held group that re-uses exactly its set's D oldest lines (a
            // cyclic stream) leaves a stale prefix: the tail moves past it and
            // a compact ring stays compact
            const uint32_t D = __popc(lb & sm0);
            const bool front = gheld && pm0 == 0 && ((w0 - 1u - m0.x) & rmask) < D;
            const uint32_t fb = __ballot_sync(kFull, gheld && pm0 == 0);
            const uint32_t ob = __ballot_sync(kFull, front);
            uint32_t *rg0 = ring + (size_t)(gheld ? set : 0u) * R;
            if (gheld && pm0 == 0) rg0[w0 - 1] = kStale;
            __syncwarp();
            if (last && gheld) {
                const uint32_t p = (m0.y + __popc(lb & sm0 & lt)) & rmask;
                rg0[p] = line;
                tab[line] = (uint16_t)(p + 1);
            }
            if (gheld && (sm0 & ~(lt | (1u << lane))) == 0) {
                const bool adv = m0.w && (ob & sm0) == (fb & sm0);
                meta[set] = make_uint4(adv ? m0.x + D : m0.x, m0.y + D, m0.z, adv ? 1u : 0u);
            }
            __syncwarp();
        }
        if (pure) {
            for (uint32_t todo = nlead; todo; todo &= todo - 1) {
                const int ld = __ffs(todo) - 1;
                const uint32_t s0 = __shfl_sync(kFull, set, ld);
                const uint32_t gmask = __shfl_sync(kFull, sm0, ld);
                nohit_step(s0, line, last && ((gmask >> lane) & 1u), lane, lt);
            }
            return head && !gheld;
        }
        const Grouped g = group_heads(line, set, head, lane, lt, perm);
        const uint32_t a = ways;
        const uint32_t gm = g.gmask;
        const uint32_t gs = g.act ? (uint32_t)__popc(gm) : 0u;
        const uint32_t j = (uint32_t)lane - g.gb;
        const uint32_t lm = __match_any_sync(kFull, g.act ? g.x : (0x80000000u | (uint32_t)lane));
        const uint32_t pm = lm & lt;
        const int prev = pm ? 31 - __clz(pm) : -1;
        const bool first = g.act && prev < 0;
        const bool lastocc = g.act && (lm & ~(lt | (1u << lane))) == 0;
        uint32_t *rg = ring + (size_t)(g.act ? g.set : 0) * R;
        uint4 m = g.act ? meta[g.set] : make_uint4(0, 0, 0, 0);
        // compaction of nearly full rings (one set at a time, rare)
        uint32_t need = __ballot_sync(kFull, g.act && lane == (int)g.gb && m.y - m.x > R - 64);
        while (need) {
            const uint32_t gl = __ffs(need) - 1;
            need &= need - 1;
            const uint32_t s = __shfl_sync(kFull, g.set, gl);
            uint4 ms = meta[s];
            ms = compact(s, ms, lane, lt);
            if (g.act && g.set == s) m = ms;
        }
        // windows: up to kWin rounds of g positions per group
        constexpr int kWin = 8;
        uint32_t wbal[kWin];
        uint32_t wlive = 0, nround = 0;
        bool done = !g.act;
#pragma unroll
        for (int r = 0; r < kWin; ++r) {
            const uint32_t p = m.x + (uint32_t)r * gs + j;
            const uint32_t e = (!done && p < m.y) ? rg[p & rmask] : kStale;
            wbal[r] = __ballot_sync(kFull, e != kStale) & gm;
            if (!done) {
                wlive += __popc(wbal[r]);
                nround = (uint32_t)r + 1;
                if (wlive >= gs || m.x + (uint32_t)(r + 1) * gs >= m.y) done = true;
            }
            if (__all_sync(kFull, done)) break;
        }
        // a group whose window is still short (stale entries in the way) is
        // compacted and scanned again in one round
        uint32_t redo = __ballot_sync(kFull, !done && lane == (int)g.gb);
        if (redo) {
            while (redo) {
                const uint32_t gl = __ffs(redo) - 1;
                redo &= redo - 1;
                const uint32_t s = __shfl_sync(kFull, g.set, gl);
                uint4 ms = compact(s, meta[s], lane, lt);
                if (g.act && g.set == s) m = ms;
            }
            const bool again = !done;
            const uint32_t p = m.x + j;
            const uint32_t e = (again && p < m.y) ? rg[p & rmask] : kStale;
            const uint32_t bal = __ballot_sync(kFull, e != kStale) & gm;
            if (again) {
                wbal[0] = bal;
                wlive = __popc(bal);
                nround = 1;
            }
        }
        __syncwarp();
        const uint32_t w1 = g.act ? tab[g.x] : 0u;
        bool miss = false;
        if (__all_sync(kFull, !g.act || (first && w1 == 0))) {
            // every head is its line's first use in the step and the line is
            // not held (a thrashing stream): all of them miss
            miss = g.act;
        } else {
            // rank of each head's resident line among the window's live entries
            uint32_t rank = 32;
            if (w1) {
                const uint32_t off = (w1 - 1 - m.x) & rmask;
                if (off < nround * gs) {
                    const uint32_t r0 = off / gs, j0 = off - r0 * gs;
                    uint32_t rk = 0;
#pragma unroll
                    for (int r = 0; r < kWin; ++r) {
                        if ((uint32_t)r < r0) rk += __popc(wbal[r]);
                        else if ((uint32_t)r == r0)
                            rk += __popc(wbal[r] & ((1u << (g.gb + j0)) - 1u));
                    }
                    if (rk < gs) rank = rk;
                }
            }
            // lines older than this one or new, first used earlier in the group
            const uint32_t key = first ? (w1 == 0 ? 0u : rank + 1) : 63u;
            const uint32_t older = lanes_below(key, rank + 1) & gm & lt;
            // distinct lines strictly between a repeat and its previous use
            const uint32_t pkey = g.act ? (uint32_t)(prev + 1) : 63u;
            const uint32_t pthr = prev < 0 ? 0u : (uint32_t)prev + 1;
            const uint32_t between = lanes_below(pkey, pthr) & gm & lt &
                                     ~((prev < 0) ? 0u : ((2u << prev) - 1u));
            if (g.act) {
                if (first) {
                    if (w1 == 0) miss = true;
                    else if (rank < 32) miss = (m.z - 1 - rank) + __popc(older) >= a;
                } else {
                    miss = (uint32_t)__popc(between) >= a;
                }
            }
        }
        // ----- updates, every group at once
        const uint32_t lastbal = __ballot_sync(kFull, lastocc);
        const uint32_t D = __popc(lastbal & gm);
        const uint32_t Rb = __popc(__ballot_sync(kFull, first && w1 != 0) & gm);
        if (first && w1) rg[w1 - 1] = kStale;
        __syncwarp();
        const uint32_t keep_old = D <= a ? a - D : 0u;
        const uint32_t old_live = m.z - Rb;
        const uint32_t E = old_live > keep_old ? old_live - keep_old : 0u;
        uint32_t evd = 0, new_tail = m.x + nround * gs < m.y ? m.x + nround * gs : m.y;
        bool tail_set = false;
        for (uint32_t r = 0; r < (uint32_t)kWin; ++r) {
            const bool in = g.act && r < nround;
            const uint32_t p = m.x + r * gs + j;
            const uint32_t e = (in && p < m.y) ? rg[p & rmask] : kStale;
            const bool live = e != kStale;
            const uint32_t bal = __ballot_sync(kFull, live) & gm;
            const bool ev = live && evd + __popc(bal & lt) < E;
            if (ev) {
                tab[e] = 0;
                rg[p & rmask] = kStale;
            }
            const uint32_t keep = __ballot_sync(kFull, live && !ev) & gm;
            if (in && !tail_set && keep) {
                new_tail = m.x + r * gs + (__ffs(keep) - 1 - g.gb);
                tail_set = true;
            }
            evd += __popc(bal);
            if (__all_sync(kFull, !in || r + 1 >= nround)) break;
        }
        // append the group's lines in last-use order
        if (lastocc) {
            const uint32_t q = __popc(lastbal & gm & lt);
            const uint32_t p = (m.y + q) & rmask;
            if (D > a && q < D - a) {
                rg[p] = kStale;
                tab[g.x] = 0;
            } else {
                rg[p] = g.x;
                tab[g.x] = (uint16_t)(p + 1);
            }
        }
        if (g.act && (uint32_t)lane == g.gb) {
            // no old line stays: the ring is the step's own lines, whose live
            // entries follow the D - a that do not stay
            const bool fresh = old_live == E;
            uint4 n;
            n.x = fresh ? m.y + (D > a ? D - a : 0u) : new_tail;
            n.y = m.y + D;
            n.z = D <= a ? old_live - E + D : a;
            n.w = fresh ? 1u : 0u;
            meta[g.set] = n;
        }
        __syncwarp();
        return __shfl_sync(kFull, miss ? 1u : 0u, head ? g.dest : (uint32_t)lane) != 0 && head;
    }
};

// --------------------------------------------------------------- unit loop
// cp.async (Ampere-style asynchronous global -> shared copies, 4 bytes a lane)
__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// ORs one step's miss bits into the unit's bitmap (words zeroed beforehand):
// lanes hold increasing positions, so lanes sharing a word are consecutive;
// each run of them is OR-reduced and its first lane issues one reduction.
__device__ __forceinline__ void emit_bits(uint32_t *bm, uint32_t pos, bool miss, bool act,
                                          int lane) {
    const uint32_t p0 = __shfl_sync(kFull, pos, 0);
    if (__all_sync(kFull, act && pos == p0 + (uint32_t)lane)) {
        // 32 consecutive positions: at most two words
        const uint32_t bits = __ballot_sync(kFull, miss);
        if (lane == 0) {
            const uint32_t sh = p0 & 31u;
            atomicOr(bm + (p0 >> 5), bits << sh);
            if (sh && (bits >> (32u - sh))) atomicOr(bm + (p0 >> 5) + 1, bits >> (32u - sh));
        }
        return;
    }
    const uint32_t w = act ? pos >> 5 : 0xFFFFFFFFu;
    uint32_t b = miss ? 1u << (pos & 31u) : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t vb = __shfl_down_sync(kFull, b, o);
        const uint32_t vw = __shfl_down_sync(kFull, w, o);
        if (lane + o < 32 && vw == w) b |= vb;
    }
    const uint32_t wp = __shfl_up_sync(kFull, w, 1);
    if (act && b && (lane == 0 || wp != w)) atomicOr(bm + w, b);
}

// Kinds of set state: mode * 3 + policy.
enum : uint32_t {
    kScanLru = kModeScan * 3 + PCHASE_LRU,
    kScanFifo = kModeScan * 3 + PCHASE_FIFO,
    kScanRandom = kModeScan * 3 + PCHASE_RANDOM,
    kTableLru = kModeTable * 3 + PCHASE_LRU,
    kTableFifo = kModeTable * 3 + PCHASE_FIFO,
    kTableRandom = kModeTable * 3 + PCHASE_RANDOM,
    kBatchLru = kModeBatch * 3 + PCHASE_LRU,
    kBatchFifo = kModeBatch * 3 + PCHASE_FIFO,
    kBatchRandom = kModeBatch * 3 + PCHASE_RANDOM,
    // way scans whose set state lives in global memory (caches too large for
    // any shared-memory arena)
    kGlobalScanLru = 9 + PCHASE_LRU,
    kGlobalScanFifo = 9 + PCHASE_FIFO,
    kGlobalScanRandom = 9 + PCHASE_RANDOM,
};

// POOL: the kernel of the global-state pool, whose units all keep their set
// state in global memory (way scans); the other kernel has no such unit, so
// neither instantiation carries the other's resolvers.
// Every set mode behind one resolve call.  The state's views are rebuilt
// from the arena each step (a few integer ops), so all modes share one copy
// of the unit loop: the form for launches whose warps run units of many
// kinds side by side, where per-kind copies of the loop would not stay in
// the instruction cache together.
template <bool POOL>
struct AnyResolver {
    uint8_t *sp;
    const SimItem *it;
    uint32_t kind;
    __device__ __forceinline__ void bind(uint8_t *arena, const SimItem &i) {
        sp = arena;
        it = &i;
        const uint32_t pol = i.policy < 2u ? i.policy : 2u;
        kind = POOL ? (uint32_t)kGlobalScanLru + pol : (uint32_t)i.mode * 3u + pol;
    }
    template <typename R>
    __device__ __forceinline__ bool run(uint32_t line, uint32_t set, bool head, uint32_t pos,
                                        int lane, uint32_t lt, uint32_t step) {
        R r;
        r.bind(sp, *it);
        return r.resolve(line, set, head, pos, lane, lt, step);
    }
    __device__ __forceinline__ bool resolve(uint32_t line, uint32_t set, bool head, uint32_t pos,
                                            int lane, uint32_t lt, uint32_t step) {
        if constexpr (POOL) {
            switch (kind) {
            case kGlobalScanLru:
                return run<RoundResolver<ScanSets<PCHASE_LRU>>>(line, set, head, pos, lane, lt, step);
            case kGlobalScanFifo:
                return run<RoundResolver<ScanSets<PCHASE_FIFO>>>(line, set, head, pos, lane, lt, step);
            default:
                return run<RoundResolver<ScanSets<PCHASE_RANDOM>>>(line, set, head, pos, lane, lt, step);
            }
        }
        switch (kind) {
        case kScanLru:
            return run<RoundResolver<ScanSets<PCHASE_LRU>>>(line, set, head, pos, lane, lt, step);
        case kScanFifo:
            return run<RoundResolver<ScanSets<PCHASE_FIFO>>>(line, set, head, pos, lane, lt, step);
        case kScanRandom:
            return run<RoundResolver<ScanSets<PCHASE_RANDOM>>>(line, set, head, pos, lane, lt, step);
        case kTableLru:
            return run<RoundResolver<TableSets<PCHASE_LRU>>>(line, set, head, pos, lane, lt, step);
        case kTableFifo:
            return run<RoundResolver<TableSets<PCHASE_FIFO>>>(line, set, head, pos, lane, lt, step);
        case kTableRandom:
            return run<RoundResolver<TableSets<PCHASE_RANDOM>>>(line, set, head, pos, lane, lt, step);
        case kBatchLru:
            return run<BatchLRU>(line, set, head, pos, lane, lt, step);
        case kBatchFifo:
            return run<BatchFR<PCHASE_FIFO>>(line, set, head, pos, lane, lt, step);
        default:
            return run<BatchFR<PCHASE_RANDOM>>(line, set, head, pos, lane, lt, step);
        }
    }
};

template <bool POOL>
__device__ __forceinline__ void clear_state(uint32_t kind, uint8_t *st, uint8_t *gst,
                                            const SimItem &it, int lane) {
    if constexpr (POOL) {
        switch (kind) {
        case kGlobalScanLru: { ScanSets<PCHASE_LRU> S; S.bind(gst, it); S.clear(it, lane); return; }
        case kGlobalScanFifo: {
            ScanSets<PCHASE_FIFO> S; S.bind(gst, it); S.clear(it, lane); return; }
        default: { ScanSets<PCHASE_RANDOM> S; S.bind(gst, it); S.clear(it, lane); return; }
        }
    }
    switch (kind) {
    case kScanLru: { ScanSets<PCHASE_LRU> S; S.bind(st, it); S.clear(it, lane); break; }
    case kScanFifo: { ScanSets<PCHASE_FIFO> S; S.bind(st, it); S.clear(it, lane); break; }
    case kScanRandom: { ScanSets<PCHASE_RANDOM> S; S.bind(st, it); S.clear(it, lane); break; }
    case kTableLru: { TableSets<PCHASE_LRU> S; S.bind(st, it); S.clear(it, lane); break; }
    case kTableFifo: { TableSets<PCHASE_FIFO> S; S.bind(st, it); S.clear(it, lane); break; }
    case kTableRandom: { TableSets<PCHASE_RANDOM> S; S.bind(st, it); S.clear(it, lane); break; }
    case kBatchLru: { BatchLRU S; S.bind(st, it); S.clear(it, lane); break; }
    case kBatchFifo: { BatchFR<PCHASE_FIFO> S; S.bind(st, it); S.clear(it, lane); break; }
    default: { BatchFR<PCHASE_RANDOM> S; S.bind(st, it); S.clear(it, lane); break; }
    }
}

// Matcher: true when the candidate's distance, summed atomically by its other
// units, plus this unit's own part is already above the bound.  Distances at
// or under the bound are never cut short, so they stay exact; one above it is
// only known to be above it.
__device__ __forceinline__ bool over_bound(const SimOut &out, uint32_t cand, uint64_t own,
                                           int lane) {
    if (out.stop_above == ~0ull) return false;
    unsigned long long d = 0;
    if (lane == 0) d = *reinterpret_cast<volatile const unsigned long long *>(out.dist + cand);
    d = __shfl_sync(kFull, d, 0);
    return d + own > out.stop_above;
}

// One unit: gather trips fill the queue with the unit's run heads, and each
// step hands the next 32 of them to the unit's set state in trace order.
// The steps of one unit with its set mode's resolver R, bound once to the
// unit's set state at sp (shared memory, or global memory for the pool).
template <typename R>
__device__ __forceinline__ void run_steps(const SimItem &it, uint32_t arena, uint8_t *st,
                                          uint8_t *sp, uint32_t kind, const SimOut &out,
                                          int lane) {
    uint2 *const queue = reinterpret_cast<uint2 *>(g_smem + arena);
    R res;
    res.bind(sp, it);
    const uint32_t len = it.len;
    const uint32_t *__restrict__ idxp = it.idx;
    const uint32_t N = it.n_elems;
    const uint32_t lsh = it.lsh & 255u, mk = (it.lsh >> 8) & 255u;  // line shift, mapping
    // unequal sets: the residue r = line mod M (M in gsets) goes to set r mod T
    // below T * a (a: it.kmagic), else to set 0
    const bool uneq = (it.lsh >> 16) & 1u;
    const uint32_t uta = uneq ? it.sets * it.kmagic : 0u;
    // compact lines: a strided chain visits only the multiples of lstep, so
    // the unit keys its state by line / lstep (dense ids, small line tables)
    const bool lcomp = (it.lsh >> 18) & 1u;
    const uint32_t lstep = lcomp ? it.gsets : 1u;
    const uint32_t sets = it.sets, mm = it.magic_m, s1 = it.s1, s2 = it.s2;
    const bool split = it.kcnt > 1;
    const uint32_t gT = it.gsets, gm = it.gmagic, gs1 = it.gs1, gs2 = it.gs2;
    auto set_of = [&](uint32_t l) -> uint32_t {
        if (uneq) {
            const uint32_t r = l - div_q(l, gm, gs1, gs2) * gT;
            return r < uta ? r - div_q(r, mm, s1, s2) * sets : 0u;
        }
        return l - div_q(l, mm, s1, s2) * sets;
    };
    const uint32_t psh = it.psh, K = it.kcnt, kres = it.kres;
    const uint32_t km = it.kmagic, ks1 = it.ks1, ks2 = it.ks2;
    const uint32_t pmask = (1u << psh) - 1u;
    const uint32_t warmup = it.warmup;
    const uint32_t lt = lanemask_lt();
    const bool ham = out.dist != nullptr;
    const uint32_t *const observed = out.observed;
    const uint64_t stop_above = out.stop_above;
    uint32_t *const bm = out.bitmaps
        ? out.bitmaps + (out.word_offsets ? out.word_offsets[it.out_item] : it.word_off)
        : nullptr;
    const uint64_t obase = ham ? out.obs_word_offsets[it.obs] : 0;

    uint32_t tot = 0, aft = 0, bad = 0;
    uint64_t dsum = 0;  // Hamming distance so far (warp-uniform)

    // analytic chain: access t visits (t * stride) mod N
    uint32_t aj = 0, ainc = 0;
    if (!idxp && N) {
        aj = (uint32_t)(((uint64_t)lane * it.stride) % N);
        ainc = (uint32_t)((32ull * it.stride) % N);
    }
    if (it.direct == 2 && out.parts) {
        // ---- a part of an item split by sets: its heads come gathered, in
        // trace order, from its head stream; a step takes the next 32 of them
        // (the grouping a queued unit's steps have), four steps' entries in flight
        const PartInfo pi = out.parts[out.item_slot[it.out_item] + it.kres];
        const uint2 *const es = out.ents + pi.start;
        const uint32_t n = pi.len;
        const uint2 none = make_uint2(kInvalidLine, 0u);
        uint2 ef[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            ef[q] = (uint32_t)lane + 32u * q < n ? es[lane + 32 * q] : none;
        uint32_t ccarry = kInvalidLine, step = 0;
        for (uint32_t b = 0; b < n; b += 32) {
            const uint2 e = ef[0];
            ef[0] = ef[1];
            ef[1] = ef[2];
            ef[2] = ef[3];
            const uint32_t nx = b + 128u + (uint32_t)lane;
            ef[3] = nx < n ? es[nx] : none;
            const bool act = b + (uint32_t)lane < n;
            const uint32_t line = e.x, pos = e.y;
            const uint32_t set = set_of(line * lstep);
            const uint32_t rot = __shfl_sync(kFull, line, (lane + 31) & 31);
            const uint32_t prev = lane == 0 ? ccarry : rot;
            ccarry = rot;
            const bool head = act && line != prev;
            ++step;
            const bool miss = res.resolve(line, set, head, pos, lane, lt, step);
            const uint32_t bits = __ballot_sync(kFull, miss);
            tot += __popc(bits);
            aft += __popc(__ballot_sync(kFull, miss && pos >= warmup));
            if (bm && bits) emit_bits(bm, pos, miss, act, lane);
        }
    } else if (it.direct == 1) {
        // ---- direct: nearly every access is a head, so each step takes 32
        // consecutive accesses as they come (repeats ride along as hits) and
        // the unit, sole writer of its words, stores 32 steps' words at once
        const uint32_t nsteps = (len + 31) >> 5;
        // a time part of an LRU item (whole sets, ks1 = 1) runs steps
        // [kres, kmagic) only, from the set state its first access sees
        const bool tpart = K == 1 && ks1 != 0 && kind == kBatchLru;
        const uint32_t sfirst = tpart ? min(kres, nsteps) : 0u;
        const uint32_t send = tpart ? min(km, nsteps) : nsteps;
        uint32_t carry = kInvalidLine, myword = 0;
        if (sfirst && sfirst < send) {
            // index of access t, and its line as the steps see it
            auto index_at = [&](uint32_t t) -> uint32_t {
                return idxp ? idxp[t] : (N ? (uint32_t)(((uint64_t)t * it.stride) % N) : 0u);
            };
            auto line_of = [&](uint32_t j) -> uint32_t {
                const uint32_t ln = j >> lsh;
                if (lcomp) return div_q(ln, gm, gs1, gs2);
                return mk ? remap_line(ln, mk, gT, gm, gs1, gs2) : ln;
            };
            BatchLRU S;
            S.bind(st, it);
            // the census of the item's sets, when the run took one
            const uint32_t *tgt = nullptr;
            if (out.targets && out.item_slot) {
                const uint32_t sl = out.item_slot[it.out_item];
                if (sl != 0xFFFFFFFFu) tgt = out.targets + out.parts[sl].start;
            }
            S.rebuild(sfirst << 5, sets, lane, lt, [&](uint32_t t) -> uint32_t {
                const uint32_t j = index_at(t);
                return j < N ? line_of(j) : kInvalidLine;
            }, tgt);
            carry = line_of(index_at((sfirst << 5) - 1));
            if (!idxp && N)
                aj = (uint32_t)((((uint64_t)(sfirst << 5) + (uint32_t)lane) * it.stride) % N);
        }
        // the trace is read four steps ahead (a step is about one memory
        // latency, so a unit's chain of steps would otherwise wait on each load)
        const uint32_t t1 = (sfirst << 5) + (uint32_t)lane;
        uint32_t pf[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            pf[q] = (idxp && t1 + 32u * q < len) ? idxp[t1 + 32u * q] : 0u;
        // matcher: the observed word of the step, loaded one step ahead
        uint32_t pw = (ham && len) ? observed[obase + sfirst] : 0u;
        for (uint32_t s0 = sfirst; s0 < send; ++s0) {
            const uint32_t t = (s0 << 5) + (uint32_t)lane;
            bool active = t < len;
            uint32_t j;
            if (idxp) {
                j = pf[0];
                pf[0] = pf[1];
                pf[1] = pf[2];
                pf[2] = pf[3];
                const uint32_t tn = t + 128;
                pf[3] = tn < len ? idxp[tn] : 0u;
            } else {
                j = aj;
                aj = (aj >= N - ainc) ? aj - (N - ainc) : aj + ainc;
            }
            if (active && j >= N) {
                bad = 1;
                active = false;
            }
            uint32_t ln = j >> lsh;
            if (mk) ln = remap_line(ln, mk, gT, gm, gs1, gs2);
            const uint32_t set = set_of(ln);
            if (lcomp) ln = div_q(ln, gm, gs1, gs2);
            const uint32_t rot = __shfl_sync(kFull, ln, (lane + 31) & 31);
            const uint32_t prev = lane == 0 ? carry : rot;
            carry = rot;
            const bool head = active && ln != prev;
            const bool miss = res.resolve(ln, set, head, t, lane, lt, s0 + 1);
            const uint32_t bits = __ballot_sync(kFull, miss);
            const uint32_t base = s0 << 5;
            const uint32_t after = base >= warmup ? kFull
                                 : (warmup - base >= 32 ? 0u : ~((1u << (warmup - base)) - 1u));
            tot += __popc(bits);
            aft += __popc(bits & after);
            if (ham) {
                // every step: its 32 outcomes against the observed word
                const uint32_t ow = pw;
                pw = s0 + 1 < nsteps ? observed[obase + s0 + 1] : 0u;
                const uint32_t valid = len - base >= 32 ? kFull : ((1u << (len - base)) - 1u);
                dsum += __popc((bits ^ ow) & valid);
                if (dsum > stop_above) break;
                if ((s0 & 31) == 31 && over_bound(out, it.cand, dsum, lane)) break;
                continue;
            }
            const uint32_t slot = s0 & 31;
            if ((uint32_t)lane == slot) myword = bits;
            if (slot == 31 || s0 + 1 == send) {
                const uint32_t w0 = s0 & ~31u;
                if ((uint32_t)lane <= slot && bm) bm[w0 + lane] = myword;
                myword = 0;
            }
        }
    } else {
        uint32_t qw = 0, qr = 0;         // queue entries written / read (warp-uniform)
        uint32_t ocarry = kInvalidLine;  // line of the access before the next chunk
        uint32_t ccarry = kInvalidLine;  // local line of the last head handed out
        uint32_t step = 0;
        // staging ring: chunk c (32 accesses) lands in ring[c % kRing][lane],
        // its observed word in oring[c % kRing]; kRing - 1 chunks in flight.
        // Each lane reads back only what it copied itself.
        uint32_t *const ring = reinterpret_cast<uint32_t *>(g_smem + arena + kQueueBytes);
        uint32_t *const oring = ring + kRing * 32;
        const uint32_t nchunks = (len + 31) >> 5;
        // a lower level of a hierarchy: a filter word per chunk (in the slot
        // the matcher uses for observed words; the two never meet)
        const uint32_t *const fbits =
            out.filter ? out.filter + out.filter_word_offsets[it.out_item] : nullptr;
        auto issue = [&](uint32_t c) {
            if (c < nchunks) {
                const uint32_t t = (c << 5) + (uint32_t)lane;
                if (idxp && t < len) cp_async4(ring + (c % kRing) * 32 + lane, idxp + t);
                if (ham && lane == 0) cp_async4(oring + (c % kRing), observed + obase + c);
                if (fbits && lane == 0) cp_async4(oring + (c % kRing), fbits + c);
            }
            cp_async_commit();
        };
        for (uint32_t c = 0; c + 1 < kRing; ++c) issue(c);
        uint32_t cin = 0;  // next chunk to gather

        for (;;) {
            if (qw - qr < 32 && cin < nchunks) {
                // ---- gather one chunk (at most 31 + 32 entries queued)
                issue(cin + kRing - 1);
                cp_async_wait<kRing - 1>();
                const uint32_t t = (cin << 5) + (uint32_t)lane;
                bool valid = t < len;
                uint32_t j;
                if (idxp) {
                    j = ring[(cin % kRing) * 32 + lane];
                } else {
                    j = aj;
                    aj = (aj >= N - ainc) ? aj - (N - ainc) : aj + ainc;
                }
                const uint32_t ow =
                    ham ? __shfl_sync(kFull, lane == 0 ? oring[cin % kRing] : 0u, 0) : 0u;
                if (valid && j >= N) {
                    bad = 1;
                    valid = false;
                }
                uint32_t ln = j >> lsh;
                if (mk) ln = remap_line(ln, mk, gT, gm, gs1, gs2);
                // one rotate: lane i gets lane i-1's line; lane 0 gets lane
                // 31's, the previous access of the next chunk's lane 0
                const uint32_t rot = __shfl_sync(kFull, ln, (lane + 31) & 31);
                const uint32_t prevl = lane == 0 ? ocarry : rot;
                ocarry = rot;
                bool mine = valid;
                uint32_t lp = lcomp ? div_q(ln, gm, gs1, gs2) : ln;
                if (split) {
                    const uint32_t q = div_q(ln, gm, gs1, gs2);
                    const uint32_t set = ln - q * gT;
                    const uint32_t sg = set >> psh;
                    const uint32_t kq = div_q(sg, km, ks1, ks2);
                    mine = valid && sg - kq * K == kres;
                    lp = ((kq << psh) | (set & pmask)) + q * sets;
                }
                // filtered: every kept access is queued (its predecessor in the
                // kept stream is not known here; the step drops repeats itself)
                const uint32_t fw =
                    fbits ? __shfl_sync(kFull, lane == 0 ? oring[cin % kRing] : 0u, 0) : kFull;
                const bool take =
                    mine && ((fw >> lane) & 1u) && (fbits != nullptr || ln != prevl);
                const uint32_t bal = __ballot_sync(kFull, take);
                if (take) {
                    const uint32_t pv = ham ? (t | (((ow >> lane) & 1u) << 31)) : t;
                    queue[(qw + __popc(bal & lt)) & (kQueueEntries - 1)] = make_uint2(lp, pv);
                }
                qw += __popc(bal);
                if (ham) {
                    // dropped repeats hit: they differ where a miss was observed
                    const uint32_t rep = __ballot_sync(kFull, mine && !take);
                    dsum += __popc(rep & ow);
                }
                ++cin;
                continue;
            }
            const uint32_t avail = qw - qr;
            if (avail == 0) break;
            // ---- one step over the next (up to) 32 heads
            __syncwarp();
            const bool act = (uint32_t)lane < avail;
            const uint2 e = act ? queue[(qr + (uint32_t)lane) & (kQueueEntries - 1)]
                                : make_uint2(kInvalidLine, 0u);
            qr += avail < 32 ? avail : 32u;
            __syncwarp();
            const uint32_t line = e.x;
            const uint32_t pos = e.y & 0x7FFFFFFFu;
            const uint32_t set = set_of(line * lstep);
            const uint32_t rot = __shfl_sync(kFull, line, (lane + 31) & 31);
            const uint32_t prev = lane == 0 ? ccarry : rot;
            ccarry = rot;
            const bool head = act && line != prev;
            ++step;
            const bool miss = res.resolve(line, set, head, pos, lane, lt, step);
            const uint32_t bits = __ballot_sync(kFull, miss);
            tot += __popc(bits);
            aft += __popc(__ballot_sync(kFull, miss && pos >= warmup));
            if (ham) {
                dsum += __popc(__ballot_sync(kFull, act && miss != ((e.y >> 31) != 0)));
                if (dsum > stop_above) break;
                if ((step & 31) == 0 && over_bound(out, it.cand, dsum, lane)) break;
            } else if (bm && bits) {
                emit_bits(bm, pos, miss, act, lane);
            }
        }
        // copies still in flight (an early stop) must land before the arena
        // is handed to the next unit
        cp_async_wait_all();
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(out.status, PCHASE_DEV_INDEX_RANGE);
    if (lane == 0) {
        if (ham) {
            if (dsum)
                atomicAdd(reinterpret_cast<unsigned long long *>(out.dist + it.cand),
                          (unsigned long long)dsum);
        } else if (out.miss_counts) {
            unsigned long long *mc =
                reinterpret_cast<unsigned long long *>(out.miss_counts + 2ull * it.out_item);
            if (tot) atomicAdd(mc, (unsigned long long)tot);
            if (aft) atomicAdd(mc + 1, (unsigned long long)aft);
        }
    }
}

// SPEC: one copy of the unit loop per set mode, chosen once per unit (the
// form for units that run alone on an SM); else AnyResolver's shared loop.
template <bool POOL, bool SPEC>
__device__ __forceinline__ void run_unit(const SimItem &it, uint32_t arena, const SimOut &out,
                                         int lane) {
    // arena: [queue + staging ring (units that compact their heads)][set state]
    uint8_t *const st = g_smem + arena + (it.direct == 1 ? 0u : kStageBytes);
    // WEIGHTED runs the RANDOM code with its own victim ways
    const uint32_t pol = it.policy < 2u ? it.policy : 2u;
    // set state in global memory (lsh bit 17): way scans at 16 * kres bytes
    // into the plan's state area, owned by this unit alone
    const bool gmem = POOL;  // the planner puts every global-state unit in the pool
    uint8_t *const gst = gmem ? out.gstate + 16ull * it.kres : nullptr;
    const uint32_t kind = gmem ? (uint32_t)kGlobalScanLru + pol : (uint32_t)it.mode * 3u + pol;
    // matcher: a candidate whose other units already exceed the bound is out
    if (out.dist && over_bound(out, it.cand, 0, lane)) return;
    clear_state<POOL>(kind, st, gst, it, lane);
    __syncwarp();
    if constexpr (!SPEC) {
        return run_steps<AnyResolver<POOL>>(it, arena, st, POOL ? gst : st, kind, out, lane);
    }
    // one dispatch per unit: every step then calls its resolver directly
    if constexpr (POOL) {
        switch (kind) {
        case kGlobalScanLru:
            return run_steps<RoundResolver<ScanSets<PCHASE_LRU>>>(it, arena, st, gst, kind, out, lane);
        case kGlobalScanFifo:
            return run_steps<RoundResolver<ScanSets<PCHASE_FIFO>>>(it, arena, st, gst, kind, out, lane);
        default:
            return run_steps<RoundResolver<ScanSets<PCHASE_RANDOM>>>(it, arena, st, gst, kind, out, lane);
        }
    }
    switch (kind) {
    case kScanLru:
        return run_steps<RoundResolver<ScanSets<PCHASE_LRU>>>(it, arena, st, st, kind, out, lane);
    case kScanFifo:
        return run_steps<RoundResolver<ScanSets<PCHASE_FIFO>>>(it, arena, st, st, kind, out, lane);
    case kScanRandom:
        return run_steps<RoundResolver<ScanSets<PCHASE_RANDOM>>>(it, arena, st, st, kind, out, lane);
    case kTableLru:
        return run_steps<RoundResolver<TableSets<PCHASE_LRU>>>(it, arena, st, st, kind, out, lane);
    case kTableFifo:
        return run_steps<RoundResolver<TableSets<PCHASE_FIFO>>>(it, arena, st, st, kind, out, lane);
    case kTableRandom:
        return run_steps<RoundResolver<TableSets<PCHASE_RANDOM>>>(it, arena, st, st, kind, out, lane);
    case kBatchLru:
        return run_steps<BatchLRU>(it, arena, st, st, kind, out, lane);
    case kBatchFifo:
        return run_steps<BatchFR<PCHASE_FIFO>>(it, arena, st, st, kind, out, lane);
    default:
        return run_steps<BatchFR<PCHASE_RANDOM>>(it, arena, st, st, kind, out, lane);
    }
}

template <bool POOL, bool SPEC>
__global__ void __launch_bounds__(512) sim_kernel(const SimItem *__restrict__ items,
                                                  const __grid_constant__ SlotLayout L,
                                                  uint32_t *queues, SimOut out) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t arena = L.warp_off[warp];
    const uint32_t top = L.warp_class[warp];
    // class this lane watches (pad + lane <= top), in every group
    const uint32_t wc = L.pad + (uint32_t)lane;
    const bool watch = wc <= top && wc < L.nclasses;
    const uint32_t nrep = out.n_rep ? out.n_rep : 1u;
    const bool prune = out.dist != nullptr && out.stop_above != ~0ull;
    // this warp's group: the CTA's home group with affinity, else none
    uint32_t grp = kUnitGroups;
    if (L.affinity) {
        const uint32_t site = blockIdx.x % L.home_mod;
        grp = 0;
        while (grp + 1 < (uint32_t)kUnitGroups && site >= L.home_end[grp]) ++grp;
    }
    // the cost of the next unit of (g, this lane's class) as an ordered key, 0: none
    auto head_key = [&](uint32_t g) -> uint32_t {
        if (!watch) return 0u;
        const uint32_t h = *reinterpret_cast<volatile uint32_t *>(queues + g * kQueueStride + wc);
        return h < L.cls_count[g][wc] * nrep
                   ? __float_as_uint(fmaxf(items[L.cls_first[g][wc] + h / nrep].cost, 1.0f))
                   : 0u;
    };
    // First pops staggered by slot (up to 4 us apart, a bounded sleep; the
    // planner scales it to the plan's longest unit): slot 0 of every CTA,
    // which holds every class, takes the costliest units first, one per SM,
    // instead of whichever SM's warps reach the queues first taking several
    // of the long units side by side.
    if (warp > 0 && L.stagger_ns) __nanosleep(L.stagger_ns * (uint32_t)warp);
    for (;;) {
        // longest first: the class whose next unit costs most, in this warp's
        // group while it has one for this slot, else in any group
        uint32_t key = 0, kg = grp;
        if (grp < (uint32_t)kUnitGroups) key = head_key(grp);
        uint32_t kmax = __reduce_max_sync(kFull, key);
        if (kmax == 0) {
            for (uint32_t g = 0; g < (uint32_t)kUnitGroups; ++g) {
                const uint32_t k = head_key(g);
                if (k > key) {
                    key = k;
                    kg = g;
                }
            }
            kmax = __reduce_max_sync(kFull, key);
            if (kmax == 0) break;  // every class this slot can hold is done
        }
        const int src = __ffs(__ballot_sync(kFull, key == kmax)) - 1;
        const uint32_t g = __shfl_sync(kFull, kg, src);
        if (L.affinity) grp = g;
        const uint32_t c = L.pad + (uint32_t)src;
        const uint32_t cfirst = L.cls_first[g][c];
        const uint32_t cper = L.cls_count[g][c];
        const uint32_t total = cper * nrep;
        uint32_t *const queue = queues + g * kQueueStride + c;
        // matcher with a bound over several observations: take up to 32 queue
        // entries at once (unit-major, so one unit for up to 32 observations),
        // screen them against their candidates' distances in parallel and run
        // only the survivors (most entries belong to candidates already out)
        const uint32_t grab = prune ? (nrep < 32u ? nrep : 32u) : 1u;
        uint32_t k0 = 0;
        if (lane == src) k0 = atomicAdd(queue, grab);
        k0 = __shfl_sync(kFull, k0, src);
        if (k0 >= total) continue;  // taken meanwhile: look again
        uint32_t todo = 1u;
        if (prune) {
            const uint32_t kk = k0 + (uint32_t)lane;
            bool alive = false;
            if (lane < (int)grab && kk < total) {
                const uint32_t uu = kk / nrep, rr = kk - uu * nrep;
                const uint32_t cand = items[cfirst + uu].cand;
                const unsigned long long d = *reinterpret_cast<volatile const unsigned long long *>(
                    out.dist + rr * out.rep_dist_stride + cand);
                alive = d <= out.stop_above;
            }
            todo = __ballot_sync(kFull, alive);
        }
        while (todo) {
            const uint32_t k = k0 + (uint32_t)(__ffs(todo) - 1);
            todo &= todo - 1;
            // unit-major: each unit runs for every observation in turn, so the
            // costliest (most discriminating) units come first for all of them
            const uint32_t u = k / nrep, rep = k - u * nrep;
            const SimItem it = items[cfirst + u];
            SimOut o = out;
            if (L.pool16)  // global set state: this warp's region of the pool
                o.gstate = out.gstate + ((uint64_t)blockIdx.x * L.nwarps + (uint32_t)warp) *
                                            ((uint64_t)L.pool16 << 4);
            if (rep) {
                o.dist += rep * out.rep_dist_stride;
                o.observed += rep * out.rep_obs_stride;
            }
            uint64_t t_start = 0;
            if (out.timeline) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
            run_unit<POOL, SPEC>(it, arena, o, lane);
            __syncwarp();
            if (out.timeline && lane == 0) {
                // units of a split item share the entry: first start, last end
                uint64_t t_end;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
                uint32_t smid;
                asm("mov.u32 %0, %%smid;" : "=r"(smid));
                unsigned long long *tl =
                    reinterpret_cast<unsigned long long *>(out.timeline + 4ull * it.out_item);
                atomicMin(tl, (unsigned long long)t_start);
                const unsigned long long prev_end = atomicMax(tl + 1, (unsigned long long)t_end);
                if (prev_end <= t_end) {
                    tl[2] = smid;
                    tl[3] = (unsigned long long)warp;
                }
            }
        }
    }
}

// One warp per unit; the lead unit of each caller item clears its outputs.
__global__ void __launch_bounds__(256) sim_zero_kernel(const SimItem *__restrict__ items,
                                                       uint64_t n_units, SimOut out) {
    const int lane = threadIdx.x & 31;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_units;
         i += nw) {
        const SimItem &it = items[i];
        if (!it.lead) continue;
        const uint32_t item = it.out_item;
        if (out.bitmaps) {
            uint32_t *bm = out.bitmaps + (out.word_offsets ? out.word_offsets[item] : it.word_off);
            const uint32_t nwords = (it.len + 31) >> 5;
            for (uint32_t k = (uint32_t)lane; k < nwords; k += 32) bm[k] = 0;
        }
        if (out.miss_counts && lane < 2) out.miss_counts[2ull * item + lane] = 0;
        if (out.timeline && lane < 4) out.timeline[4ull * item + lane] = lane == 0 ? ~0ull : 0ull;
    }
}

}  // namespace

cudaError_t launch_sim(const SimItem *items, const SlotLayout &layout, uint32_t *queues, int grid,
                       const SimOut &out, cudaStream_t st) {
    // the pool's layout (pool16 set) runs the global-state instantiation; a
    // layout with spec set, the per-mode unit loops
    const auto k = layout.pool16 ? sim_kernel<true, false>
                                 : layout.spec ? sim_kernel<false, true> : sim_kernel<false, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)layout.smem_bytes);
    if (e != cudaSuccess) return e;
    k<<<grid, layout.nwarps * 32, layout.smem_bytes, st>>>(items, layout, queues, out);
    return cudaGetLastError();
}

cudaError_t launch_sim_zero(const SimItem *items, uint64_t n_units, int sms, const SimOut &out,
                            cudaStream_t st) {
    if (!n_units || !(out.bitmaps || out.miss_counts || out.timeline)) return cudaSuccess;
    const uint64_t blocks = std::min<uint64_t>((n_units + 7) / 8, (uint64_t)std::max(sms, 1) * 8);
    sim_zero_kernel<<<(unsigned)blocks, 256, 0, st>>>(items, n_units, out);
    return cudaGetLastError();
}

int sim_max_ctas_per_sm(const SlotLayout &layout) {
    const auto k = layout.spec ? sim_kernel<false, true> : sim_kernel<false, false>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)layout.smem_bytes) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, layout.nwarps * 32,
                                                      layout.smem_bytes) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace pchase
