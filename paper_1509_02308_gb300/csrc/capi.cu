// C ABI entry points (include/pchase.h): argument checks, the simulation
// planner, workspace layout, and launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pchase_internal.cuh"

namespace pchase {
cudaError_t build_uniform(uint32_t n, uint32_t s, uint64_t len, uint32_t *trace,
                          uint32_t *array_out, cudaStream_t st, int sms);
cudaError_t build_chain(const uint32_t *next, uint32_t n, uint64_t len, uint32_t *trace,
                        uint32_t *status, cudaStream_t st);
cudaError_t build_uniform_batch(const pchase_trace *traces, uint32_t count, uint32_t *out,
                                const uint64_t *offsets, cudaStream_t st);
size_t classify_meta_bytes(uint32_t n_obs);
size_t classify_bucket_bytes(uint32_t n_obs, uint64_t max_len);
cudaError_t classify_thresholds(const float *lat, const uint64_t *offsets, uint32_t n_obs,
                                uint64_t max_len, void *meta_mem, void *bucket_mem,
                                float *thresh_out, cudaStream_t st, int sms);
cudaError_t classify_bits(const float *lat, const uint64_t *seg_offsets, int per_seg,
                          uint32_t n_seg, uint64_t max_seg_len, const void *meta_mem,
                          uint32_t *bits, const uint64_t *word_offsets, cudaStream_t st, int sms);
cudaError_t canonical_pick(const pchase_geom *geoms, const uint64_t *dist, uint32_t n,
                           uint32_t *pick, cudaStream_t st, uint32_t n_obs = 1);
cudaError_t batch_offsets(const uint64_t *seg, const uint64_t *owo, uint32_t T, uint32_t n_obs,
                          uint64_t L, uint64_t obs_words, uint64_t *obs_off, uint64_t *seg_out,
                          uint64_t *wo_out, cudaStream_t st);
cudaError_t probe_latency(const uint32_t *A, uint32_t n, uint32_t start, uint32_t warmup,
                          uint32_t iters, int mode, uint32_t *lat, uint32_t *idx, uint32_t *ovh,
                          uint32_t *status, cudaStream_t st);
cudaError_t probe_smem(uint32_t max_stride, uint32_t repeats, float *cycles, uint32_t *degree,
                       cudaStream_t st);
cudaError_t probe_smem_copy(uint32_t ctas, uint32_t threads, uint32_t ilp, uint32_t iters,
                            unsigned long long *t0, unsigned long long *t1, uint32_t *smid,
                            cudaStream_t st);
cudaError_t probe_gmem(int kind, uint32_t vec_bytes, uint32_t ctas, uint32_t threads,
                       uint32_t ilp, const void *src, void *dst, uint64_t bytes, uint32_t reps,
                       double *gbs, cudaStream_t st);
}  // namespace pchase

using namespace pchase;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    g_err = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return PCHASE_ECUDA;
}

#define PCHASE_CUDA(call, where)                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

bool is_pow2(uint32_t x) { return x && !(x & (x - 1)); }

uint32_t ilog2(uint32_t x) {
    uint32_t l = 0;
    while ((1u << l) < x) ++l;
    return l;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

constexpr uint32_t kMaxLines = 1u << 24;  // with the set state in global memory above 227 KB
constexpr uint32_t kMaxBatchObs = 1024;  // observations per infer_geometry_batch call
constexpr uint32_t kMaxArena = 232448;  // 227 KB, one warp per CTA
// size classes of unit arenas (bytes; queued units add their queue and staging ring)
const uint32_t kCaps[] = {1024,  2560,  3072,  4096,   5120,   6144,   8192,   10240,  12288,
                          16384, 20480, 24576, 32768,  40960,  49152,  65536,  81920,
                          98304, 112640, 131072, 163840, 196608, kMaxArena};

// Planner cost model: ns of one warp on GB300 with the SM fully loaded, fitted
// to per-item times of the batched workload.  A step in each set mode (batch
// by policy; scan and table plus a cost per extra round of same-set heads),
// and the gather of every 32 trace accesses a queued unit reads.
// per policy: LRU, FIFO, RANDOM
constexpr double kStepBatchNs[3] = {1900.0, 1660.0, 1780.0};
constexpr double kStepScanNs[3] = {765.0, 770.0, 845.0};
constexpr double kRoundScanNs[3] = {200.0, 200.0, 265.0};
constexpr double kStepTableNs[3] = {690.0, 635.0, 730.0};
constexpr double kRoundTableNs[3] = {130.0, 110.0, 160.0};
// A step whose heads are all held (every access hits): batch mode by policy,
// and table mode for FIFO / RANDOM, where such a hit changes nothing.
constexpr double kStepHeldBatchNs[3] = {630.0, 445.0, 450.0};
constexpr double kStepHeldTableNs = 435.0;
// A batch step whose sets are each all hits or all misses (LRU / FIFO over
// cyclic streams): FIFO, and LRU plus a cost per set in the step.
constexpr double kStepNoHitFifoNs = 1060.0;
constexpr double kStepNoHitLruNs = 900.0, kNoHitLruSetNs = 720.0;
constexpr double kGatherNs = 350.0;
// A step of a split part that reads its heads from its head stream instead
// (the entries' loads run two steps ahead; the streams' own pass is apart).
constexpr double kStreamStepNs = 20.0;
// Only items at least this long get head streams: below it the pass's own
// cost and the extra parts it invites outweigh the gathering it saves.
constexpr uint32_t kStreamMinLen = 1u << 18;
// SMs keep to one kind of unit only when the slot-mix launch holds at least
// this much estimated work per SM (ns): a short batch gains less from a warm
// instruction cache than it loses to the kinds' uneven shares of SMs.
constexpr double kAffinityMinNsPerSm = 20.0e6;
// The units that set a long plan's length run alone on an SM (the one-warp
// launch): the costliest kIsolateMax within kIsolateFrac of the costliest.
constexpr double kIsolateFrac = 0.6;
constexpr size_t kIsolateMax = 12;
// Way scans over set state in global memory (L2-resident) against shared memory.
constexpr double kGlobalScanFactor = 2.0;
// A time part's backward read of 32 accesses while it rebuilds the recency
// order: while lines are still being taken, and once every line read is taken
// or in a full set.
constexpr double kRebuildNs = 300.0, kRebuildSkipNs = 60.0;
constexpr double kBatchRounds = 6.0;   // this many rounds: batch mode whatever T'
constexpr double kPlanSms = 152.0;     // SMs the automatic split target assumes
// the global-state pool: warps of its launch (one state region each), their
// CTA width, and the most memory its regions take together
constexpr uint64_t kPoolMaxWarps = 608;
constexpr uint32_t kPoolWarpsPerCta = 4;
constexpr uint64_t kPoolMaxBytes = 16ull << 30;

// The tuning knobs as the planner reads them, and whether the plan's split
// parts read head streams (plans of explicit pairs that are not a lower level
// of a hierarchy; the matcher and filtered runs gather instead).
struct PlanTune : pchase_tune {
    bool streams = false;
};

// What the planner assumes about an item's access stream, from its trace's
// stride (exact for uniform chains, a hint for explicit traces).
struct ItemShape {
    double heads = 0.0;    // expected run heads (accesses that change line)
    double visited = 1.0;  // sets the stream visits
    uint32_t psh = 0;      // visited sets are multiples of 2^psh
    uint32_t groups = 1;   // T >> psh: the set groups a split divides among its parts
    bool held = false;     // no set ever receives more than a distinct lines
    bool cyclic = false;   // each set cycles through its lines in a fixed order every pass
    double cold = 0.0;     // accesses before every line has been touched
    double cost = 0.0;
    uint32_t lstep = 1;    // analytic chain visiting only the multiples of lstep lines:
                           // a whole unit keys its state by line / lstep (compact lines)
};

struct UnitShape {
    bool direct = false;  // steps over consecutive accesses, no queue
    uint32_t mode = 0, sets = 0, table_n = 0, ring = 0;
    uint64_t arena = 0;
    double cost = 0.0;
};

uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// The geometry's mapping field: bits 0-7 the shift m of set = (line >> m)
// mod T; bits 8-15 the extra ways of set 0 in a cache with unequal sets.
uint32_t map_shift(const pchase_geom &G) { return G.mapping & 255u; }
uint32_t extra_ways(const pchase_geom &G) { return (G.mapping >> 8) & 255u; }

// Largest line id a unit sees: (n_elems - 1) >> lsh, renumbered when the
// mapping takes the set from higher bits (id = ((hi << m) | lo) * T + set).
uint64_t top_line(const pchase_geom &G, uint32_t n_elems) {
    const uint64_t top = (uint64_t)(n_elems - 1) / (G.line_bytes / 4);
    const uint32_t m = map_shift(G);
    if (!m) return top;
    const uint64_t T = G.sets;
    return ((top >> m) / T + 1) * (T << m) - 1;
}

void item_shape(const pchase_geom &G, const pchase_trace &Tr, ItemShape &sh) {
    const uint64_t sb = 4ull * (Tr.stride % Tr.n_elems);  // bytes between accesses
    const uint64_t b = G.line_bytes;
    double density = 1.0;
    uint64_t delta = 1;  // lines between consecutive heads
    if (sb && sb < b) density = (double)sb / (double)b;
    else if (sb >= b && sb % b == 0) delta = sb / b;
    sh.heads = std::max(1.0, (double)Tr.len * density);
    const uint64_t T = G.sets;
    const uint64_t gfull = gcd64(delta % T ? delta % T : T, T);
    sh.visited = (double)(T / gfull);
    const uint64_t t2 = T & (~T + 1);
    const uint64_t g2 = gfull & (~gfull + 1);
    sh.psh = ilog2((uint32_t)std::min(g2, t2));
    sh.groups = (uint32_t)(T >> sh.psh);
    // Held steady state: when no set can receive more than a distinct lines,
    // nothing is ever evicted and every access after a line's first touch
    // hits.  Any trace touches lines 0..top only; a uniform chain touches the
    // multiples of g = gcd(N, s) once per pass of N / g accesses.
    // Cyclic: each pass visits every line of the stream once in the same
    // order (or in one ascending sweep).  A set receiving more than a lines
    // then has each line come back after at least a others of its set, so
    // under LRU and FIFO all its accesses miss; every other set holds its
    // lines.  Either way each set's heads are all hits or all misses.
    const uint64_t N = Tr.n_elems;
    const uint64_t top = (4ull * (N - 1)) / b;
    uint64_t per_set = (top + T) / T;
    uint64_t pass = N;
    const uint64_t se = Tr.stride % N;
    if (Tr.stride && !se) {
        // the chain never leaves element 0
        sh.heads = 1.0;
        per_set = 1;
        pass = 1;
    } else if (se) {
        const uint64_t g = gcd64(N, se);
        const uint64_t P = N / g;
        pass = P;
        const uint64_t gb = 4 * g;
        if (gb % b == 0) {
            const uint64_t dl = gb / b;  // lines k * dl, k < P, each once a pass
            const uint64_t V = T / gcd64(dl % T ? dl % T : T, T);
            per_set = std::min(per_set, (P + V - 1) / V);
            sh.visited = std::min(sh.visited, (double)std::min(V, P));
            sh.cyclic = true;
        } else if (b % gb == 0) {
            const uint64_t n = (4 * (N - g)) / b + 1;  // lines 0 .. n-1
            per_set = std::min(per_set, (n + T - 1) / T);
            sh.visited = std::min(sh.visited, (double)std::min(T, n));
            sh.cyclic = se == g;  // one ascending sweep a pass
        }
    }
    if (map_shift(G)) {
        // sets from higher line bits: only the bound over all line ids holds
        sh.visited = (double)T;
        sh.psh = 0;
        sh.groups = (uint32_t)T;
        sh.cyclic = false;
        per_set = (top_line(G, Tr.n_elems) + T) / T;
        if (Tr.stride && !se) per_set = 1;
    }
    sh.held = per_set <= G.ways;
    if (extra_ways(G)) {
        // unequal sets: no prediction, and no split (set 0 is unlike the rest)
        sh.visited = (double)T;
        sh.psh = 0;
        sh.groups = 1;
        sh.cyclic = false;
        sh.held = false;
    }
    sh.cold = std::min((double)Tr.len, (double)pass);
    // compact lines: an analytic chain (no index array to hold anything else)
    // with gcd(N, s) a whole number of lines visits only the lines k * lstep,
    // lstep = 4 gcd(N, s) / b; a whole unit numbers them k, so its line
    // table holds the chain's lines, not the array's
    if (!Tr.idx && se && !map_shift(G) && !extra_ways(G)) {
        const uint64_t gb = 4 * gcd64(N, se);
        if (gb % b == 0 && gb / b >= 2 && gb / b <= 0xFFFFFFFFull) sh.lstep = (uint32_t)(gb / b);
    }
}

// A whole unit of an item with compact lines keys its state by line / lstep.
void apply_compact(SimItem &it, const ItemShape &sh) {
    if (sh.lstep < 2) return;
    it.lsh |= 1u << 18;
    it.gsets = sh.lstep;
    const DivMagic dm = make_div_magic(sh.lstep);
    it.gmagic = dm.m;
    it.gs1 = (uint8_t)dm.s1;
    it.gs2 = (uint8_t)dm.s2;
}

// Bytes of set state of a whole way-scan unit: {line, stamp} per way slot,
// and RANDOM's eviction counters.
uint64_t scan_state_bytes(const pchase_geom &G) {
    const uint64_t T = G.sets, amax = G.ways + extra_ways(G);
    return align16(8 * T * amax + (G.policy >= PCHASE_RANDOM ? 4 * T : 0));
}

// A whole item whose set state fits no shared-memory arena: way scans with
// the state in global memory (only the queue and staging of a queued unit
// stay in shared memory).
void global_unit(const pchase_geom &G, const SimItem &it, const ItemShape &sh,
                 const PlanTune &tn, UnitShape &u) {
    const uint32_t amax = G.ways + extra_ways(G);
    const int pol = G.policy > PCHASE_RANDOM ? PCHASE_RANDOM : (int)G.policy;
    const double rounds = std::ceil(32.0 / std::min(32.0, std::max(1.0, sh.visited)));
    const double step_ns = (kStepScanNs[pol] + kRoundScanNs[pol] * (rounds - 1.0)) *
                           std::max(1.0, (double)amax / std::max(1u, tn.scan_max_ways)) *
                           kGlobalScanFactor;
    const double chunks = std::ceil((double)it.len / 32.0);
    const double steps = std::ceil(sh.heads / 32.0);
    const double direct_cost = chunks * step_ns;
    const double queued_cost = steps * step_ns + chunks * kGatherNs;
    u.direct = direct_cost <= queued_cost && !tn.filtered;
    u.mode = kModeScan;
    u.sets = G.sets;
    u.table_n = 0;
    u.ring = 0;
    u.arena = u.direct ? 0u : kStageBytes;
    u.cost = u.direct ? direct_cost : queued_cost;
}

// Set mode, arena and cost of one unit of a K-way split (K = 1: whole).
bool unit_shape(const pchase_geom &G, const SimItem &it, uint32_t K, const ItemShape &sh,
                const PlanTune &tn, UnitShape &u) {
    if (extra_ways(G)) {
        // unequal sets run as way scans (the mode that keeps a way count per
        // set), whole: T sets of a + extra way slots, set 0 using all of them
        if (K != 1) return false;
        const uint32_t T = G.sets, amax = G.ways + extra_ways(G);
        const int pol = (int)G.policy;
        const double rounds = std::ceil(32.0 / std::min(32.0, (double)T));
        const double step_ns = (kStepScanNs[pol] + kRoundScanNs[pol] * (rounds - 1.0)) *
                               std::max(1.0, (double)amax / std::max(1u, tn.scan_max_ways));
        const double chunks = std::ceil((double)it.len / 32.0);
        const double steps = std::ceil(sh.heads / 32.0);
        const double direct_cost = chunks * step_ns;
        const double queued_cost = steps * step_ns + chunks * kGatherNs;
        u.direct = direct_cost <= queued_cost && !tn.filtered;
        u.mode = kModeScan;
        u.sets = T;
        u.table_n = 0;
        u.ring = 0;
        u.arena = align16(8ull * T * amax) + (u.direct ? 0u : kStageBytes);
        u.cost = u.direct ? direct_cost : queued_cost;
        return u.arena <= kMaxArena;
    }
    const uint32_t T = G.sets, a = G.ways;
    const uint32_t Tl = T / K;
    const uint64_t lines = (uint64_t)Tl * a;
    uint64_t top = top_line(G, it.n_elems);  // largest line id
    if (K == 1 && sh.lstep > 1) top /= sh.lstep;  // compact lines
    const uint64_t table_n = K > 1 ? (uint64_t)Tl * (top / T + 1) : top + 1;
    const double parts = (double)K;
    const double vis = std::max(1.0, sh.visited / parts);
    const double rounds = std::ceil(32.0 / std::min(32.0, vis));
    const double steps = std::ceil(sh.heads / parts / 32.0);
    // LRU recency ring per set: compacted when more than R - 64 positions are
    // in use, so it holds a lines plus a step's 32 appends for R >= a + 64;
    // the slack above that sets how often it compacts (cyclic streams keep
    // their rings compact and never do)
    uint32_t ring = 128;
    while (ring < a + 96) ring <<= 1;
    uint64_t batch = 256 + 16ull * Tl + 2ull * table_n;
    // WEIGHTED runs the RANDOM code and costs like it
    const bool randomish = G.policy == PCHASE_RANDOM || G.policy == PCHASE_WEIGHTED;
    if (G.policy == PCHASE_LRU) batch += 4ull * Tl * ring;
    else batch += ((4 * lines + 15) & ~15ull) + (randomish ? 8 * lines : 0);
    batch = align16(batch);
    u.sets = Tl;
    u.table_n = (uint32_t)std::min<uint64_t>(table_n, 0xFFFFFFFFull);
    // candidates: batch mode (eligible for T' <= batch_max_sets, or when many
    // same-set heads per step make rounds costly, as long as the unit fits
    // one warp's arena) and the round-based scan / table mode; each
    // with its cost per step while lines are first touched (cold) and after
    // (a batch arena above half the CTA budget runs in the one-warp launch)
    const bool many_rounds = rounds >= kBatchRounds && kStageBytes + batch <= kMaxArena;
    const bool batch_ok = tn.batch_max_sets && (Tl <= tn.batch_max_sets || many_rounds) &&
                          kStageBytes + batch <= kMaxArena && ring <= 32768;
    const bool scan = a <= tn.scan_max_ways;
    const int pol = randomish ? PCHASE_RANDOM : (int)G.policy;
    struct Option {
        uint32_t mode, ring;
        uint64_t arena;
        double cold_ns, warm_ns;
    } opt[3];
    int n_opt = 0;
    if (batch_ok) {
        Option o{kModeBatch, ring, batch, kStepBatchNs[pol], kStepBatchNs[pol]};
        // held streams: steps after the first pass take the all-held path;
        // cyclic LRU / FIFO streams: every step takes the path for sets that
        // all hit or all miss
        if (sh.held) o.warm_ns = kStepHeldBatchNs[pol];
        if (sh.cyclic && !sh.held && pol != PCHASE_RANDOM) {
            const double sets_per_step = std::min(32.0, vis);
            if (pol == PCHASE_FIFO) o.cold_ns = o.warm_ns = kStepNoHitFifoNs;
            else if (sets_per_step <= 8.0)
                o.cold_ns = o.warm_ns = kStepNoHitLruNs + kNoHitLruSetNs * sets_per_step;
        }
        opt[n_opt++] = o;
    }
    {
        const double round_ns = scan ? kStepScanNs[pol] + kRoundScanNs[pol] * (rounds - 1.0)
                                     : kStepTableNs[pol] + kRoundTableNs[pol] * (rounds - 1.0);
        Option o{scan ? kModeScan : kModeTable, 0u,
                 scan ? 8 * lines + (randomish ? 4ull * Tl : 0)
                      : 8ull * Tl + 4 * lines + (G.policy == PCHASE_LRU ? 4 * lines : 0) +
                            2ull * table_n,
                 round_ns, round_ns};
        if (!scan && sh.held && pol != PCHASE_LRU) o.warm_ns = kStepHeldTableNs;
        opt[n_opt++] = o;
    }
    if (!scan) {
        // way scans keep no line table, so they fit streams over any line
        // range: the fallback when the table modes do not fit (a scan costs
        // in proportion to the ways past the ones the fit covers)
        const double f = std::max(1.0, (double)a / std::max(1u, tn.scan_max_ways));
        const double ns = (kStepScanNs[pol] + kRoundScanNs[pol] * (rounds - 1.0)) * f;
        opt[n_opt++] = Option{kModeScan, 0u, 8 * lines + (randomish ? 4ull * Tl : 0), ns, ns};
    }
    // a whole item steps over its accesses as they come (direct) when that
    // beats gathering and compacting its heads (queued); a split part always
    // queues its own sets' heads.  The cheapest option that fits is taken.
    const double chunks = std::ceil((double)it.len / 32.0);
    const double cold_chunks = std::min(chunks, std::ceil(sh.cold / 32.0) + 1.0);
    const double cold_frac = it.len ? std::min(1.0, sh.cold / (double)it.len) : 1.0;
    const double cold_steps = std::min(steps, std::ceil(steps * cold_frac) + 1.0);
    bool have = false;
    for (int k = 0; k < n_opt; ++k) {
        const Option &o = opt[k];
        const double direct_cost = cold_chunks * o.cold_ns + (chunks - cold_chunks) * o.warm_ns;
        const double gather = K > 1 && tn.streams && it.len >= kStreamMinLen
                                  ? steps * kStreamStepNs
                                  : chunks * kGatherNs;
        const double queued_cost = cold_steps * o.cold_ns + (steps - cold_steps) * o.warm_ns +
                                   gather;
        const bool direct = K == 1 && direct_cost <= queued_cost && !tn.filtered;
        const uint64_t arena = align16(o.arena) + (direct ? 0u : kStageBytes);
        const double cost = direct ? direct_cost : queued_cost;
        const bool fits = arena <= kMaxArena;
        // prefer options that fit; among those (or among none), the cheapest
        if (!have || (fits && u.arena > kMaxArena) ||
            ((fits || u.arena > kMaxArena) && cost < u.cost)) {
            u.mode = o.mode;
            u.ring = o.ring;
            u.direct = direct;
            u.arena = arena;
            u.cost = cost;
            have = true;
        }
    }
    return u.arena <= kMaxArena;
}

void apply_unit(SimItem &it, const UnitShape &u) {
    it.direct = u.direct ? 1 : 0;
    it.mode = (uint8_t)u.mode;
    it.sets = u.sets;
    const DivMagic dm = make_div_magic(u.sets);
    it.magic_m = dm.m;
    it.s1 = (uint8_t)dm.s1;
    it.s2 = (uint8_t)dm.s2;
    it.table_n = u.table_n;
    it.ring = u.ring;
    it.arena_bytes = (uint32_t)u.arena;
}

int check_geom(const pchase_geom &g, uint32_t i) {
    char buf[160];
    if (g.line_bytes < 4 || !is_pow2(g.line_bytes)) {
        snprintf(buf, sizeof buf, "geometry %u: line size %u is not a power of two >= 4", i,
                 g.line_bytes);
        return fail(PCHASE_EINVAL, buf);
    }
    const uint32_t m = map_shift(g), extra = extra_ways(g);
    const uint64_t lines = (uint64_t)g.sets * g.ways + extra;
    if (g.ways == 0 || g.sets == 0 || lines * g.line_bytes != (uint64_t)g.C_bytes) {
        snprintf(buf, sizeof buf, "geometry %u: (sets*ways + extra)*line ((%u*%u + %u)*%u) != C (%u)",
                 i, g.sets, g.ways, extra, g.line_bytes, g.C_bytes);
        return fail(PCHASE_EINVAL, buf);
    }
    if (g.policy > PCHASE_WEIGHTED || m > 16 || (uint64_t)g.sets << m > (1ull << 30) ||
        (g.mapping >> 16) != 0 || (g.policy == PCHASE_WEIGHTED && g.ways < 3)) {
        snprintf(buf, sizeof buf,
                 "geometry %u: unknown policy %u, mapping %u above 16 (or T << mapping above 2^30),"
                 " bits above 15 set, or WEIGHTED with fewer than 3 ways", i, g.policy, m);
        return fail(PCHASE_EINVAL, buf);
    }
    if (extra && (m != 0 || g.policy > PCHASE_FIFO)) {
        snprintf(buf, sizeof buf,
                 "geometry %u: unequal sets take LRU or FIFO and the plain mapping", i);
        return fail(PCHASE_EINVAL, buf);
    }
    if (lines > kMaxLines) {
        snprintf(buf, sizeof buf, "geometry %u: %llu lines is above the limit of %u", i,
                 (unsigned long long)lines, kMaxLines);
        return fail(PCHASE_ERANGE, buf);
    }
    return PCHASE_OK;
}

int check_trace(const pchase_trace &t, uint32_t i) {
    char buf[160];
    if (t.n_elems == 0) {
        snprintf(buf, sizeof buf, "trace %u: n_elems is 0", i);
        return fail(PCHASE_EINVAL, buf);
    }
    if (t.len >= (1ull << 31)) {
        snprintf(buf, sizeof buf, "trace %u: length %llu is not below 2^31", i,
                 (unsigned long long)t.len);
        return fail(PCHASE_ERANGE, buf);
    }
    return PCHASE_OK;
}

}  // namespace

int pchase::set_last_error(int code, const char *msg) { return fail(code, msg); }

struct pchase_sim_plan {
    std::vector<SimItem> items;
    SlotLayout layout{};
    SlotLayout jumbo{};   // items too large for the main slot mix (nwarps 0: none)
    SlotLayout gpool{};   // units with global set state, one pool region per warp
    uint32_t pool_warps = 0;    // warps (and state regions) of the pool launch
    uint64_t pool_region = 0;   // bytes of one region
    uint32_t jumbo_first_class = 0;
    uint64_t n_jumbo = 0;
    uint64_t bitmap_words = 0;
    uint64_t n_items = 0;  // caller's items
    uint64_t n_units = 0;  // units (items, or parts of split items)
    size_t ws_bytes = 0, off_items = 0, off_geoms = 0, off_seg = 0, off_obs_words = 0,
           off_pool = 0;
    bool cross = false;
    uint32_t n_geom = 0, n_trace = 0;
    std::vector<pchase_geom> geoms;
    std::vector<uint64_t> seg_offsets;     // n_trace + 1 (element offsets of trace latencies)
    std::vector<uint64_t> obs_word_offsets;  // n_trace
    uint64_t obs_words = 0, total_len = 0, max_trace_len = 0;
    // planner estimates (ns of one warp): all units, the longest unit that
    // cannot split further, the split target, the longest unit planned
    double est_sum = 0.0, est_critical = 0.0, est_target = 0.0, est_max_unit = 0.0;
    bool filtered = false;  // every unit queued (pchase_sim_run_filtered)
    // runtime state, set on the first run
    int device = -1, sms = 0, grid = 0, jgrid = 0, ggrid = 0;
    uint64_t n_isolated = 0;  // units given an SM of their own (in the jumbo launch)
    uint64_t n_gmem = 0;        // units with their set state in global memory
    uint64_t gstate_bytes = 0;  // their state area (workspace, after the pooled offsets)
    size_t off_gstate = 0;
    std::vector<uint32_t> class_caps;  // arena cap of each size class present
    // head streams of the split items (streams.cu): jobs, each segment's job,
    // each caller item's first part slot (or ~0), and the sizes of the count,
    // part and entry arrays
    std::vector<StreamJob> jobs;
    std::vector<uint32_t> seg_job, item_slot;
    uint64_t n_cnt = 0, n_ents = 0, n_tgt = 0;
    uint32_t n_slots = 0, n_census = 0;
    size_t off_jobs = 0, off_segjob = 0, off_itemslot = 0, off_cnt = 0, off_parts = 0,
           off_ents = 0, off_tgt = 0;
    double gwork_main[kUnitGroups] = {};  // estimated work of each unit group in the
                                          // slot-mix launch
    bool affinity = false;
    cudaStream_t side = nullptr, side2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, fork2 = nullptr, join2 = nullptr;

    ~pchase_sim_plan() {
        if (side) cudaStreamDestroy(side);
        if (side2) cudaStreamDestroy(side2);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (fork2) cudaEventDestroy(fork2);
        if (join2) cudaEventDestroy(join2);
    }
};

namespace {

// Unit-group homes of the slot-mix launch: `sites` SMs (CTA b sits on site
// b mod sites) shared among the groups with work in proportion to their
// estimated work, at least one each.  Affinity (and with it the per-kind
// unit loops) stays off with fewer than two groups, fewer sites than groups,
// or under kAffinityMinNsPerSm of work per site.
void set_homes(SlotLayout &L, const double *work, bool on, uint32_t sites) {
    // with affinity, the per-kind unit loops: an SM then holds few kinds' code
    L.spec = on ? 1u : 0u;
    L.affinity = 0;
    L.home_mod = sites;
    for (int g = 0; g < kUnitGroups; ++g) L.home_end[g] = sites;
    double total = 0.0;
    uint32_t with = 0;
    for (int g = 0; g < kUnitGroups; ++g)
        if (work[g] > 0.0) {
            total += work[g];
            ++with;
        }
    if (!on || with < 2 || sites < with || total < kAffinityMinNsPerSm * sites) {
        L.spec = 0;
        return;
    }
    uint32_t n[kUnitGroups] = {}, sum = 0;
    for (int g = 0; g < kUnitGroups; ++g)
        if (work[g] > 0.0) {
            n[g] = std::max<uint32_t>(1, (uint32_t)std::lround(sites * work[g] / total));
            sum += n[g];
        }
    while (sum > sites) {  // take from the group with the least work per site that can spare one
        int best = -1;
        for (int g = 0; g < kUnitGroups; ++g)
            if (n[g] > 1 && (best < 0 || work[g] / n[g] < work[best] / n[best])) best = g;
        --n[best];
        --sum;
    }
    while (sum < sites) {  // give to the group with the most work per site
        int best = -1;
        for (int g = 0; g < kUnitGroups; ++g)
            if (work[g] > 0.0 && (best < 0 || work[g] / n[g] > work[best] / n[best])) best = g;
        ++n[best];
        ++sum;
    }
    uint32_t end = 0;
    for (int g = 0; g < kUnitGroups; ++g) {
        end += n[g];
        L.home_end[g] = end;
    }
    L.affinity = 1;
}

int plan_runtime(pchase_sim_plan *p) {
    int dev = 0;
    PCHASE_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (p->device >= 0) {
        if (dev != p->device) return fail(PCHASE_EINVAL, "plan used on another device");
        return PCHASE_OK;
    }
    p->sms = sm_count();
    if (p->sms <= 0) return fail(PCHASE_ECUDA, "no CUDA device");
    // A CTA of either launch fills an SM's shared memory, so a main launch
    // started over every SM would hold them all.  A one-warp launch of a few
    // units (the isolated ones among them) gets an SM per unit, kept out of
    // the main grid; one of many units takes SMs as main CTAs leave.
    int jsms = 0;
    if (p->jumbo.nwarps && p->layout.nwarps && p->n_jumbo <= 32 &&
        (int)p->n_jumbo < p->sms / 2)
        jsms = (int)p->n_jumbo;
    if (p->layout.nwarps) {
        const int per = sim_max_ctas_per_sm(p->layout);
        if (per <= 0) return fail(PCHASE_ECUDA, "simulator kernel cannot be resident");
        p->grid = (int)std::max<uint64_t>(
            1, std::min<uint64_t>((uint64_t)per * (p->sms - jsms), p->n_units - p->n_jumbo));
        set_homes(p->layout, p->gwork_main, p->affinity,
                  (uint32_t)std::max(1, std::min(p->grid, p->sms - jsms)));
    }
    if (p->jumbo.nwarps) {
        const int per = sim_max_ctas_per_sm(p->jumbo);
        if (per <= 0) return fail(PCHASE_ECUDA, "simulator kernel cannot be resident");
        p->jgrid = (int)std::max<uint64_t>(
            1, std::min<uint64_t>((uint64_t)per * (jsms ? jsms : p->sms), p->n_jumbo));
        PCHASE_CUDA(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking), "cudaStreamCreate");
        PCHASE_CUDA(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming), "cudaEventCreate");
        PCHASE_CUDA(cudaEventCreateWithFlags(&p->join, cudaEventDisableTiming), "cudaEventCreate");
    }
    if (p->gpool.nwarps) {
        // the pool launch has exactly pool_warps warps: one state region each
        p->ggrid = (int)(p->pool_warps / p->gpool.nwarps);
        PCHASE_CUDA(cudaStreamCreateWithFlags(&p->side2, cudaStreamNonBlocking), "cudaStreamCreate");
        PCHASE_CUDA(cudaEventCreateWithFlags(&p->fork2, cudaEventDisableTiming), "cudaEventCreate");
        PCHASE_CUDA(cudaEventCreateWithFlags(&p->join2, cudaEventDisableTiming), "cudaEventCreate");
    }
    p->device = dev;
    return PCHASE_OK;
}

int plan_launch(pchase_sim_plan *p, void *ws, const SimOut &out, cudaStream_t st) {
    int rc = plan_runtime(p);
    if (rc) return rc;
    uint8_t *w = static_cast<uint8_t *>(ws);
    PCHASE_CUDA(cudaMemsetAsync(w, 0, kQueueHeader, st), "cudaMemsetAsync(queues)");
    SimOut o = out;
    if (!o.status) o.status = reinterpret_cast<uint32_t *>(w + kStatusOffset);
    o.gstate = w + p->off_gstate;
    const SimItem *items = reinterpret_cast<const SimItem *>(w + p->off_items);
    uint32_t *queues = reinterpret_cast<uint32_t *>(w);
    PCHASE_CUDA(launch_sim_zero(items, p->n_units, p->sms, o, st), "output clear");
    if (!p->jobs.empty() && !o.dist && !o.filter) {
        // the split parts' head streams, before any launch that reads them
        o.item_slot = reinterpret_cast<const uint32_t *>(w + p->off_itemslot);
        o.parts = reinterpret_cast<const PartInfo *>(w + p->off_parts);
        o.ents = reinterpret_cast<const uint2 *>(w + p->off_ents);
        o.targets = p->n_census ? reinterpret_cast<const uint32_t *>(w + p->off_tgt) : nullptr;
        // the census bitmaps start empty every run
        if (p->n_census)
            PCHASE_CUDA(cudaMemsetAsync(w + p->off_cnt, 0, p->n_cnt * sizeof(uint32_t), st),
                        "cudaMemsetAsync(census)");
        PCHASE_CUDA(launch_streams(items, reinterpret_cast<const StreamJob *>(w + p->off_jobs),
                                   (uint32_t)p->jobs.size(),
                                   reinterpret_cast<const uint32_t *>(w + p->off_segjob),
                                   (uint32_t)p->seg_job.size(),
                                   reinterpret_cast<uint32_t *>(w + p->off_cnt),
                                   reinterpret_cast<PartInfo *>(w + p->off_parts),
                                   reinterpret_cast<uint2 *>(w + p->off_ents),
                                   reinterpret_cast<uint32_t *>(w + p->off_tgt), o.status, st),
                    "head streams");
    }
    if (p->gpool.nwarps) {
        // units with global set state first (the longest of a hierarchy's
        // large levels), on a side stream of their own joined back below
        PCHASE_CUDA(cudaEventRecord(p->fork2, st), "cudaEventRecord");
        PCHASE_CUDA(cudaStreamWaitEvent(p->side2, p->fork2, 0), "cudaStreamWaitEvent");
        PCHASE_CUDA(launch_sim(items, p->gpool, queues, p->ggrid, o, p->side2), "pool launch");
        PCHASE_CUDA(cudaEventRecord(p->join2, p->side2), "cudaEventRecord");
    }
    if (p->jumbo.nwarps) {
        // jumbo items first, on a side stream joined back before returning
        PCHASE_CUDA(cudaEventRecord(p->fork, st), "cudaEventRecord");
        PCHASE_CUDA(cudaStreamWaitEvent(p->side, p->fork, 0), "cudaStreamWaitEvent");
        PCHASE_CUDA(launch_sim(items, p->jumbo, queues, p->jgrid, o, p->side), "jumbo launch");
        PCHASE_CUDA(cudaEventRecord(p->join, p->side), "cudaEventRecord");
    }
    if (p->layout.nwarps)
        PCHASE_CUDA(launch_sim(items, p->layout, queues, p->grid, o, st), "simulator launch");
    if (p->jumbo.nwarps) PCHASE_CUDA(cudaStreamWaitEvent(st, p->join, 0), "cudaStreamWaitEvent");
    if (p->gpool.nwarps) PCHASE_CUDA(cudaStreamWaitEvent(st, p->join2, 0), "cudaStreamWaitEvent");
    return PCHASE_OK;
}

}  // namespace

extern "C" {

const char *pchase_last_error_string(void) { return g_err.c_str(); }
const char *pchase_version(void) { return "pchase-gb300 0.1 (sm_103a)"; }
int pchase_device_sm_count(void) { return sm_count(); }

int pchase_build(uint32_t n_elems, uint32_t stride, const uint32_t *next, uint64_t len,
                 uint32_t *trace_out, uint32_t *array_out, uint32_t *dev_status,
                 pchase_stream_t stream) {
    if (n_elems == 0) return fail(PCHASE_EINVAL, "pchase_build: n_elems is 0");
    if (len && !trace_out) return fail(PCHASE_EINVAL, "pchase_build: trace_out is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (next) {
        if (!dev_status) return fail(PCHASE_EINVAL, "pchase_build: chain walk needs dev_status");
        PCHASE_CUDA(build_chain(next, n_elems, len, trace_out, dev_status, st), "chain walk");
        if (array_out) PCHASE_CUDA(build_uniform(n_elems, stride, 0, nullptr, array_out, st, sm_count()),
                                   "uniform array");
        return PCHASE_OK;
    }
    PCHASE_CUDA(build_uniform(n_elems, stride, len, trace_out, array_out, st, sm_count()),
                "uniform trace");
    return PCHASE_OK;
}

int pchase_build_batch(const pchase_trace *traces, uint32_t n, uint32_t *trace_out,
                       const uint64_t *word_offsets, pchase_stream_t stream) {
    if (n == 0) return PCHASE_OK;
    if (!traces || !trace_out || !word_offsets)
        return fail(PCHASE_EINVAL, "pchase_build_batch: NULL argument");
    for (uint32_t i = 0; i < n; ++i) {
        if (traces[i].n_elems == 0) return fail(PCHASE_EINVAL, "pchase_build_batch: n_elems is 0");
    }
    PCHASE_CUDA(build_uniform_batch(traces, n, trace_out, word_offsets,
                                    reinterpret_cast<cudaStream_t>(stream)),
                "batched uniform traces");
    return PCHASE_OK;
}

int pchase_sim_plan_create(const pchase_geom *geoms, uint32_t n_geom, const pchase_trace *traces,
                           uint32_t n_trace, const pchase_pair *pairs, uint32_t n_pairs,
                           const pchase_tune *tune, pchase_sim_plan **plan_out) {
    if (!plan_out) return fail(PCHASE_EINVAL, "plan_out is NULL");
    *plan_out = nullptr;
    if ((n_geom && !geoms) || (n_trace && !traces) || (n_pairs && !pairs))
        return fail(PCHASE_EINVAL, "NULL descriptor array");
    PlanTune tn;
    static_cast<pchase_tune &>(tn) =
        pchase_tune{4, 220 * 1024, 16, 0, 64, 32, 0, 0, (uint32_t)kPoolMaxWarps, 1, 1, 1};
    if (tune) {
        if (tune->batch_max_sets) tn.batch_max_sets = tune->batch_max_sets == 0xFFFFFFFFu ? 0 : tune->batch_max_sets;
        if (tune->scan_max_ways) tn.scan_max_ways = std::min<uint32_t>(tune->scan_max_ways, 32);
        if (tune->smem_budget_bytes) tn.smem_budget_bytes = std::min(tune->smem_budget_bytes, kMaxArena);
        if (tune->max_warps_per_cta)
            tn.max_warps_per_cta = std::min<uint32_t>(tune->max_warps_per_cta, kMaxWarpsPerCta);
        tn.ctas_per_sm_cap = tune->ctas_per_sm_cap;
        if (tune->max_split) tn.max_split = std::min<uint32_t>(tune->max_split, 192);
        tn.split_cost_ns = tune->split_cost_ns;
        tn.filtered = tune->filtered ? 1u : 0u;
        if (tune->pool_warps)
            tn.pool_warps = std::min<uint32_t>(tune->pool_warps, (uint32_t)kPoolMaxWarps);
        if (tune->big_slots) tn.big_slots = std::min<uint32_t>(tune->big_slots, 4);
        tn.kind_affinity = tune->kind_affinity == 0xFFFFFFFFu ? 0u : 1u;
        tn.head_streams = tune->head_streams == 0xFFFFFFFFu ? 0u : 1u;
    }
    tn.streams = pairs != nullptr && !tn.filtered && tn.head_streams;
    for (uint32_t i = 0; i < n_geom; ++i) {
        int rc = check_geom(geoms[i], i);
        if (rc) return rc;
    }
    for (uint32_t i = 0; i < n_trace; ++i) {
        int rc = check_trace(traces[i], i);
        if (rc) return rc;
    }
    auto *p = new (std::nothrow) pchase_sim_plan();
    if (!p) return fail(PCHASE_ENOMEM, "plan allocation");
    p->cross = pairs == nullptr;
    p->n_geom = n_geom;
    p->n_trace = n_trace;
    p->geoms.assign(geoms, geoms + n_geom);
    const uint64_t n_items = p->cross ? (uint64_t)n_geom * n_trace : n_pairs;
    if (n_items > 0xFFFFFFFFull) {
        delete p;
        return fail(PCHASE_ERANGE, "more than 2^32-1 items");
    }
    p->n_items = n_items;
    // per-trace layouts used by the matcher
    p->seg_offsets.resize(n_trace + 1, 0);
    p->obs_word_offsets.resize(n_trace, 0);
    for (uint32_t t = 0; t < n_trace; ++t) {
        p->seg_offsets[t + 1] = p->seg_offsets[t] + traces[t].len;
        p->obs_word_offsets[t] = p->obs_words;
        p->obs_words += (traces[t].len + 31) / 32;
        p->max_trace_len = std::max<uint64_t>(p->max_trace_len, traces[t].len);
    }
    p->total_len = p->seg_offsets[n_trace];

    // ---- items -> units.  Each item gets a base unit; a long one is split
    // by sets into 2^ksh units (see SimItem) so no unit dominates the launch.
    std::vector<SimItem> base;
    std::vector<ItemShape> shape;
    std::vector<uint8_t> gmem;      // set state in global memory
    std::vector<UnitShape> gshape;  // and its unit
    try {
        base.resize(n_items);
        shape.resize(n_items);
        gmem.assign(n_items, 0);
        gshape.resize(n_items);
    } catch (...) {
        delete p;
        return fail(PCHASE_ENOMEM, "item table allocation");
    }
    uint64_t word = 0;
    double total = 0.0;
    const uint32_t max_split = std::max<uint32_t>(1, tn.max_split);
    for (uint64_t i = 0; i < n_items; ++i) {
        uint32_t g, t;
        if (p->cross) {
            g = (uint32_t)(i / n_trace);
            t = (uint32_t)(i % n_trace);
        } else {
            g = pairs[i].geom;
            t = pairs[i].trace;
            if (g >= n_geom || t >= n_trace) {
                delete p;
                return fail(PCHASE_EINVAL, "pair refers to a missing geometry or trace");
            }
        }
        const pchase_geom &G = geoms[g];
        const pchase_trace &Tr = traces[t];
        SimItem &it = base[i];
        memset(&it, 0, sizeof it);
        it.idx = Tr.idx;
        it.len = (uint32_t)Tr.len;
        it.warmup = (uint32_t)std::min<uint64_t>(Tr.warmup, Tr.len);
        it.n_elems = Tr.n_elems;
        it.stride = Tr.stride % Tr.n_elems;
        it.ways = G.ways;
        it.policy = (uint8_t)G.policy;
        it.lsh = (ilog2(G.line_bytes) - 2) | (map_shift(G) << 8) |
                 (extra_ways(G) ? 1u << 16 : 0u);
        it.seed = G.seed;
        it.word_off = word;
        word += (Tr.len + 31) / 32;
        it.out_item = (uint32_t)i;
        it.cand = g;
        it.obs = t;
        it.gsets = G.sets;
        if (extra_ways(G)) {
            // unequal sets: M = T*a + extra residues, set 0 with a + extra ways
            it.gsets = G.sets * G.ways + extra_ways(G);
            it.ways = G.ways + extra_ways(G);
            it.kmagic = G.ways;
        }
        const DivMagic gdm = make_div_magic(it.gsets);
        it.gmagic = gdm.m;
        it.gs1 = (uint8_t)gdm.s1;
        it.gs2 = (uint8_t)gdm.s2;
        it.lead = 1;
        it.kcnt = 1;
        ItemShape &sh = shape[i];
        item_shape(G, Tr, sh);
        UnitShape u;
        if (!unit_shape(G, it, 1, sh, tn, u)) {
            // too much set state for one warp: some split into set-parts must fit
            uint64_t need = u.arena;
            bool fits = false;
            for (uint32_t K = 2; !fits && K <= max_split && K <= sh.groups && K <= sh.visited;
                 ++K) {
                const uint32_t odd = K % 3 == 0 ? K / 3 : K;
                if ((odd & (odd - 1)) != 0 || sh.groups % K != 0) continue;
                UnitShape uk;
                fits = unit_shape(G, it, K, sh, tn, uk);
                if (fits) u.cost = uk.cost * K;
                need = std::min(need, (uint64_t)uk.arena);
            }
            // no shared-memory arena holds it, even split, or every split
            // that does costs more warp time in all (each part re-reads the
            // whole trace): way scans over set state in global memory
            UnitShape gu;
            global_unit(G, it, sh, tn, gu);
            if (!fits || gu.cost < u.cost) {
                u = gu;
                gmem[i] = 1;
                gshape[i] = gu;
            }
        }
        sh.cost = u.cost;
        total += u.cost;
    }
    p->bitmap_words = word;
    p->filtered = tn.filtered != 0;
    // Split target: no unit above the plan's share per warp slot, but no
    // split below what the longest unsplittable work takes anyway (splitting
    // costs a gather pass per part and only the critical path gains).
    // parts of a split: K = 2^j or 3 * 2^j dividing the item's set groups
    auto best_split = [&](uint64_t i, double target, uint32_t &k_out, UnitShape &u_out) {
        const pchase_geom &G = geoms[base[i].cand];
        const ItemShape &sh = shape[i];
        // the whole item if it fits, else the first split that does
        k_out = 0;
        if (unit_shape(G, base[i], 1, sh, tn, u_out)) {
            k_out = 1;
            if (u_out.cost <= target) return;
        }
        for (uint32_t K = 2; K <= max_split && K <= sh.groups && K <= sh.visited; ++K) {
            const uint32_t odd = K % 3 == 0 ? K / 3 : K;
            if ((odd & (odd - 1)) != 0 || sh.groups % K != 0) continue;
            UnitShape u;
            if (!unit_shape(G, base[i], K, sh, tn, u)) continue;
            if (k_out == 0 || u.cost < u_out.cost * 0.97) {
                u_out = u;
                k_out = K;
            }
            if (u_out.cost <= target) break;
        }
    };
    // An LRU item stepped directly whose sets do not split is cut in time
    // instead: P parts of whole 1024-access blocks (so every bitmap word has
    // one writer), each part after the first first reading the trace back
    // until every set holds its a most recent lines (the LRU stack property:
    // that is the whole set state).  Returns P (1: no cut) and the costliest
    // part; bounds gets the parts' first steps and the end, pcost their costs.
    auto time_split = [&](uint64_t i, const UnitShape &u, double tgt, double &pmax_cost,
                          std::vector<uint32_t> *bounds, std::vector<double> *pcost) -> uint32_t {
        const SimItem &b = base[i];
        const ItemShape &sh = shape[i];
        const pchase_geom &G = geoms[b.cand];
        pmax_cost = u.cost;
        const uint32_t nsteps = (b.len + 31) / 32, nblk = (nsteps + 31) / 32;
        if (G.policy != PCHASE_LRU || !u.direct || u.mode != kModeBatch || u.cost <= tgt)
            return 1;
        const uint32_t pmax = std::min({max_split, 16u, nblk});
        // accesses read back before every line met is taken or in a full set
        // (after that the read skips ahead, to the trace's start if a set
        // never fills)
        const double fill = 1.5 * sh.cold + 1024.0;
        // (with a census of the sets' lines the read stops once every set has
        // all the lines it will get, held or not)
        const bool census = tn.streams && u.table_n <= kCensusMaxLines && u.sets <= kCensusMaxSets;
        const bool fills = census || (!sh.held && sh.visited >= (double)G.sets);
        auto bound = [&](uint32_t j, uint32_t P) {
            return std::min(nsteps, (uint32_t)((uint64_t)nblk * j / P) * 32);
        };
        auto part_cost = [&](uint32_t j, uint32_t P) {
            const uint32_t s0 = bound(j, P), s1 = bound(j + 1, P);
            const double back = 32.0 * s0;
            const double rb = j ? std::min(back, fill) / 32.0 * kRebuildNs +
                                      (fills ? 0.0 : std::max(0.0, back - fill) / 32.0 * kRebuildSkipNs)
                                : 0.0;
            return u.cost * (s1 - s0) / nsteps + rb;
        };
        uint32_t best_p = 1;
        for (uint32_t P = 2; P <= pmax; ++P) {
            double mx = 0.0;
            for (uint32_t j = 0; j < P; ++j) mx = std::max(mx, part_cost(j, P));
            if (mx < pmax_cost * 0.97) {
                pmax_cost = mx;
                best_p = P;
            }
            if (pmax_cost <= tgt) break;
        }
        if (bounds && best_p > 1) {
            bounds->clear();
            pcost->clear();
            for (uint32_t j = 0; j <= best_p; ++j) bounds->push_back(bound(j, best_p));
            for (uint32_t j = 0; j < best_p; ++j) pcost->push_back(part_cost(j, best_p));
        }
        return best_p;
    };
    double critical = 0.0;
    for (uint64_t i = 0; i < n_items; ++i) {
        if (gmem[i]) {
            critical = std::max(critical, gshape[i].cost);
            continue;
        }
        uint32_t k;
        UnitShape u;
        best_split(i, 0.0, k, u);
        double c = u.cost;
        UnitShape whole;
        if (k == 1) {
            time_split(i, u, 0.0, c, nullptr, nullptr);
        } else if (unit_shape(geoms[base[i].cand], base[i], 1, shape[i], tn, whole)) {
            double tc;
            if (time_split(i, whole, 0.0, tc, nullptr, nullptr) > 1) c = std::min(c, tc);
        }
        critical = std::max(critical, c);
    }
    // (0.6 of the critical estimate: the estimates scatter by about that
    // much, and a split unit near the critical one costs little once the
    // other work has drained)
    const double target = tn.split_cost_ns
                              ? (double)tn.split_cost_ns
                              : std::max({total / (kPlanSms * 36.0), 0.6 * critical, 2.0e5});
    p->est_critical = critical;
    p->est_target = target;
    std::vector<SimItem> items, gitems;
    std::vector<double> cost;
    try {
        items.reserve(n_items);
        cost.reserve(n_items);
        for (uint64_t i = 0; i < n_items; ++i) {
            const pchase_geom &G = geoms[base[i].cand];
            const ItemShape &sh = shape[i];
            if (gmem[i]) {
                // one whole unit; its set state goes in the pool region of
                // the warp that runs it (kres 0: at the region's start)
                SimItem it = base[i];
                apply_unit(it, gshape[i]);
                apply_compact(it, sh);
                it.lsh |= 1u << 17;
                it.kres = 0;
                p->pool_region = std::max<uint64_t>(p->pool_region, scan_state_bytes(G));
                it.cost = (float)gshape[i].cost;
                gitems.push_back(it);
                p->est_sum += gshape[i].cost;
                p->est_max_unit = std::max(p->est_max_unit, gshape[i].cost);
                p->n_gmem += 1;
                continue;
            }
            // smallest split that meets the target, else the cheapest one
            uint32_t best_k;
            UnitShape best;
            best_split(i, target, best_k, best);
            {
                double part_max = best.cost;
                std::vector<uint32_t> bounds;
                std::vector<double> pcost;
                uint32_t P = 1;
                UnitShape whole;
                if (best_k == 1) {
                    P = time_split(i, best, target, part_max, &bounds, &pcost);
                } else if (unit_shape(G, base[i], 1, sh, tn, whole)) {
                    // an LRU item that splits by sets may do better cut in time:
                    // a set-part re-reads the whole trace, a time part only
                    // what it reads back
                    double tmax;
                    std::vector<uint32_t> tb;
                    std::vector<double> tc;
                    const uint32_t tp = time_split(i, whole, target, tmax, &tb, &tc);
                    double tsum = 0.0;
                    for (double c : tc) tsum += c;
                    const bool better =
                        tp > 1 && (tmax <= target ? best.cost > target || tsum < best.cost * best_k
                                                  : tmax < best.cost);
                    if (better) {
                        P = tp;
                        part_max = tmax;
                        bounds.swap(tb);
                        pcost.swap(tc);
                        best = whole;
                        best_k = 1;
                    }
                }
                if (P > 1) {
                    for (uint32_t j = 0; j < P; ++j) {
                        SimItem it = base[i];
                        apply_unit(it, best);
                        apply_compact(it, sh);
                        it.ks1 = 1;
                        it.kres = bounds[j];
                        it.kmagic = bounds[j + 1];
                        it.lead = j == 0;
                        it.cost = (float)pcost[j];
                        items.push_back(it);
                        cost.push_back(it.cost);
                        p->est_sum += it.cost;
                        p->est_max_unit = std::max(p->est_max_unit, (double)it.cost);
                    }
                    continue;
                }
            }
            const DivMagic kdm = make_div_magic(best_k);
            for (uint32_t r = 0; r < best_k; ++r) {
                SimItem it = base[i];
                it.psh = (uint8_t)(best_k > 1 ? sh.psh : 0);
                it.kcnt = (uint8_t)best_k;
                if (!extra_ways(G)) it.kmagic = kdm.m;  // unequal sets keep a there
                it.ks1 = (uint8_t)kdm.s1;
                it.ks2 = (uint8_t)kdm.s2;
                it.kres = r;
                it.lead = r == 0;
                apply_unit(it, best);
                if (best_k == 1) apply_compact(it, sh);
                if (best_k > 1 && tn.streams && it.len >= kStreamMinLen)
                    it.direct = 2;  // reads its head stream
                it.cost = (float)best.cost;
                items.push_back(it);
                cost.push_back(best.cost);
                p->est_sum += best.cost;
                p->est_max_unit = std::max(p->est_max_unit, best.cost);
            }
        }
    } catch (...) {
        delete p;
        return fail(PCHASE_ENOMEM, "unit table allocation");
    }
    const uint64_t n_units = items.size();  // units of the size classes (the pool's apart)
    p->n_units = n_units + gitems.size();
    if (!gitems.empty()) {
        // the pool: one region per warp, at most 608 warps (4 per SM of a
        // full GPU) and 16 GB in all
        const uint64_t region = align16(p->pool_region);
        p->pool_region = region;
        uint64_t w = std::min<uint64_t>(gitems.size(), tn.pool_warps);
        w = std::min<uint64_t>(w, std::max<uint64_t>(1, kPoolMaxBytes / region));
        w = (w + kPoolWarpsPerCta - 1) / kPoolWarpsPerCta * kPoolWarpsPerCta;
        if (region * w > (64ull << 30) || (region >> 4) > 0xFFFFFFFFull) {
            delete p;
            return fail(PCHASE_ERANGE, "set state in global memory above 64 GB");
        }
        p->pool_warps = (uint32_t)w;
        p->gstate_bytes = region * w;
        std::stable_sort(gitems.begin(), gitems.end(),
                         [](const SimItem &x, const SimItem &y) { return x.cost > y.cost; });
    }

    // size classes, costliest units first inside each class
    std::vector<int> cls(n_units);
    const int ncap = (int)(sizeof kCaps / sizeof kCaps[0]);
    for (uint64_t i = 0; i < n_units; ++i) {
        int c = 0;
        while (kCaps[c] < items[i].arena_bytes) ++c;
        cls[i] = c;
    }
    // The few units that set the plan's length (the kIsolateMax costliest within kIsolateFrac
    // of the costliest, when the plan has far more work than they do) run
    // alone on an SM: given the largest class, they go to the one-warp launch,
    // whose CTAs fill an SM's shared memory, so no other warp slows their
    // dependent chains down.
    if (n_units > 64) {
        double cmax = 0.0, csum = 0.0;
        for (uint64_t i = 0; i < n_units; ++i) {
            cmax = std::max(cmax, cost[i]);
            csum += cost[i];
        }
        std::vector<uint64_t> top;
        for (uint64_t i = 0; i < n_units; ++i)
            if (cost[i] >= kIsolateFrac * cmax) top.push_back(i);
        std::sort(top.begin(), top.end(), [&](uint64_t x, uint64_t y) { return cost[x] > cost[y]; });
        if (top.size() > kIsolateMax) top.resize(kIsolateMax);
        if (csum > 64.0 * cmax) {
            for (uint64_t i : top) cls[i] = ncap - 1;
            p->n_isolated = top.size();
        }
    }
    std::vector<uint64_t> order(n_units);
    for (uint64_t i = 0; i < n_units; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](uint64_t x, uint64_t y) {
        if (cls[x] != cls[y]) return cls[x] > cls[y];
        const uint32_t gx = unit_group(items[x].mode, items[x].policy),
                       gy = unit_group(items[y].mode, items[y].policy);
        if (gx != gy) return gx < gy;
        return cost[x] > cost[y];
    });
    p->items.reserve(n_units + gitems.size());
    for (uint64_t k = 0; k < n_units; ++k) p->items.push_back(items[order[k]]);
    // the pool's units after every size class, costliest first
    for (const SimItem &it : gitems) p->items.push_back(it);
    // head streams: one job per caller item whose parts read them, its K
    // streams side by side in an entry area as long as its trace
    try {
        bool any = false;
        for (const SimItem &it : p->items) any = any || it.direct == 2;
        if (any) {
            p->item_slot.assign(n_items, 0xFFFFFFFFu);
            uint64_t ent = 0, cntw = 0;
            uint32_t seg = 0, slot = 0;
            for (uint64_t k = 0; k < p->items.size(); ++k) {
                const SimItem &it = p->items[k];
                if (it.direct != 2 || p->item_slot[it.out_item] != 0xFFFFFFFFu) continue;
                StreamJob J{};
                J.ent_base = ent;
                J.cnt_off = cntw;
                J.unit = (uint32_t)k;
                J.K = it.kcnt;
                J.nseg = (it.len + kSegAccesses - 1) / kSegAccesses;
                J.seg_first = seg;
                J.slot_first = slot;
                p->item_slot[it.out_item] = slot;
                for (uint32_t s = 0; s < J.nseg; ++s) p->seg_job.push_back((uint32_t)p->jobs.size());
                p->jobs.push_back(J);
                ent += it.len;
                cntw += (uint64_t)J.nseg * J.K;
                seg += J.nseg;
                slot += J.K;
            }
            p->n_ents = ent;
            p->n_cnt = cntw;
            p->n_slots = slot;
        }
        // census jobs: LRU items cut in time, small enough line tables
        if (tn.streams) {
            for (uint64_t k = 0; k < p->items.size(); ++k) {
                const SimItem &it = p->items[k];
                const bool tpart = it.kcnt == 1 && it.ks1 != 0 && it.direct == 1 &&
                                   it.mode == kModeBatch && it.policy == PCHASE_LRU &&
                                   !((it.lsh >> 17) & 1u);
                if (!tpart || it.table_n > kCensusMaxLines || it.sets > kCensusMaxSets) continue;
                if (p->item_slot.empty()) p->item_slot.assign(n_items, 0xFFFFFFFFu);
                if (p->item_slot[it.out_item] != 0xFFFFFFFFu) continue;
                StreamJob J{};
                J.kind = kJobCensus;
                J.ent_base = p->n_tgt;
                J.cnt_off = p->n_cnt;
                J.unit = (uint32_t)k;
                J.K = 1;
                J.nseg = (it.len + kSegAccesses - 1) / kSegAccesses;
                J.seg_first = (uint32_t)p->seg_job.size();
                J.slot_first = p->n_slots;
                p->item_slot[it.out_item] = p->n_slots;
                for (uint32_t s = 0; s < J.nseg; ++s) p->seg_job.push_back((uint32_t)p->jobs.size());
                p->jobs.push_back(J);
                p->n_tgt += it.sets;
                p->n_cnt += kCensusMaxLines / 32;
                p->n_slots += 1;
                p->n_census += 1;
            }
        }
    } catch (...) {
        delete p;
        return fail(PCHASE_ENOMEM, "head stream table allocation");
    }
    // queues: one per size class, smallest class first
    SlotLayout &L = p->layout;
    memset(&L, 0, sizeof L);
    std::vector<double> work(ncap, 0.0);
    std::vector<double> gwork[kUnitGroups];
    for (auto &v : gwork) v.assign(ncap, 0.0);
    uint32_t nclass = 0;
    {
        // classes present, in increasing cap order, renumbered 0..nclass-1
        std::vector<int> present;
        for (int c = 0; c < ncap; ++c) {
            bool any = false;
            for (uint64_t i = 0; i < n_units && !any; ++i) any = cls[i] == c;
            if (any) present.push_back(c);
        }
        nclass = (uint32_t)present.size();
        if (nclass > (uint32_t)kMaxClasses) {
            delete p;
            return fail(PCHASE_ERANGE, "too many size classes");
        }
        // sorted table is class-descending, then by group: find each run
        for (uint32_t q = 0; q < nclass; ++q) {
            const int c = present[q];
            for (uint32_t g = 0; g < (uint32_t)kUnitGroups; ++g) {
                uint64_t first = n_units, count = 0;
                for (uint64_t k = 0; k < n_units; ++k)
                    if (cls[order[k]] == c &&
                        unit_group(items[order[k]].mode, items[order[k]].policy) == g) {
                        if (first == n_units) first = k;
                        ++count;
                        work[q] += cost[order[k]];
                        gwork[g][q] += cost[order[k]];
                    }
                L.cls_first[g][q] = (uint32_t)(count ? first : 0);
                L.cls_count[g][q] = (uint32_t)count;
            }
        }
        L.nclasses = nclass;
        // Slot mix.  Classes whose arena exceeds half the CTA budget ("jumbo")
        // get a launch of their own, one warp per CTA.  For the others, slots
        // are added one at a time to minimise the estimated makespan
        // max_q (work of classes >= q) / (slots that can hold class q), since a
        // slot also serves every smaller class.
        std::vector<uint32_t> caps(nclass), slots(nclass, 0);
        for (uint32_t q = 0; q < nclass; ++q) caps[q] = kCaps[present[q]];
        p->class_caps = caps;
        const uint32_t budget = tn.smem_budget_bytes;
        int main_top = -1;
        for (uint32_t q = 0; q < nclass; ++q)
            if (caps[q] * 2 <= budget) main_top = (int)q;
        p->jumbo_first_class = (uint32_t)(main_top + 1);
        auto makespan = [&](const std::vector<uint32_t> &sl) {
            double worst = 0.0, wsum = 0.0;
            uint32_t ssum = 0;
            for (int q = main_top; q >= 0; --q) {
                wsum += work[q];
                ssum += sl[q];
                if (wsum > 0.0) worst = std::max(worst, ssum ? wsum / ssum : 1e300);
            }
            return worst;
        };
        uint32_t used = 0, nw = 0;
        if (main_top >= 0) {
            slots[main_top] = 1;
            used = caps[main_top];
            nw = 1;
            // extra large slots first (big_slots - 1 of them, each the largest
            // class that leaves half of what is left to the greedy fill): the
            // greedy alone spends the budget on small slots before the large
            // classes' work, which only the first slot holds, would pay
            for (uint32_t k = 1; k < tn.big_slots && nw < tn.max_warps_per_cta; ++k) {
                int q2 = -1;
                for (int q = main_top; q >= 0; --q)
                    if (caps[q] <= (budget - used) / 2 && work[q] > 0.0) { q2 = q; break; }
                if (q2 < 0) break;
                slots[q2] += 1;
                used += caps[q2];
                nw += 1;
            }
            while (nw < tn.max_warps_per_cta) {
                int best = -1;
                double best_ms = makespan(slots);
                for (int q = 0; q <= main_top; ++q) {
                    if (used + caps[q] > budget) continue;
                    slots[q] += 1;
                    const double ms = makespan(slots);
                    slots[q] -= 1;
                    if (ms < best_ms * (1.0 - 1e-9)) { best_ms = ms; best = q; }
                }
                if (best < 0) {
                    // no slot lowers the makespan: spend what is left on the
                    // smallest class with work (more warps to hide latency)
                    for (int q = 0; q <= main_top; ++q)
                        if (work[q] > 0.0 && used + caps[q] <= budget) { best = q; break; }
                    if (best < 0) break;
                }
                slots[best] += 1;
                used += caps[best];
                nw += 1;
            }
        }
        uint32_t off = 0, w = 0;
        for (int q = main_top; q >= 0; --q)
            for (uint32_t k = 0; k < slots[q]; ++k) {
                L.warp_class[w] = (uint32_t)q;
                L.warp_off[w] = off;
                off += caps[q];
                ++w;
            }
        L.nwarps = w;
        L.smem_bytes = off;
        // first-pop stagger: 4 us per slot for plans of long units, a
        // 2000th of the longest unit's estimate below that
        L.stagger_ns = (uint32_t)std::min(4000.0, p->est_max_unit / 2000.0);
        for (int g = 0; g < kUnitGroups; ++g)
            for (int q = 0; q <= main_top; ++q) p->gwork_main[g] += gwork[g][q];
        p->affinity = tn.kind_affinity != 0;
        // jumbo layout: one warp, the largest jumbo arena; serves jumbo classes
        SlotLayout &J = p->jumbo;
        memset(&J, 0, sizeof J);
        J.nclasses = nclass;
        memcpy(J.cls_first, L.cls_first, sizeof J.cls_first);
        memcpy(J.cls_count, L.cls_count, sizeof J.cls_count);
        if (main_top + 1 < (int)nclass) {
            J.nwarps = 1;
            J.spec = 1;  // one warp per SM: no other unit's code competes for its cache
            J.warp_class[0] = nclass - 1;
            J.warp_off[0] = 0;
            J.smem_bytes = caps[nclass - 1];
            // the jumbo warp must not steal main classes
            J.pad = (uint32_t)(main_top + 1);
            uint64_t nj = 0;
            for (uint32_t q = main_top + 1; q < nclass; ++q)
                for (int g = 0; g < kUnitGroups; ++g) nj += L.cls_count[g][q];
            p->n_jumbo = nj;
        }
    }
    // pool layout: kPoolWarpsPerCta warps per CTA, each with a queued unit's
    // staging arena, serving the one class after the size classes
    {
        SlotLayout &Gp = p->gpool;
        memset(&Gp, 0, sizeof Gp);
        if (!gitems.empty()) {
            const uint32_t gc = nclass;  // queue counter of the pool's class
            Gp.nclasses = gc + 1;
            Gp.pad = gc;
            // one queue (group 0's) for all of them, costliest first
            Gp.cls_first[0][gc] = (uint32_t)n_units;
            Gp.cls_count[0][gc] = (uint32_t)gitems.size();
            Gp.nwarps = kPoolWarpsPerCta;
            for (uint32_t w = 0; w < kPoolWarpsPerCta; ++w) {
                Gp.warp_class[w] = gc;
                Gp.warp_off[w] = w * kStageBytes;
            }
            Gp.smem_bytes = kPoolWarpsPerCta * kStageBytes;
            Gp.pool16 = (uint32_t)(p->pool_region >> 4);
        }
    }
    // workspace: [queues + status: kQueueHeader][items][geoms][seg offsets][obs word
    // offsets][pool]
    size_t off = kQueueHeader;
    p->off_items = off;
    off = align256(off + p->n_units * sizeof(SimItem));  // size classes and pool
    p->off_geoms = off;
    off = align256(off + (size_t)n_geom * sizeof(pchase_geom));
    p->off_seg = off;
    off = align256(off + (size_t)(n_trace + 1) * sizeof(uint64_t));
    p->off_obs_words = off;
    off = align256(off + (size_t)n_trace * sizeof(uint64_t));
    p->off_pool = off;
    off = align256(off + 2 * sizeof(uint64_t));
    p->off_gstate = off;
    off = align256(off + p->gstate_bytes);
    p->off_jobs = off;
    off = align256(off + p->jobs.size() * sizeof(StreamJob));
    p->off_segjob = off;
    off = align256(off + p->seg_job.size() * sizeof(uint32_t));
    p->off_itemslot = off;
    off = align256(off + p->item_slot.size() * sizeof(uint32_t));
    p->off_cnt = off;
    off = align256(off + p->n_cnt * sizeof(uint32_t));
    p->off_parts = off;
    off = align256(off + (size_t)p->n_slots * sizeof(PartInfo));
    p->off_ents = off;
    off = align256(off + p->n_ents * sizeof(uint2));
    p->off_tgt = off;
    off = align256(off + p->n_tgt * sizeof(uint32_t));
    p->ws_bytes = off;
    *plan_out = p;
    return PCHASE_OK;
}

void pchase_sim_plan_destroy(pchase_sim_plan *plan) { delete plan; }

size_t pchase_sim_plan_upload_bytes(const pchase_sim_plan *plan) {
    if (!plan) return 0;
    return plan->items.size() * sizeof(SimItem) + plan->geoms.size() * sizeof(pchase_geom) +
           plan->seg_offsets.size() * sizeof(uint64_t) +
           plan->obs_word_offsets.size() * sizeof(uint64_t) + 2 * sizeof(uint64_t) +
           (plan->jobs.empty() ? 0
                               : plan->jobs.size() * sizeof(StreamJob) +
                                     plan->seg_job.size() * sizeof(uint32_t) +
                                     plan->item_slot.size() * sizeof(uint32_t));
}

size_t pchase_sim_plan_workspace_bytes(const pchase_sim_plan *plan) {
    return plan ? plan->ws_bytes : 0;
}
uint64_t pchase_sim_plan_items(const pchase_sim_plan *plan) { return plan ? plan->n_items : 0; }
uint64_t pchase_sim_plan_bitmap_words(const pchase_sim_plan *plan) {
    return plan ? plan->bitmap_words : 0;
}
uint32_t pchase_sim_plan_launches(const pchase_sim_plan *plan) {
    if (!plan) return 0;
    // output clear + head streams (offsets; count and write when there are
    // segments) + main slot-mix launch + side launch of jumbo units + pool
    return (plan->n_units ? 1u : 0u) + (plan->jobs.empty() ? 0u : 1u) +
           (plan->seg_job.empty() ? 0u : 2u) + (plan->layout.nwarps ? 1u : 0u) +
           (plan->jumbo.nwarps ? 1u : 0u) + (plan->gpool.nwarps ? 1u : 0u);
}

size_t pchase_sim_plan_units(const pchase_sim_plan *plan, pchase_unit_info *out, size_t cap) {
    if (!plan) return 0;
    const size_t n = plan->items.size();
    for (size_t k = 0; k < n && k < cap && out; ++k) {
        const SimItem &it = plan->items[k];
        pchase_unit_info &u = out[k];
        memset(&u, 0, sizeof u);
        const bool gm = (it.lsh >> 17) & 1u, uneq = (it.lsh >> 16) & 1u;
        const bool tpart = it.kcnt == 1 && it.ks1 != 0 && !gm;
        const uint32_t nsteps = (it.len + 31) / 32;
        u.item = it.out_item;
        u.mode = it.mode;
        u.parts = it.kcnt;
        u.residue = it.kcnt > 1 ? it.kres : 0u;
        u.first_step = tpart ? it.kres : 0u;
        u.end_step = tpart ? it.kmagic : nsteps;
        u.flags = (it.direct == 1 ? PCHASE_UNIT_DIRECT : 0u) | (tpart ? PCHASE_UNIT_TIME_PART : 0u) |
                  (gm ? PCHASE_UNIT_GLOBAL_STATE : 0u) | (uneq ? PCHASE_UNIT_UNEQUAL : 0u) |
                  (it.lead ? PCHASE_UNIT_LEAD : 0u);
        u.arena_bytes = it.arena_bytes;
        u.est_ns = it.cost;
        u.policy = it.policy;
        if (gm) {
            // in the pool region of the warp that runs it, from its start
            u.state_offset = 0;
            u.state_bytes = scan_state_bytes(plan->geoms[it.cand]);
        }
    }
    return n;
}

size_t pchase_sim_plan_describe(const pchase_sim_plan *plan, char *buf, size_t bytes) {
    std::string d;
    if (plan) {
        uint64_t modes[3] = {0, 0, 0}, split = 0, direct = 0, tsplit = 0, gmem = 0;
        for (const SimItem &it : plan->items) {
            modes[it.mode < 3 ? it.mode : 0]++;
            split += it.kcnt > 1 && it.lead;
            tsplit += it.kcnt == 1 && it.ks1 && it.lead;
            gmem += (it.lsh >> 17) & 1u;
            direct += it.direct == 1;
        }
        char tmp[256];
        snprintf(tmp, sizeof tmp,
                 "items=%llu units=%llu split=%llu time_split=%llu global_state=%llu scan=%llu "
                 "table=%llu batch=%llu direct=%llu jumbo=%llu classes=%u warps=%u smem=%u slots=",
                 (unsigned long long)plan->n_items, (unsigned long long)plan->n_units,
                 (unsigned long long)split, (unsigned long long)tsplit, (unsigned long long)gmem,
                 (unsigned long long)modes[0],
                 (unsigned long long)modes[1], (unsigned long long)modes[2],
                 (unsigned long long)direct,
                 (unsigned long long)plan->n_jumbo, plan->layout.nclasses, plan->layout.nwarps,
                 plan->layout.smem_bytes);
        d = tmp;
        for (uint32_t w = 0; w < plan->layout.nwarps; ++w) {
            const uint32_t next = w + 1 < plan->layout.nwarps ? plan->layout.warp_off[w + 1]
                                                              : plan->layout.smem_bytes;
            snprintf(tmp, sizeof tmp, "%s%u", w ? "," : "", next - plan->layout.warp_off[w]);
            d += tmp;
        }
        d += " class_items=";
        for (uint32_t q = 0; q < plan->layout.nclasses; ++q) {
            uint32_t n = 0;
            for (int g = 0; g < kUnitGroups; ++g) n += plan->layout.cls_count[g][q];
            snprintf(tmp, sizeof tmp, "%s%u", q ? "," : "", n);
            d += tmp;
        }
        // each class's arena cap and its units' summed estimate
        d += " class_caps=";
        for (uint32_t q = 0; q < plan->class_caps.size(); ++q) {
            snprintf(tmp, sizeof tmp, "%s%u", q ? "," : "", plan->class_caps[q]);
            d += tmp;
        }
        d += " class_ms=";
        for (uint32_t q = 0; q < plan->layout.nclasses; ++q) {
            double w = 0.0;
            for (int g = 0; g < kUnitGroups; ++g)
                for (uint32_t k = 0; k < plan->layout.cls_count[g][q]; ++k)
                    w += plan->items[plan->layout.cls_first[g][q] + k].cost;
            snprintf(tmp, sizeof tmp, "%s%.1f", q ? "," : "", w * 1e-6);
            d += tmp;
        }
        snprintf(tmp, sizeof tmp, " est_ms=%.2f,%.2f,%.2f,%.1f", plan->est_critical * 1e-6,
                 plan->est_target * 1e-6, plan->est_max_unit * 1e-6, plan->est_sum * 1e-6);
        d += tmp;
        // the slot-mix launch's estimated work per unit group (mode * 3 +
        // policy) and whether SMs start on a home group
        d += " group_ms=";
        for (int g = 0; g < kUnitGroups; ++g) {
            snprintf(tmp, sizeof tmp, "%s%.1f", g ? "," : "", plan->gwork_main[g] * 1e-6);
            d += tmp;
        }
        snprintf(tmp, sizeof tmp, " affinity=%d", plan->affinity ? 1 : 0);
        d += tmp;
        if (!plan->jobs.empty()) {
            // head streams: split items, their parts, entries (8 bytes each);
            // census: LRU items cut in time whose sets' lines are counted
            snprintf(tmp, sizeof tmp, " streams=%zu,%u,%llu census=%u",
                     plan->jobs.size() - plan->n_census, plan->n_slots - plan->n_census,
                     (unsigned long long)plan->n_ents, plan->n_census);
            d += tmp;
        }
        if (plan->gpool.nwarps) {
            // the global-state pool: warps (one region each) x region bytes
            snprintf(tmp, sizeof tmp, " pool=%ux%llu", plan->pool_warps,
                     (unsigned long long)plan->pool_region);
            d += tmp;
        }
    }
    if (buf && bytes) {
        const size_t n = d.size() < bytes - 1 ? d.size() : bytes - 1;
        memcpy(buf, d.data(), n);
        buf[n] = 0;
    }
    return d.size();
}

int pchase_sim_plan_upload(const pchase_sim_plan *plan, void *workspace, size_t workspace_bytes,
                           pchase_stream_t stream) {
    if (!plan || !workspace) return fail(PCHASE_EINVAL, "plan or workspace is NULL");
    if (workspace_bytes < plan->ws_bytes) return fail(PCHASE_ERANGE, "workspace too small");
    if (reinterpret_cast<uintptr_t>(workspace) & 255)
        return fail(PCHASE_EINVAL, "workspace is not 256-byte aligned");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint8_t *w = static_cast<uint8_t *>(workspace);
    if (!plan->items.empty())
        PCHASE_CUDA(cudaMemcpyAsync(w + plan->off_items, plan->items.data(),
                                    plan->items.size() * sizeof(SimItem), cudaMemcpyHostToDevice, st),
                    "upload items");
    if (!plan->geoms.empty())
        PCHASE_CUDA(cudaMemcpyAsync(w + plan->off_geoms, plan->geoms.data(),
                                    plan->geoms.size() * sizeof(pchase_geom), cudaMemcpyHostToDevice,
                                    st),
                    "upload geometries");
    PCHASE_CUDA(cudaMemcpyAsync(w + plan->off_seg, plan->seg_offsets.data(),
                                plan->seg_offsets.size() * sizeof(uint64_t), cudaMemcpyHostToDevice,
                                st),
                "upload offsets");
    if (!plan->obs_word_offsets.empty())
        PCHASE_CUDA(cudaMemcpyAsync(w + plan->off_obs_words, plan->obs_word_offsets.data(),
                                    plan->obs_word_offsets.size() * sizeof(uint64_t),
                                    cudaMemcpyHostToDevice, st),
                    "upload word offsets");
    const uint64_t pool[2] = {0, plan->total_len};
    PCHASE_CUDA(cudaMemcpyAsync(w + plan->off_pool, pool, sizeof pool, cudaMemcpyHostToDevice, st),
                "upload pooled offsets");
    if (!plan->jobs.empty()) {
        PCHASE_CUDA(cudaMemcpyAsync(w + plan->off_jobs, plan->jobs.data(),
                                    plan->jobs.size() * sizeof(StreamJob), cudaMemcpyHostToDevice, st),
                    "upload stream jobs");
        if (!plan->seg_job.empty())
            PCHASE_CUDA(cudaMemcpyAsync(w + plan->off_segjob, plan->seg_job.data(),
                                        plan->seg_job.size() * sizeof(uint32_t),
                                        cudaMemcpyHostToDevice, st),
                        "upload stream segments");
        PCHASE_CUDA(cudaMemcpyAsync(w + plan->off_itemslot, plan->item_slot.data(),
                                    plan->item_slot.size() * sizeof(uint32_t),
                                    cudaMemcpyHostToDevice, st),
                    "upload stream slots");
    }
    return PCHASE_OK;
}

int pchase_sim_run(const pchase_sim_plan *plan, void *workspace, uint32_t *bitmaps,
                   const uint64_t *word_offsets, uint64_t *miss_counts, uint32_t *dev_status,
                   pchase_stream_t stream) {
    if (!plan || !workspace) return fail(PCHASE_EINVAL, "plan or workspace is NULL");
    if (plan->n_items == 0) return PCHASE_OK;
    SimOut out{};
    out.bitmaps = bitmaps;
    out.word_offsets = word_offsets;
    out.miss_counts = miss_counts;
    out.status = dev_status;
    return plan_launch(const_cast<pchase_sim_plan *>(plan), workspace, out,
                       reinterpret_cast<cudaStream_t>(stream));
}

int pchase_sim_run_filtered(const pchase_sim_plan *plan, void *workspace,
                            const uint32_t *filter, const uint64_t *filter_word_offsets,
                            uint32_t *bitmaps, const uint64_t *word_offsets,
                            uint64_t *miss_counts, uint32_t *dev_status, pchase_stream_t stream) {
    if (!plan || !workspace) return fail(PCHASE_EINVAL, "plan or workspace is NULL");
    if (!plan->filtered)
        return fail(PCHASE_EINVAL, "pchase_sim_run_filtered: plan not created with tune.filtered");
    if (!filter || !filter_word_offsets)
        return fail(PCHASE_EINVAL, "pchase_sim_run_filtered: filter or its offsets are NULL");
    if (plan->n_items == 0) return PCHASE_OK;
    SimOut out{};
    out.bitmaps = bitmaps;
    out.word_offsets = word_offsets;
    out.miss_counts = miss_counts;
    out.status = dev_status;
    out.filter = filter;
    out.filter_word_offsets = filter_word_offsets;
    return plan_launch(const_cast<pchase_sim_plan *>(plan), workspace, out,
                       reinterpret_cast<cudaStream_t>(stream));
}

int pchase_sim_run_profiled(const pchase_sim_plan *plan, void *workspace, uint32_t *bitmaps,
                            const uint64_t *word_offsets, uint64_t *miss_counts,
                            uint32_t *dev_status, uint64_t *timeline, pchase_stream_t stream) {
    if (!plan || !workspace || !timeline) return fail(PCHASE_EINVAL, "plan, workspace or timeline is NULL");
    if (plan->n_items == 0) return PCHASE_OK;
    SimOut out{};
    out.bitmaps = bitmaps;
    out.word_offsets = word_offsets;
    out.miss_counts = miss_counts;
    out.status = dev_status;
    out.timeline = timeline;
    return plan_launch(const_cast<pchase_sim_plan *>(plan), workspace, out,
                       reinterpret_cast<cudaStream_t>(stream));
}

int cache_sim_batch(const pchase_geom *geoms, uint32_t n_geom, const pchase_trace *traces,
                    uint32_t n_trace, const pchase_pair *pairs, uint32_t n_pairs,
                    uint32_t *bitmaps, const uint64_t *word_offsets, uint64_t *miss_counts,
                    uint32_t *dev_status, void *workspace, size_t *workspace_bytes,
                    pchase_stream_t stream) {
    if (!workspace_bytes) return fail(PCHASE_EINVAL, "workspace_bytes is NULL");
    pchase_sim_plan *p = nullptr;
    int rc = pchase_sim_plan_create(geoms, n_geom, traces, n_trace, pairs, n_pairs, nullptr, &p);
    if (rc) return rc;
    if (!workspace || *workspace_bytes < p->ws_bytes) {
        *workspace_bytes = p->ws_bytes;
        pchase_sim_plan_destroy(p);
        return fail(PCHASE_ERANGE, "workspace too small; *workspace_bytes holds the need");
    }
    rc = pchase_sim_plan_upload(p, workspace, *workspace_bytes, stream);
    if (!rc) rc = pchase_sim_run(p, workspace, bitmaps, word_offsets, miss_counts, dev_status, stream);
    pchase_sim_plan_destroy(p);
    return rc;
}

size_t pchase_classify_workspace_bytes(uint32_t n_obs, uint64_t max_len) {
    return classify_meta_bytes(n_obs) + align256(classify_bucket_bytes(n_obs, max_len));
}

int pchase_classify(const float *lat, const uint64_t *offsets, uint32_t n_obs, uint64_t max_len,
                    uint32_t *bits_out, const uint64_t *bit_word_offsets, float *thresh_out,
                    void *workspace, pchase_stream_t stream) {
    if (n_obs == 0) return PCHASE_OK;
    if (!lat || !offsets || !bits_out || !bit_word_offsets || !workspace)
        return fail(PCHASE_EINVAL, "pchase_classify: NULL argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint8_t *w = static_cast<uint8_t *>(workspace);
    void *meta = w;
    void *bk = w + classify_meta_bytes(n_obs);
    const int sms = sm_count();
    PCHASE_CUDA(classify_thresholds(lat, offsets, n_obs, max_len, meta, bk, thresh_out, st, sms),
                "classify thresholds");
    PCHASE_CUDA(classify_bits(lat, offsets, 1, n_obs, max_len,
                              meta, bits_out, bit_word_offsets, st, sms),
                "classify bits");
    return PCHASE_OK;
}

int pchase_match_run(const pchase_sim_plan *plan, void *workspace, const uint32_t *observed,
                     const uint64_t *obs_word_offsets, uint64_t stop_above, uint64_t *dist_out,
                     uint32_t *dev_status, pchase_stream_t stream) {
    if (!plan || !workspace || !observed || !obs_word_offsets || !dist_out)
        return fail(PCHASE_EINVAL, "pchase_match_run: NULL argument");
    if (!plan->cross) return fail(PCHASE_EINVAL, "matcher needs a candidates x traces plan");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    PCHASE_CUDA(cudaMemsetAsync(dist_out, 0, (size_t)plan->n_geom * sizeof(uint64_t), st),
                "cudaMemsetAsync(dist)");
    if (plan->n_items == 0) return PCHASE_OK;
    SimOut out{};
    out.status = dev_status;
    out.observed = observed;
    out.obs_word_offsets = obs_word_offsets;
    out.stop_above = stop_above;
    out.dist = dist_out;
    return plan_launch(const_cast<pchase_sim_plan *>(plan), workspace, out, st);
}

int pchase_canonical_pick(const pchase_geom *geoms, const uint64_t *dist, uint32_t n_cand,
                          uint32_t *pick_out, pchase_stream_t stream) {
    if (!geoms || !dist || !pick_out) return fail(PCHASE_EINVAL, "pchase_canonical_pick: NULL");
    PCHASE_CUDA(canonical_pick(geoms, dist, n_cand, pick_out, reinterpret_cast<cudaStream_t>(stream)),
                "canonical pick");
    return PCHASE_OK;
}

size_t pchase_infer_scratch_bytes(const pchase_sim_plan *plan) {
    if (!plan) return 0;
    return classify_meta_bytes(1) + align256(classify_bucket_bytes(1, plan->total_len)) +
           align256(plan->obs_words * sizeof(uint32_t) + 4);
}

int infer_geometry(const pchase_sim_plan *plan, void *workspace, const float *lat, void *scratch,
                   uint64_t stop_above, uint64_t *dist_out, uint32_t *pick_out,
                   uint32_t *dev_status, pchase_stream_t stream) {
    if (!plan || !workspace || !lat || !scratch || !dist_out || !pick_out)
        return fail(PCHASE_EINVAL, "infer_geometry: NULL argument");
    if (!plan->cross) return fail(PCHASE_EINVAL, "infer_geometry needs a candidates x traces plan");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint8_t *w = static_cast<uint8_t *>(workspace);
    uint8_t *s = static_cast<uint8_t *>(scratch);
    void *meta = s;
    void *bk = s + classify_meta_bytes(1);
    uint32_t *obs = reinterpret_cast<uint32_t *>(s + classify_meta_bytes(1) +
                                                 align256(classify_bucket_bytes(1, plan->total_len)));
    const uint64_t *pool = reinterpret_cast<const uint64_t *>(w + plan->off_pool);
    const uint64_t *seg = reinterpret_cast<const uint64_t *>(w + plan->off_seg);
    const uint64_t *owo = reinterpret_cast<const uint64_t *>(w + plan->off_obs_words);
    const int sms = sm_count();
    PCHASE_CUDA(classify_thresholds(lat, pool, 1, plan->total_len, meta, bk, nullptr, st, sms),
                "classify thresholds");
    PCHASE_CUDA(classify_bits(lat, seg, 0, plan->n_trace, plan->max_trace_len, meta, obs, owo,
                              st, sms),
                "classify bits");
    int rc = pchase_match_run(plan, workspace, obs, owo, stop_above, dist_out, dev_status, stream);
    if (rc) return rc;
    PCHASE_CUDA(canonical_pick(reinterpret_cast<const pchase_geom *>(w + plan->off_geoms), dist_out,
                               plan->n_geom, pick_out, st),
                "canonical pick");
    return PCHASE_OK;
}

size_t pchase_infer_batch_scratch_bytes(const pchase_sim_plan *plan, uint32_t n_obs) {
    if (!plan || n_obs == 0) return 0;
    const uint64_t T = plan->n_trace;
    return classify_meta_bytes(n_obs) + align256(classify_bucket_bytes(n_obs, plan->total_len)) +
           align256((n_obs + 1ull) * 8) + align256((n_obs * T + 1) * 8) +
           align256(n_obs * T * 8) + align256(n_obs * plan->obs_words * 4 + 4);
}

int infer_geometry_batch(const pchase_sim_plan *plan, void *workspace, const float *lat,
                         uint32_t n_obs, void *scratch, uint64_t stop_above, uint64_t *dist_out,
                         uint32_t *pick_out, uint32_t *dev_status, pchase_stream_t stream) {
    if (!plan || !workspace || !lat || !scratch || !dist_out || !pick_out)
        return fail(PCHASE_EINVAL, "infer_geometry_batch: NULL argument");
    if (!plan->cross) return fail(PCHASE_EINVAL, "infer_geometry_batch needs a candidates x traces plan");
    if (plan->n_gmem)
        return fail(PCHASE_EINVAL,
                    "infer_geometry_batch: a unit keeps its set state in global memory and "
                    "cannot run for several observations at once (use infer_geometry)");
    if (n_obs == 0) return PCHASE_OK;
    if ((uint64_t)n_obs * plan->n_trace > 65535 || n_obs > kMaxBatchObs)
        return fail(PCHASE_ERANGE, "infer_geometry_batch: too many observations for one call");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint8_t *w = static_cast<uint8_t *>(workspace);
    uint8_t *s = static_cast<uint8_t *>(scratch);
    const uint64_t T = plan->n_trace, L = plan->total_len;
    size_t off = 0;
    void *meta = s;
    off += classify_meta_bytes(n_obs);
    void *bk = s + off;
    off += align256(classify_bucket_bytes(n_obs, L));
    uint64_t *obs_off = reinterpret_cast<uint64_t *>(s + off);
    off += align256((n_obs + 1ull) * 8);
    uint64_t *seg_b = reinterpret_cast<uint64_t *>(s + off);
    off += align256((n_obs * T + 1) * 8);
    uint64_t *wo_b = reinterpret_cast<uint64_t *>(s + off);
    off += align256(n_obs * T * 8);
    uint32_t *bits = reinterpret_cast<uint32_t *>(s + off);
    const uint64_t *seg = reinterpret_cast<const uint64_t *>(w + plan->off_seg);
    const uint64_t *owo = reinterpret_cast<const uint64_t *>(w + plan->off_obs_words);
    const int sms = sm_count();
    PCHASE_CUDA(batch_offsets(seg, owo, (uint32_t)T, n_obs, L, plan->obs_words, obs_off, seg_b,
                              wo_b, st),
                "batch offsets");
    PCHASE_CUDA(classify_thresholds(lat, obs_off, n_obs, L, meta, bk, nullptr, st, sms),
                "classify thresholds");
    PCHASE_CUDA(classify_bits(lat, seg_b, (int)T, n_obs * (uint32_t)T, plan->max_trace_len, meta,
                              bits, wo_b, st, sms),
                "classify bits");
    PCHASE_CUDA(cudaMemsetAsync(dist_out, 0, (size_t)n_obs * plan->n_geom * sizeof(uint64_t), st),
                "cudaMemsetAsync(dist)");
    SimOut out{};
    out.status = dev_status;
    out.observed = bits;
    out.obs_word_offsets = owo;
    out.stop_above = stop_above;
    out.dist = dist_out;
    out.n_rep = n_obs;
    out.rep_dist_stride = plan->n_geom;
    out.rep_obs_stride = plan->obs_words;
    int rc = plan_launch(const_cast<pchase_sim_plan *>(plan), workspace, out, st);
    if (rc) return rc;
    PCHASE_CUDA(canonical_pick(reinterpret_cast<const pchase_geom *>(w + plan->off_geoms), dist_out,
                               plan->n_geom, pick_out, st, n_obs),
                "canonical pick");
    return PCHASE_OK;
}

int pchase_probe_latency(const uint32_t *array, uint32_t n_elems, uint32_t start, uint32_t warmup,
                         uint32_t iters, int cache_mode, uint32_t *lat_out, uint32_t *idx_out,
                         uint32_t *overhead_out, uint32_t *dev_status, pchase_stream_t stream) {
    if (!array || n_elems == 0 || !dev_status || (iters && (!lat_out || !idx_out)))
        return fail(PCHASE_EINVAL, "pchase_probe_latency: bad argument");
    if (iters > (1u << 24) || warmup > (1u << 26))
        return fail(PCHASE_ERANGE, "pchase_probe_latency: iters or warmup above the limit");
    if (cache_mode < 0 || cache_mode > 2) return fail(PCHASE_EINVAL, "unknown cache_mode");
    PCHASE_CUDA(probe_latency(array, n_elems, start, warmup, iters, cache_mode, lat_out, idx_out,
                              overhead_out, dev_status, reinterpret_cast<cudaStream_t>(stream)),
                "latency probe");
    return PCHASE_OK;
}

int pchase_probe_smem_bank(uint32_t max_stride, uint32_t repeats, float *cycles_out,
                           uint32_t *degree_out, pchase_stream_t stream) {
    if (max_stride < 1 || max_stride > 64 || repeats < 1 || repeats > 64 || !cycles_out || !degree_out)
        return fail(PCHASE_EINVAL, "pchase_probe_smem_bank: bad argument");
    PCHASE_CUDA(probe_smem(max_stride, repeats, cycles_out, degree_out,
                           reinterpret_cast<cudaStream_t>(stream)),
                "smem probe");
    return PCHASE_OK;
}

int pchase_probe_smem_throughput(uint32_t ctas, uint32_t threads, uint32_t ilp, uint32_t iters,
                                 uint64_t *t0_out, uint64_t *t1_out, uint32_t *smid_out,
                                 pchase_stream_t stream) {
    if (ctas == 0 || ctas > (1u << 20) || threads == 0 || threads > 1024 || (threads & 31) ||
        (ilp != 1 && ilp != 2 && ilp != 4 && ilp != 6 && ilp != 8) || iters == 0 ||
        iters > (1u << 20) || !t0_out || !t1_out || !smid_out)
        return fail(PCHASE_EINVAL, "pchase_probe_smem_throughput: bad argument");
    if (8ull * ilp * threads > 227ull * 1024)
        return fail(PCHASE_ERANGE, "pchase_probe_smem_throughput: 8 * ilp * threads above 227 KB");
    PCHASE_CUDA(probe_smem_copy(ctas, threads, ilp, iters,
                                reinterpret_cast<unsigned long long *>(t0_out),
                                reinterpret_cast<unsigned long long *>(t1_out), smid_out,
                                reinterpret_cast<cudaStream_t>(stream)),
                "shared-memory throughput probe");
    return PCHASE_OK;
}

int pchase_probe_global_throughput(int kind, uint32_t vec_bytes, uint32_t ctas, uint32_t threads,
                                   uint32_t ilp, const void *src, void *dst, uint64_t bytes,
                                   uint32_t reps, double *gbs_out, pchase_stream_t stream) {
    if (kind < 0 || kind > 2 || (vec_bytes != 4 && vec_bytes != 16) || ctas == 0 || threads == 0 ||
        threads > 1024 || (threads & 31) || (ilp != 1 && ilp != 2 && ilp != 4 && ilp != 8) ||
        reps == 0 || reps > 1000 || !gbs_out || !dst || (kind != 1 && !src) || bytes == 0 ||
        bytes % ((uint64_t)vec_bytes * ilp))
        return fail(PCHASE_EINVAL, "pchase_probe_global_throughput: bad argument");
    PCHASE_CUDA(probe_gmem(kind, vec_bytes, ctas, threads, ilp, src, dst, bytes, reps, gbs_out,
                           reinterpret_cast<cudaStream_t>(stream)),
                "throughput probe");
    return PCHASE_OK;
}

}  // extern "C"

// ------------------------------------------------------------ probe_* names
// The probe calls under the short names of the library's call list; same
// arguments, same behaviour.
extern "C" int probe_pchase(const uint32_t *array, uint32_t n_elems, uint32_t start,
                            uint32_t warmup, uint32_t iters, int cache_mode, uint32_t *lat_out,
                            uint32_t *idx_out, uint32_t *overhead_out, uint32_t *dev_status,
                            pchase_stream_t stream) {
    return pchase_probe_latency(array, n_elems, start, warmup, iters, cache_mode, lat_out,
                                idx_out, overhead_out, dev_status, stream);
}

extern "C" int probe_smem_bank(uint32_t max_stride, uint32_t repeats, float *cycles_out,
                               uint32_t *degree_out, pchase_stream_t stream) {
    return pchase_probe_smem_bank(max_stride, repeats, cycles_out, degree_out, stream);
}

extern "C" int probe_global_throughput(int kind, uint32_t vec_bytes, uint32_t ctas,
                                       uint32_t threads, uint32_t ilp, const void *src, void *dst,
                                       uint64_t bytes, uint32_t reps, double *gbs_out,
                                       pchase_stream_t stream) {
    return pchase_probe_global_throughput(kind, vec_bytes, ctas, threads, ilp, src, dst, bytes,
                                          reps, gbs_out, stream);
}

