/*
 * pchase.h - C ABI of the GB300 (sm_103a) fine-grained P-chase library.
 *
 * The library mechanises the method of Mei & Chu, "Dissecting GPU Memory
 * Hierarchy through Microbenchmarking" (arXiv:1509.02308):
 *   - P-chase trace construction (Listing 1, Sec. 4.1; non-uniform chains of
 *     Fig. 10, Sec. 5.2),
 *   - a batched set-associative cache simulator over many geometries
 *     (Assumptions 1-3 and Fig. 2, Sec. 4.1),
 *   - latency -> hit/miss classification and the exhaustive geometry matcher
 *     (the two-stage procedure of Fig. 6, Sec. 4.2),
 *   - probe kernels for the GPU itself: fine-grained P-chase (Listing 3,
 *     Sec. 4.2), shared-memory bank conflicts (Listing 4, Sec. 6.2) and
 *     global-memory throughput (Sec. 5.1).
 *
 * Conventions for every call:
 *   - Array indices are 4-byte elements; the byte address of element j is 4*j
 *     (Sec. 4.2 counts N and s in elements, Sec. 4.3 uses 4-byte elements).
 *   - The caller allocates and owns every buffer.  Pointers marked "device"
 *     must be device memory of the current CUDA device; pointers marked "host"
 *     are ordinary host memory.  The library keeps no pointer after a call
 *     returns, except inside an explicitly created handle (pchase_sim_plan).
 *   - Device work is queued on `stream` (a cudaStream_t; NULL is the legacy
 *     default stream) and is asynchronous unless the call says otherwise.
 *   - Every call returns a pchase_status.  Host-side validation failures are
 *     returned before anything is queued.  Errors found by a kernel while it
 *     runs (an index >= N, a chain leaving its array, a bounded wait that gave
 *     up) are OR-ed into the caller's device status word as PCHASE_DEV_* bits;
 *     the call itself cannot see them.  pchase_last_error_string() describes
 *     the last host-side failure of the calling thread.
 */
#ifndef PCHASE_H
#define PCHASE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pchase_stream_t; /* same type as cudaStream_t */

typedef enum {
    PCHASE_OK = 0,
    PCHASE_EINVAL = 1,   /* bad argument or geometry (T*a*b != C, b not a power of two, ...) */
    PCHASE_ERANGE = 2,   /* a size above a stated limit, or a buffer too small */
    PCHASE_ENOMEM = 3,   /* host allocation failed */
    PCHASE_ETIMEOUT = 4, /* a bounded wait gave up */
    PCHASE_ECUDA = 5     /* a CUDA runtime call failed; see pchase_last_error_string() */
} pchase_status;

/* Bits a kernel ORs into the caller's device status word (uint32). */
#define PCHASE_DEV_INDEX_RANGE 1u   /* a trace index was >= n_elems; the access was skipped */
#define PCHASE_DEV_CHAIN_RANGE 2u   /* a chain pointed outside its array; the walk stopped */
#define PCHASE_DEV_TIMEOUT 4u       /* a probe's iteration cap, or a bounded wait, ended a loop */

typedef enum {
    PCHASE_LRU = 0,
    PCHASE_FIFO = 1,
    PCHASE_RANDOM = 2,
    PCHASE_WEIGHTED = 3 /* the Fermi L1 data cache's policy (Sec. 4.5), see below */
} pchase_policy;

/*
 * Cache geometry (Assumption 1, Sec. 4.1): `sets` (T) sets of `ways` (a) lines
 * of `line_bytes` (b) bytes, C = T*a*b.  b must be a power of two >= 4.
 * Lines map to sets by set = (line >> mapping) mod T with line = (4*index) / b:
 * mapping 0 is the modular reading of Assumption 2; mapping m (at most 16)
 * puts the set bits m bits higher, so 2^m consecutive lines share a set (the
 * texture L1 cache of Sec. 4.3 is b = 32, T = 4, mapping 2: address bits 7-8).
 * Replacement: LRU (Assumption 3), FIFO, RANDOM, whose k-th eviction in set s
 * takes way
 *   floor(((h >> 32) * a) / 2^32),  h = SplitMix64(seed ^ (s << 40) ^ k),
 * SplitMix64 being the first output of Steele-Lea-Flood's generator whose
 * state is its argument, or WEIGHTED (a >= 3): evictions k = 0, 2, 4, ... of
 * set s take way 2, the others way r or r + 1 (r < 2 or r >= 2), where
 * r = floor(((h >> 32) * (a - 1)) / 2^32) with h as for RANDOM; on four ways
 * that replaces way 2 half of the time and each other way a sixth.  A miss
 * fills the lowest-numbered invalid way first.  32 bytes.
 */
typedef struct {
    uint32_t C_bytes;
    uint32_t line_bytes;
    uint32_t ways;
    uint32_t sets;
    uint32_t policy;  /* pchase_policy */
    uint32_t mapping; /* bits 0-7: m, set = (line >> m) mod T (0: set = line mod T, at most
                         16).  Bits 8-15: extra, unequal sets as in the L2 TLB of Sec. 4.4
                         (Fig. 9: one set of 17 entries, six of 8): set 0 has ways + extra
                         ways, C = (sets*ways + extra) * line_bytes, and line residue
                         r = line mod (sets*ways + extra) goes to set r mod sets when
                         r < sets*ways, else to set 0 (a reading: the paper gives the set
                         sizes, not the rule).  Unequal sets take m = 0 and LRU or FIFO,
                         run as way scans and are never split.  Bits 16-31: zero. */
    uint64_t seed;    /* RANDOM and WEIGHTED only */
} pchase_geom;

/*
 * One access trace.  `idx` (device) holds `len` element indices, each below
 * `n_elems`; idx == NULL selects the analytic uniform chain of Listing 1 walked
 * from j = 0, whose access t visits (t * stride) mod n_elems.  The first
 * `warmup` accesses (the preheat pass of Listing 3) are counted apart.
 * len < 2^31.  32 bytes.
 */
typedef struct {
    const uint32_t *idx;
    uint64_t len;
    uint64_t warmup;
    uint32_t n_elems;
    uint32_t stride;
} pchase_trace;

/* One simulation item: geometry `geom` replays trace `trace`. */
typedef struct {
    uint32_t geom;
    uint32_t trace;
} pchase_pair;

/* ------------------------------------------------------------------ S1 */

/*
 * Listing 1 (Sec. 4.1) and the chase of Listings 2-3: writes into trace_out
 * (device, len uint32) the indices visited by j = A[j] from j = 0.
 *   next == NULL: uniform chain A[i] = (i + stride) mod n_elems, so
 *                 trace_out[t] = (t * stride) mod n_elems (parallel).
 *   next != NULL: caller-built chain (device, n_elems entries), such as the
 *                 non-uniform chains of Fig. 10; walked by one thread.  A
 *                 link >= n_elems sets PCHASE_DEV_CHAIN_RANGE in *dev_status
 *                 (device) and the rest of trace_out is left unwritten.
 * array_out (device, n_elems uint32, may be NULL) receives the uniform array
 * of Listing 1 itself, for the probe of pchase_probe_latency.
 * Errors: EINVAL if n_elems == 0, or next != NULL and dev_status == NULL.
 */
int pchase_build(uint32_t n_elems, uint32_t stride, const uint32_t *next, uint64_t len,
                 uint32_t *trace_out, uint32_t *array_out, uint32_t *dev_status,
                 pchase_stream_t stream);

/*
 * Batched uniform chains: trace i (host descriptor traces[i], idx ignored) is
 * written to trace_out + word_offsets[i] (host offsets, in uint32 elements).
 * One launch for all n traces.
 */
int pchase_build_batch(const pchase_trace *traces, uint32_t n, uint32_t *trace_out,
                       const uint64_t *word_offsets, pchase_stream_t stream);

/* ---------------------------------------------------------- S2, S3, S6 */

/*
 * Tuning knobs of the simulator, chosen by the autotuner or left at their
 * defaults (pass NULL).  See pchase_sim_plan_create.
 */
typedef struct {
    uint32_t scan_max_ways;      /* a <= this: way-scan sets; above: line-table sets (default 4) */
    uint32_t smem_budget_bytes;  /* shared memory per CTA for the slot mix (default 220 KB) */
    uint32_t max_warps_per_cta;  /* (default 16) */
    uint32_t ctas_per_sm_cap;    /* 0 = as many as fit */
    uint32_t batch_max_sets;     /* T <= this: whole-step batch resolution per set (default 64;
                                    0 keeps the default, 0xFFFFFFFF disables batch mode) */
    uint32_t max_split;          /* most parts a long item's sets are split into (2^j or
                                    3 * 2^j, default 32; 1 = never split).  An LRU item
                                    whose sets do not split is cut in time instead, into at
                                    most min(this, 16) parts of whole 1024-access blocks */
    uint32_t split_cost_ns;      /* split items whose estimated warp time is above this
                                    (0 = automatic, from the whole plan's estimated work) */
    uint32_t filtered;           /* 1: the plan is a lower level of a hierarchy; every unit
                                    gathers its accesses, so pchase_sim_run_filtered can skip
                                    the ones a filter bitmap leaves out (default 0) */
    uint32_t pool_warps;         /* most warps of the global-state pool launch, each owning
                                    one state region (default and at most 608; rounded up
                                    to a multiple of 4) */
    uint32_t big_slots;          /* slots per CTA placed for the largest size classes before
                                    the greedy fill of the slot mix (default 1, at most 4) */
    uint32_t kind_affinity;      /* 0 (default) or 1: each SM of the slot-mix launch starts
                                    on one kind of unit (set mode x policy, WEIGHTED with
                                    RANDOM), SMs shared among the kinds by estimated work,
                                    and keeps to it while it has units, so an SM's warps
                                    mostly share one kind's code, with one copy of the unit
                                    loop per kind; 0xFFFFFFFF: every warp takes the
                                    costliest next unit of any kind, and all kinds share
                                    one unit loop */
    uint32_t head_streams;       /* 0 (default) or 1: in a plan of explicit pairs that is not
                                    filtered, the parts of items split by sets read head
                                    streams written by a pass before the simulator;
                                    0xFFFFFFFF: every part gathers its heads itself */
} pchase_tune;

typedef struct pchase_sim_plan pchase_sim_plan;

/*
 * Plans a batch of simulation items on the host (no device work).  Item i is
 * pairs[i]; pairs == NULL means all n_geom x n_trace combinations, item
 * g * n_trace + t.  geoms, traces and pairs are host arrays; the trace index
 * pointers inside `traces` are device pointers used later by pchase_sim_run.
 * Items whose estimated work dominates the batch are split by sets into
 * independent units (sets never interact, so the result is unchanged).  In a
 * plan of explicit pairs that is not a hierarchy's lower level, the parts of
 * a split item do not each gather their accesses from the whole trace: a pass
 * before the simulator writes each part's run heads (with their positions,
 * 8 bytes each, at most one per access of the item) into the workspace, and
 * the part steps over those; pchase_match_run, and plans of all pairs, gather
 * instead.  Units are sorted costliest first into shared-memory size classes served by one
 * persistent launch with a per-CTA mix of arenas (S6); units too large for
 * that mix get a second launch on a side stream.  An item whose set state fits
 * no shared-memory arena even split (a cache of many lines, or a line table
 * over a wide stream), or whose splits cost more warp time in all, runs as one
 * way-scan unit with its state in global memory: a third launch of at most
 * 608 warps, each owning one region of a pool inside the plan's workspace
 * (at most 16 GB in all; pchase_sim_plan_workspace_bytes counts it) and
 * reusing it from unit to unit.  Analytic chains (idx == NULL) whose visited
 * lines are every lstep-th line key a whole unit's state by line / lstep, so
 * their line tables cover the chain's lines, not the array's.  Errors: EINVAL
 * for a bad geometry, pair or trace; ERANGE for a geometry of more than 2^24
 * lines.
 */
int pchase_sim_plan_create(const pchase_geom *geoms, uint32_t n_geom,
                           const pchase_trace *traces, uint32_t n_trace,
                           const pchase_pair *pairs, uint32_t n_pairs,
                           const pchase_tune *tune, pchase_sim_plan **plan_out);
void pchase_sim_plan_destroy(pchase_sim_plan *plan);

/* Bytes of device workspace pchase_sim_run needs for this plan. */
size_t pchase_sim_plan_workspace_bytes(const pchase_sim_plan *plan);
/* Bytes pchase_sim_plan_upload copies from the host (the plan's tables; the
 * rest of the workspace is written on the device). */
size_t pchase_sim_plan_upload_bytes(const pchase_sim_plan *plan);
/* Number of items, and of bitmap words when the plan lays bitmaps out itself. */
uint64_t pchase_sim_plan_items(const pchase_sim_plan *plan);
uint64_t pchase_sim_plan_bitmap_words(const pchase_sim_plan *plan);
/* Kernel launches one pchase_sim_run queues (the output clear; when the plan
 * splits items by sets, the three launches of their head streams; the
 * slot-mix launch; and the side launches of jumbo and pool units, when it has
 * them); pchase_match_run queues neither the output clear nor the head
 * streams. */
uint32_t pchase_sim_plan_launches(const pchase_sim_plan *plan);
/*
 * Writes a one-line text description of the plan (items split by sets and
 * cut in time, units per set mode, units that step over their accesses
 * directly, size classes, the per-CTA slot mix,
 * and the cost model's estimates in ms of one
 * warp: est_ms=<longest unsplittable unit>,<split target>,<longest unit>,<sum>)
 * into buf (host, `bytes` long, always NUL-terminated); returns the length the
 * full text needs.
 */
size_t pchase_sim_plan_describe(const pchase_sim_plan *plan, char *buf, size_t bytes);

/* One unit of a plan, as pchase_sim_plan_units reports it (host, 56 bytes). */
typedef struct {
    uint32_t item;         /* the caller's item it simulates (part of) */
    uint32_t mode;         /* set mode: 0 way scans, 1 line table, 2 batch */
    uint32_t parts;        /* K of a split by sets (1: all of the item's sets) */
    uint32_t residue;      /* the set groups this part owns: (set >> p) mod K == residue */
    uint32_t first_step;   /* steps of 32 accesses it covers: [first_step, end_step) */
    uint32_t end_step;
    uint32_t flags;        /* PCHASE_UNIT_* bits */
    uint32_t arena_bytes;  /* shared memory the unit needs */
    uint64_t state_offset; /* PCHASE_UNIT_GLOBAL_STATE: offset of its set state in the pool */
    uint64_t state_bytes;  /*   region of the warp that runs it (0), and its size; else 0, 0 */
    float est_ns;          /* the planner's estimate of its warp time */
    uint32_t policy;       /* the item's replacement policy (PCHASE_LRU ...) */
} pchase_unit_info;
#define PCHASE_UNIT_DIRECT 1u        /* steps over consecutive accesses (no queue) */
#define PCHASE_UNIT_TIME_PART 2u     /* an LRU item cut in time (rebuilds its start state) */
#define PCHASE_UNIT_GLOBAL_STATE 4u  /* way scans over set state in global memory */
#define PCHASE_UNIT_UNEQUAL 8u       /* unequal sets (pchase_geom.mapping bits 8-15) */
#define PCHASE_UNIT_LEAD 16u         /* the one unit of its item that clears the outputs */
/*
 * Copies the plan's units, in the order the kernels take them, into out
 * (host, up to `cap` entries; out may be NULL with cap 0) and returns how
 * many units the plan has.  Host only: a view of the plan for checks and
 * tools (every bitmap word has one writer; a unit's global-memory set state
 * fits a pool region).
 */
size_t pchase_sim_plan_units(const pchase_sim_plan *plan, pchase_unit_info *out, size_t cap);

/*
 * Copies the plan's tables into `workspace` (device, at least
 * pchase_sim_plan_workspace_bytes, 256-byte aligned).  Needed once per
 * workspace before any number of pchase_sim_run calls.  Uses pageable-host
 * cudaMemcpyAsync, so it must not be called during stream capture.
 */
int pchase_sim_plan_upload(const pchase_sim_plan *plan, void *workspace, size_t workspace_bytes,
                           pchase_stream_t stream);

/*
 * Runs the planned batch: every item replays its trace through its geometry
 * from an empty cache.  Outputs (all device):
 *   bitmaps: per item ceil(len/32) uint32 words, bit t%32 of word t/32 is 1
 *     when access t misses (LSB first); item i starts at word_offsets[i]
 *     (device, uint64) or, when word_offsets == NULL, at the plan's own
 *     back-to-back layout (pchase_sim_plan_bitmap_words words in total).
 *     bitmaps may be NULL to skip them.
 *   miss_counts: 2 uint64 per item: misses over all accesses, and misses
 *     after the first `warmup` accesses.  May be NULL.
 *   dev_status: uint32 status word (PCHASE_DEV_* bits); may be NULL.
 * Only kernel launches and a memset are queued (no host copies), so the call
 * can be captured into a CUDA graph; the work fans out over internal streams
 * that join back into `stream`.
 */
int pchase_sim_run(const pchase_sim_plan *plan, void *workspace, uint32_t *bitmaps,
                   const uint64_t *word_offsets, uint64_t *miss_counts, uint32_t *dev_status,
                   pchase_stream_t stream);

/*
 * The next level of a hierarchy (Sec. 3: an L1 miss goes to L2, an L1 hit never
 * does; with page-sized lines, a TLB level of Sec. 4.4): like pchase_sim_run,
 * but item i sees only the accesses whose bit is set in its filter bitmap,
 * filter + filter_word_offsets[i] (device; packed like `bitmaps`, normally the
 * miss bitmap of the level above for the same trace), in order.  The other
 * accesses neither hit nor miss (bit 0).  The plan must have been created
 * with pchase_tune.filtered = 1 (PCHASE_EINVAL otherwise).  The level an
 * access is served from is the sum of its bits over the levels.
 */
int pchase_sim_run_filtered(const pchase_sim_plan *plan, void *workspace,
                            const uint32_t *filter, const uint64_t *filter_word_offsets,
                            uint32_t *bitmaps, const uint64_t *word_offsets,
                            uint64_t *miss_counts, uint32_t *dev_status, pchase_stream_t stream);

/*
 * pchase_sim_run that also records, per item i (in the caller's numbering),
 * timeline[4i .. 4i+3] = {start ns, end ns (the GPU's global timer), SM id,
 * warp slot}; timeline is a device buffer of 4 * items uint64.  For
 * load-balance diagnosis and the autotuner.
 */
int pchase_sim_run_profiled(const pchase_sim_plan *plan, void *workspace, uint32_t *bitmaps,
                            const uint64_t *word_offsets, uint64_t *miss_counts,
                            uint32_t *dev_status, uint64_t *timeline, pchase_stream_t stream);

/*
 * One-shot form of the three calls above (plan, upload, run, destroy) for a
 * caller-provided workspace; returns ERANGE with *workspace_bytes set to the
 * need when workspace_bytes is too small (workspace may then be NULL).
 */
int cache_sim_batch(const pchase_geom *geoms, uint32_t n_geom, const pchase_trace *traces,
                    uint32_t n_trace, const pchase_pair *pairs, uint32_t n_pairs,
                    uint32_t *bitmaps, const uint64_t *word_offsets, uint64_t *miss_counts,
                    uint32_t *dev_status, void *workspace, size_t *workspace_bytes,
                    pchase_stream_t stream);

/* --------------------------------------------------------------- S4, S5 */

/*
 * Latency -> hit/miss (S4).  Sec. 4.1 models a P-chase latency as t0 (hit)
 * or t0 + t_m (miss); the paper states no cut rule.  Reading: over one
 * observation (the `n` latencies lat[offset[o] .. offset[o+1]), device
 * float), set aside the largest floor(n/200) values, find the largest gap
 * between consecutive distinct kept values (the lowest one on ties) and cut at
 * (lo + hi) * 0.5f; a latency above the cut is a miss.  No gap: all hits.
 * Writes packed miss bits (LSB first) for observation o at
 * bits_out + bit_word_offsets[o] (device) and the cut to thresh_out[o].
 * offsets, bit_word_offsets: device uint64, n_obs + 1 and n_obs entries.
 * max_len must be at least every observation's length n: the workspace holds
 * 2 * max_len buckets per observation.  An observation with n > max_len (or
 * with offsets[o+1] < offsets[o]) is refused on the device: its thresh_out[o]
 * is NaN, its bits are all 0, and it touches no workspace byte outside its
 * own slice; the other observations are unaffected.
 * Work buffers: `workspace` (device) of pchase_classify_workspace_bytes.
 */
size_t pchase_classify_workspace_bytes(uint32_t n_obs, uint64_t max_len);
int pchase_classify(const float *lat, const uint64_t *offsets, uint32_t n_obs,
                    uint64_t max_len, uint32_t *bits_out, const uint64_t *bit_word_offsets,
                    float *thresh_out, void *workspace, pchase_stream_t stream);

/*
 * pchase_classify without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory, for
 * example a measurement loop that classifies probe latencies between probe
 * runs, where a cudaMalloc would synchronise the device and disturb the very
 * timings being taken, or a process whose device memory is owned entirely by
 * another allocator.  Same inputs, outputs, reading and max_len contract (an
 * observation longer than max_len gets a NaN cut and all-0 bits) as
 * pchase_classify; its scratch is a fixed 8 MiB array inside the library
 * (every GPU that loads the library holds it until the process exits), so the
 * request must satisfy r(16 * n_obs) + r(16 * n_obs * max_len) <= 8 MiB, r(x)
 * being x rounded up to a multiple of 256, else the call returns
 * PCHASE_ERANGE without queuing anything.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and should come
 * before any stream capture.  Every call on a device shares the one array:
 * calls whose work overlaps on the GPU (different streams, or another thread)
 * race on it; calls queued on one stream are ordered.  The kernels initialise
 * everything they read, so contents left by an earlier call are never used.
 * Calls no cudaMalloc, cudaFree or other allocating routine.
 */
int pchase_classify_noalloc(const float *lat, const uint64_t *offsets, uint32_t n_obs,
                            uint64_t max_len, uint32_t *bits_out,
                            const uint64_t *bit_word_offsets, float *thresh_out,
                            pchase_stream_t stream);
/* Size in bytes of the static scratch of pchase_classify_noalloc (8 MiB). */
size_t pchase_classify_noalloc_limit_bytes(void);

/*
 * Exhaustive matcher (S5), the mechanised form of Fig. 6 (Sec. 4.2): every
 * plan item (candidate g, plan trace t) is replayed and compared with the
 * observed miss bits of trace t (observed + obs_word_offsets[t], device); the
 * Hamming distance summed over the candidate's traces goes to dist_out[g]
 * (device uint64, zeroed by the call).  `plan` must have been created with
 * pairs == NULL over (candidates x plan traces); `stop_above`: an item stops
 * once its candidate's distance (the other items' sums so far plus its own)
 * exceeds it, and an item of a candidate already above it is skipped
 * (UINT64_MAX: never).  Every candidate whose distance is <= stop_above gets
 * its exact distance; any other gets some value above stop_above.
 */
int pchase_match_run(const pchase_sim_plan *plan, void *workspace, const uint32_t *observed,
                     const uint64_t *obs_word_offsets, uint64_t stop_above, uint64_t *dist_out,
                     uint32_t *dev_status, pchase_stream_t stream);

/*
 * Canonical pick (device, one thread block): among n_cand candidates (geoms,
 * device) with distances dist (device), the smallest distance wins, then
 * policy LRU < FIFO < RANDOM, then the larger line size, then fewer ways, then
 * the smaller capacity (identifiability reading of Sec. 4.2: geometries that
 * no plan point separates are reported as one class).  Writes the pick's
 * index and the number of candidates at the smallest distance to
 * pick_out[0], pick_out[1] (device uint32).
 */
int pchase_canonical_pick(const pchase_geom *geoms, const uint64_t *dist, uint32_t n_cand,
                          uint32_t *pick_out, pchase_stream_t stream);

/*
 * S4 + S5 in one call for one observation: classify the latencies of all plan
 * traces together, match against every candidate, pick.  lat (device float)
 * holds the plan traces' latencies back to back in trace order; the plan must
 * be a candidates x traces plan whose workspace was uploaded.  stop_above as
 * in pchase_match_run (UINT64_MAX: every distance exact; a bound B keeps the
 * pick exact whenever some candidate is within B).  Outputs (device):
 * dist_out[n_cand] (uint64), pick_out[2] (uint32).  Extra device work buffer
 * `scratch` of pchase_infer_scratch_bytes(plan).
 */
size_t pchase_infer_scratch_bytes(const pchase_sim_plan *plan);
int infer_geometry(const pchase_sim_plan *plan, void *workspace, const float *lat,
                   void *scratch, uint64_t stop_above, uint64_t *dist_out, uint32_t *pick_out,
                   uint32_t *dev_status, pchase_stream_t stream);

/*
 * infer_geometry over n_obs observations in one call (batched inference):
 * lat (device) holds n_obs observations back to back, each the plan's
 * traces' latencies in trace order (total length L = sum of trace lengths).
 * Every observation gets its own pooled threshold (R9), its own distances
 * dist_out[o * n_candidates + g] and its own canonical pick
 * pick_out[2o], pick_out[2o + 1].  The candidates' items run once per
 * observation inside the same launches.  Scratch (device, 256-byte aligned):
 * pchase_infer_batch_scratch_bytes(plan, n_obs).  Errors: EINVAL as
 * infer_geometry, or when a unit of the plan keeps its set state in global
 * memory (it cannot run for several observations at once); ERANGE when
 * n_obs > 1024 or n_obs x plan traces > 65535.
 */
size_t pchase_infer_batch_scratch_bytes(const pchase_sim_plan *plan, uint32_t n_obs);
int infer_geometry_batch(const pchase_sim_plan *plan, void *workspace, const float *lat,
                         uint32_t n_obs, void *scratch, uint64_t stop_above, uint64_t *dist_out,
                         uint32_t *pick_out, uint32_t *dev_status, pchase_stream_t stream);

/* --------------------------------------------------------------- S8-S10 */

/*
 * Fine-grained P-chase probe (Listing 3, Sec. 4.2) on this GPU.  One thread
 * walks j = array[j] (device chain of n_elems entries, e.g. from
 * pchase_build) from j = start: it first runs `warmup` untimed accesses (the
 * preheat), then `iters` timed ones.  Each timed access reads clock64 before
 * the load and after a dependent store of the loaded index into shared
 * memory, buffering up to 256 latencies and indices in shared memory before
 * copying them out; lat_out[i] is the raw cycle count of access i minus
 * overhead_out[0], the measured cost of the same clock + dependent-store
 * sequence around a shared-memory load. idx_out[i] is the index visited by
 * access i.  cache_mode: 0 = ld.global.ca (L1 and L2), 1 = ld.global.cg
 * (L2 only), 2 = ld.global.nc (read-only path).  Device outputs: lat_out,
 * idx_out (iters uint32 each), overhead_out (2 uint32: store+clock segment,
 * back-to-back clock64 reads).  Limits: iters <= 1<<24, warmup <= 1<<26.
 * A link >= n_elems sets PCHASE_DEV_CHAIN_RANGE and stops the walk.
 */
int pchase_probe_latency(const uint32_t *array, uint32_t n_elems, uint32_t start,
                         uint32_t warmup, uint32_t iters, int cache_mode, uint32_t *lat_out,
                         uint32_t *idx_out, uint32_t *overhead_out, uint32_t *dev_status,
                         pchase_stream_t stream);

/*
 * Shared-memory stride probe (Listing 4, Sec. 6.2): one warp; lane t starts
 * at word t*stride and follows 64 dependent reads of a self-pointing word, for
 * every stride in [1, max_stride] (max_stride <= 64).  cycles_out[s-1]
 * (device float) is the mean clock64 cycles per access of stride s (median of
 * `repeats` timed rounds, repeats in [1, 64]); degree_out[s-1] (device uint32)
 * is the conflict degree the bank model predicts for the same request (32
 * banks of 4-byte words, equal words broadcast).
 */
int pchase_probe_smem_bank(uint32_t max_stride, uint32_t repeats, float *cycles_out,
                           uint32_t *degree_out, pchase_stream_t stream);

/*
 * Global-memory throughput probe (Sec. 5.1, Table 5).  kind: 0 read, 1 write,
 * 2 copy (counts 2 * bytes, as the paper does).  vec_bytes: 4 (fp32) or 16
 * (int4).  ctas, threads: launch shape (threads a multiple of 32, <= 1024);
 * ilp: independent vectors per thread per loop trip (1, 2, 4 or 8).  src,
 * dst: device buffers of `bytes` (bytes a multiple of vec_bytes * ilp;
 * src unused for write, dst unused... for read a 4-byte device sink is dst).
 * SYNCHRONOUS: runs `reps` timed launches after one warm-up launch, timing
 * each with CUDA events on `stream`, and returns the median GB/s (1e9 B/s)
 * in *gbs_out (host).
 */
int pchase_probe_global_throughput(int kind, uint32_t vec_bytes, uint32_t ctas,
                                   uint32_t threads, uint32_t ilp, const void *src, void *dst,
                                   uint64_t bytes, uint32_t reps, double *gbs_out,
                                   pchase_stream_t stream);

/*
 * The three probes above under the short names of the library's call list
 * (probe_pchase = pchase_probe_latency, probe_smem_bank =
 * pchase_probe_smem_bank, probe_global_throughput =
 * pchase_probe_global_throughput): same arguments, limits and behaviour.
 */
int probe_pchase(const uint32_t *array, uint32_t n_elems, uint32_t start, uint32_t warmup,
                 uint32_t iters, int cache_mode, uint32_t *lat_out, uint32_t *idx_out,
                 uint32_t *overhead_out, uint32_t *dev_status, pchase_stream_t stream);
int probe_smem_bank(uint32_t max_stride, uint32_t repeats, float *cycles_out,
                    uint32_t *degree_out, pchase_stream_t stream);
int probe_global_throughput(int kind, uint32_t vec_bytes, uint32_t ctas, uint32_t threads,
                            uint32_t ilp, const void *src, void *dst, uint64_t bytes,
                            uint32_t reps, double *gbs_out, pchase_stream_t stream);

/*
 * Shared-memory throughput probe (Sec. 6.1, Table 6): `ctas` CTAs of
 * `threads` threads (a multiple of 32, <= 1024); every thread copies `ilp`
 * (1, 2, 4, 6 or 8) 4-byte words from one shared region to another, `iters`
 * (<= 2^20) times, so a CTA uses 8 * ilp * threads bytes of shared memory (at
 * most 227 KB) and moves 8 * ilp * threads * iters bytes (read + write).
 * Launch ctas = SMs x CTAs per SM to place that many CTAs on each SM.  For
 * CTA i the device outputs hold the SM clock64 before and after its copy loop
 * (each taken after a __syncthreads; uint64 t0_out[i], t1_out[i]) and its SM id
 * (uint32 smid_out[i]): an SM's throughput is the bytes of its CTAs over its
 * span max(t1) - min(t0) in SM cycles.  Asynchronous on `stream`.
 */
int pchase_probe_smem_throughput(uint32_t ctas, uint32_t threads, uint32_t ilp, uint32_t iters,
                                 uint64_t *t0_out, uint64_t *t1_out, uint32_t *smid_out,
                                 pchase_stream_t stream);

/* ------------------------------------------------------------------ S7 */

/*
 * Learned inverse (a build extension, not in the paper): a 1-D convolutional
 * network maps a normalised mean-latency trace over the 512 points of a probe
 * plan to (capacity class, line-size class, ways class, policy), with an
 * exhaustive least-squares matcher as fallback and judge.  The trace model is
 * Sec. 4.1's t = t0 + t_m * r, r being each point's miss rate.
 *
 * Network: 4 x [conv1d k=5, stride 2, pad 2, 64 channels, GELU] (512 -> 32
 * positions), flatten 2048 -> FC 256 + GELU -> FC 31 logits, read as heads of
 * 17 (capacity), 4 (line size), 7 (ways), 3 (policy).  BF16 GEMM operands,
 * FP32 accumulation; FP32 master weights, Adam moments and gradients.  At
 * inference the 64-channel convolutions and FC + heads run on the tcgen05
 * tensor cores with TMEM accumulators, the first layer computed by producer
 * warps straight into the second layer's operand tiles.
 *
 * Buffers: the caller allocates `params` (pchase_inverse_param_bytes; its
 * first 4 * param_count bytes are the FP32 weights in layer order, each
 * layer's weight matrix [out][in] row-major then its bias; a convolution's
 * input column is kk * in_channels + channel) and `work`
 * (pchase_inverse_work_bytes), both device memory.  The handle only records
 * sizes and offsets.
 */
typedef struct pchase_inverse pchase_inverse;

/* max_batch in [1, 65536]: the largest batch a train step or one inference
 * chunk processes. */
int pchase_inverse_create(uint32_t max_batch, pchase_inverse **out);
void pchase_inverse_destroy(pchase_inverse *h);
uint64_t pchase_inverse_param_count(const pchase_inverse *h);
size_t pchase_inverse_param_bytes(const pchase_inverse *h);
size_t pchase_inverse_work_bytes(const pchase_inverse *h);
/* The leading part of `work` that pchase_inverse_infer and
 * pchase_inverse_classify use (status, inputs, activations, logits): a handle
 * made only for inference, whose max_batch sets its chunk (larger chunks run
 * faster), may allocate just this many bytes; pchase_inverse_train_step needs
 * all of pchase_inverse_work_bytes.  The parameter layout does not depend on
 * max_batch, so handles of different max_batch share one `params`. */
size_t pchase_inverse_infer_work_bytes(const pchase_inverse *h);

/* Byte offset in `work` of a device uint32 status word: pchase_inverse_infer,
 * _classify and _train_step clear it when called, and a tensor-core
 * completion wait that gives up (after 2 s) ORs PCHASE_DEV_TIMEOUT into it. */
size_t pchase_inverse_status_offset(const pchase_inverse *h);
/* Byte offset in `work` of convolution layer `layer`'s (0..3) BF16 output,
 * [B][positions][64] for the last chunk of the last forward pass; 0 for a
 * layer out of range.  Inference computes layers 1 and 2 in one kernel and
 * layers 3 and 4 in another, whose layer-1 and layer-3 outputs never leave
 * the SM, so the buffers of layers 0 and 2 hold the last training step's.
 * For inspection and tests. */
size_t pchase_inverse_activation_offset(const pchase_inverse *h, uint32_t layer);

/* Byte offset in `params` of one of its arrays, each pchase_inverse_param_count
 * entries in the weight order above: which = 0 the FP32 master weights, 1
 * their BF16 copies (the operands every product uses), 2 the FP32 gradient of
 * the last pchase_inverse_train_step (left in place by the step), 3 and 4 the
 * FP32 Adam moments m and v.  (size_t)-1 for another `which`.  For
 * checkpoints, inspection and tests. */
size_t pchase_inverse_param_offset(const pchase_inverse *h, uint32_t which);

/* Uniform init of every weight in +-sqrt(6 / fan_in) (SplitMix64 keyed on
 * seed and index), biases 0, Adam moments 0. */
int pchase_inverse_init(const pchase_inverse *h, void *params, uint64_t seed,
                        pchase_stream_t stream);

/*
 * Synthetic traces from a miss-rate table (device `rates`, n_geoms x 512
 * FP32) and per-geometry targets (device, n_geoms x 4 uint32 class labels).
 * Sample i (global number first + i) draws its geometry, t0, t1 = t0 * rho,
 * per-point Gaussian jitter and spikes from SplitMix64 keyed on (seed, number,
 * point); noise (host, 8 floats) = {t0_lo, t0_hi, rho_lo, rho_hi, sigma,
 * spike_probability, spike_lo, spike_hi}.  Outputs (device): x_out n x 512
 * FP32 in [0, 1] (min-max normalised), labels_out n x 4, truth_out n
 * geometry indices (may be NULL).
 */
int pchase_inverse_synth(const float *rates, const uint32_t *targets, uint32_t n_geoms,
                         uint64_t seed, uint64_t first, uint32_t n, const float *noise,
                         float *x_out, uint32_t *labels_out, uint32_t *truth_out,
                         pchase_stream_t stream);

/* One Adam step (lr, beta1 0.9, beta2 0.999, eps 1e-8; `step` counts from 0)
 * on the mean cross-entropy of the four heads over a batch of B <= max_batch
 * traces (device x, B x 512 FP32; labels B x 4).  The batch's mean loss is
 * added to *loss_accum (device float).  The gradient (parameter array 2) is
 * the chain rule through the network with BF16 operands and FP32 sums; the
 * forward pass, the backward pass and the weight gradients run on the
 * tcgen05 tensor cores (the one-channel first layer on CUDA cores).  Host
 * errors return a status; a tensor-core wait that gives up sets
 * PCHASE_DEV_TIMEOUT in the device status word (pchase_inverse_status_offset)
 * and leaves the parameters undefined. */
int pchase_inverse_train_step(const pchase_inverse *h, void *params, void *work, const float *x,
                              const uint32_t *labels, uint32_t B, float lr, uint32_t step,
                              float *loss_accum, pchase_stream_t stream);

/* Forward pass over n traces (device x, n x 512) in max_batch chunks:
 * pred_out n x 4 class indices, conf_out n (product of the heads' top softmax
 * probabilities), logits_out n x 31 FP32 (may be NULL). */
int pchase_inverse_infer(const pchase_inverse *h, const void *params, void *work, const float *x,
                         uint32_t n, uint32_t *pred_out, float *conf_out, float *logits_out,
                         pchase_stream_t stream);

/*
 * Exhaustive least-squares matcher (FP32): for each trace y (device, n x 512)
 * keep the points at or below its 507th smallest value (the 5 largest are the
 * spike allowance), fit y ~ alpha + beta * r_g for every geometry g (device
 * rates, n_geoms x 512) over the kept points, and take the smallest residual
 * (the plain variance of y when the fitted slope is not positive); equal
 * residuals go to the lower geometry index, so callers order the table
 * canonically.  best_out n indices, resid_out n residuals (may be NULL).
 * Work buffer (device): pchase_lsq_work_bytes(n).
 */
size_t pchase_lsq_work_bytes(uint32_t n);
int pchase_lsq_match(const float *rates, uint32_t n_geoms, const float *y, uint32_t n,
                     uint32_t *best_out, float *resid_out, void *work, pchase_stream_t stream);

/*
 * Learned prediction with fallback, all on the device: infer, map each
 * trace's four labels through label_to_cand (17*4*7*3 uint32, index
 * ((c*4 + b)*7 + w)*3 + p, 0xFFFFFFFF = no such geometry) to a geometry
 * index; traces whose confidence is below conf_thresh or whose labels name no
 * geometry are listed in fallback_list (count in *n_fallback) and resolved by
 * pchase_lsq_match.  cand_out n geometry indices.  Scratch (device):
 * pred_scratch n x 4, conf_out n, fallback_list n, fb_rows n x 512 FP32,
 * fb_idx n, lsq_work pchase_lsq_work_bytes(n).
 */
int pchase_inverse_classify(const pchase_inverse *h, const void *params, void *work,
                            const float *x, uint32_t n, const uint32_t *label_to_cand,
                            const float *rates, uint32_t n_geoms, float conf_thresh,
                            uint32_t *pred_scratch, float *conf_out, uint32_t *cand_out,
                            uint32_t *fallback_list, uint32_t *n_fallback, float *fb_rows,
                            uint32_t *fb_idx, void *lsq_work, pchase_stream_t stream);

/*
 * Miss-rate table of a candidates x points plan (the learned inverse's
 * latency model t = t0 + t_m r, Sec. 4.1, needs r per point): from the
 * simulator's counts (device, n_geoms x n_points x 2 uint64 as
 * pchase_sim_run writes them for a pairs == NULL plan, item g * n_points + p)
 * and the measured accesses per point (device, n_points uint64: length minus
 * warm-up), rates_out[g * n_points + p] (device float) = misses after warm-up
 * / measured, divided in double and rounded once; 0 where nothing is
 * measured.
 */
int pchase_miss_rates(const uint64_t *counts, uint32_t n_geoms, uint32_t n_points,
                      const uint64_t *measured, float *rates_out, pchase_stream_t stream);

/*
 * Answer classes of candidates under a plan: single-linkage groups of rows
 * of `rates` (device, n_geoms x n_points float) whose difference is at most
 * `tol` at every point (compared exactly in double; tol = 0 groups identical
 * rows).  rep_out[g] (device uint32) is the lowest index in g's group, so a
 * table sorted canonically names each group by its canonical member.  No
 * observation of mean latencies separates the members of one group.  Work
 * buffer (device): pchase_answer_classes_work_bytes(n_geoms), the adjacency
 * bit matrix.  n_geoms <= 65536 (ERANGE above).
 */
size_t pchase_answer_classes_work_bytes(uint32_t n_geoms);
int pchase_answer_classes(const float *rates, uint32_t n_geoms, uint32_t n_points, double tol,
                          uint32_t *rep_out, void *work, pchase_stream_t stream);

/*
 * A learned-inverse model the library owns, for callers that hold only a
 * weights blob.  inverse_load copies `weights` (HOST memory, exactly
 * 4 * pchase_inverse_param_count bytes of FP32 weights in the layer order
 * above, as a checkpoint of pchase_inverse_param_offset(h, 0) holds them)
 * into device memory it allocates on the current device, with their BF16
 * copies, a work area and fallback scratch for 4096 traces at a time; it is
 * synchronous.  inverse_free releases everything (NULL is a no-op).
 * Errors: EINVAL for a NULL argument or a wrong size, ENOMEM when an
 * allocation fails.
 */
typedef struct pchase_inverse_model pchase_inverse_model;
int inverse_load(const void *weights, size_t bytes, pchase_inverse_model **handle);
void inverse_free(pchase_inverse_model *handle);

/*
 * pchase_inverse_classify on a loaded model, its scratch held by the model:
 * n traces (device x, n x 512 FP32) in chunks of 4096; cand_out (device, n)
 * the geometry index of each trace, conf_out (device, n) the network's
 * confidence, *n_fallback (device uint32) how many traces the least-squares
 * matcher resolved.  label_to_cand, rates, n_geoms and conf_thresh as in
 * pchase_inverse_classify.  Calls on one model must not overlap on the GPU.
 */
int inverse_classify(const pchase_inverse_model *model, const float *x, uint32_t n,
                     const uint32_t *label_to_cand, const float *rates, uint32_t n_geoms,
                     float conf_thresh, uint32_t *cand_out, float *conf_out,
                     uint32_t *n_fallback, pchase_stream_t stream);

/* Last host-side failure of the S7 calls on this thread. */
const char *pchase_inverse_last_error(void);

/* ------------------------------------------------------------- library */

const char *pchase_last_error_string(void);
const char *pchase_version(void);
/* Number of SMs of the current device (0 if none). */
int pchase_device_sm_count(void);

#ifdef __cplusplus
}
#endif

#endif /* PCHASE_H */
