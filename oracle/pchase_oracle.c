/*
 * Plain CPU oracle for the fine-grained pointer-chase (P-chase) method of
 * Mei & Chu, "Dissecting GPU Memory Hierarchy through Microbenchmarking".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is deliberately slow and obvious.  It
 * shares no code, header, table or constant generator with the CUDA library
 * under paper_1509_02308_gb300/.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference arm may load it.
 *
 * Every function states the passage of the paper it follows.  Where the paper
 * is silent the function states the reading it takes.
 *
 * Units: array indices are 4-byte elements (Sec. 4.2 counts N and s in array
 * elements; Sec. 4.3 fixes an element at 4 bytes), so the byte address of
 * element j is 4*j.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ERANGE 2
#define OR_ENOMEM 3

#define OR_LRU 0
#define OR_FIFO 1
#define OR_RANDOM 2
#define OR_WEIGHTED 3
#define OR_REPLAY 4   /* oracle only: victims read off a transcript */

/* ------------------------------------------------------------------------ */
/* P-chase array and chain walk                                              */
/* ------------------------------------------------------------------------ */

/* Listing 1 (Sec. 4.1): element i of the array holds the index of the next
 * element to visit, i.e. (i + stride) mod array_size. */
int or_pchase_array(uint32_t n_elems, uint32_t stride_elems, uint32_t *A)
{
    if (n_elems == 0) return OR_EINVAL;
    for (uint32_t i = 0; i < n_elems; i++)
        A[i] = (uint32_t)(((uint64_t)i + stride_elems) % n_elems);
    return OR_OK;
}

/* The chase j = A[j] of Listings 2 and 3, started at j = 0.  trace[t] is the
 * index visited by access t (the index that is loaded, before the load
 * replaces j).  A chain that points outside [0, n_elems) is an error. */
int or_pchase_walk(const uint32_t *A, uint32_t n_elems, uint64_t len, uint32_t *trace)
{
    uint32_t j = 0;
    if (len > 0 && n_elems == 0) return OR_EINVAL;
    for (uint64_t t = 0; t < len; t++) {
        trace[t] = j;
        j = A[j];
        if (j >= n_elems) return OR_ERANGE;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers for the RANDOM policy                        */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the first output of the generator whose state is
 * x.  The state advances by the golden-ratio increment, then the value goes
 * through the two xor-shift-multiply rounds. */
uint64_t or_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Victim way of the k-th eviction (0-based) in set `set` of a RANDOM cache
 * with `ways` ways.  The paper gives no generator (Sec. 4.5 only reports
 * measured victim frequencies); the reading used here keys SplitMix64 on
 * (seed, set, k) so that the choice does not depend on the order in which
 * sets are simulated, and maps the high 32 bits onto [0, ways) by a
 * multiply-shift. */
uint32_t or_random_victim(uint64_t seed, uint32_t set, uint64_t k, uint32_t ways)
{
    uint64_t key = seed ^ ((uint64_t)set << 40) ^ k;
    uint64_t h = or_splitmix64(key);
    return (uint32_t)(((h >> 32) * (uint64_t)ways) >> 32);
}

/* Victim way of the k-th eviction (0-based) in set `set` under the weighted
 * policy the paper measures on the Fermi L1 data cache (Sec. 4.5): way 2 is
 * replaced once every two misses and is three times as likely to go as each
 * other way (1/6, 1/2, 1/6, 1/6 on four ways).  The reading used here: the
 * evictions k = 0, 2, 4, ... take way 2; the others take one of the remaining
 * ways uniformly, keyed like RANDOM on (seed, set, k), the high 32 bits
 * mapped onto [0, ways - 1) and stepped past way 2.  Needs ways >= 3. */
uint32_t or_weighted_victim(uint64_t seed, uint32_t set, uint64_t k, uint32_t ways)
{
    if (k % 2 == 0) return 2;
    uint64_t key = seed ^ ((uint64_t)set << 40) ^ k;
    uint64_t h = or_splitmix64(key);
    uint32_t r = (uint32_t)(((h >> 32) * (uint64_t)(ways - 1)) >> 32);
    return r < 2 ? r : r + 1;
}

/* ------------------------------------------------------------------------ */
/* Set-associative cache                                                     */
/* ------------------------------------------------------------------------ */

/* Assumption 1 (Sec. 4.1): T sets of `ways` lines of b bytes, T*ways*b = C.
 * The oracle also accepts b as any power of two of at least 4 bytes. */
static int or_geom_ok(uint32_t C, uint32_t b, uint32_t ways, uint32_t T)
{
    if (C == 0 || b < 4 || ways == 0 || T == 0) return 0;
    if ((b & (b - 1)) != 0) return 0;
    if ((uint64_t)T * ways * b != C) return 0;
    return 1;
}

/*
 * Replays `trace` (element indices) through a cache of capacity C bytes, line
 * size b bytes, `ways` ways and T sets, starting with every line invalid.
 * miss_out[t] = 1 if access t misses, else 0.
 *
 * The model is the classical one of Sec. 4.1 (Assumptions 1-3, Fig. 2):
 *   byte address = 4 * index;  line = address / b;
 *   set = (line >> mapping) mod T;  a way holds a whole line number.
 * mapping = 0: the set bits sit right above the offset bits, which for T a
 * power of two is Assumption 2 and for other T is its modular reading.
 * mapping = m > 0: the set bits sit m bits higher, as the paper finds for the
 * texture L1 cache (Sec. 4.3: bits 7-8 with 32-byte lines, m = 2), so 2^m
 * consecutive lines share a set.
 * An access hits when its line is held by a valid way of its set.  On a miss
 * the line goes into the lowest-numbered invalid way; when the set is full a
 * victim is chosen:
 *   LRU      (Assumption 3): the way whose last use is oldest;
 *   FIFO     : the way whose fill is oldest;
 *   RANDOM   : or_random_victim(seed, set, k), k = evictions so far in the set;
 *   WEIGHTED : or_weighted_victim(seed, set, k), k as for RANDOM;
 *   REPLAY   : victims[e], e = evictions so far in the whole cache (the way
 *              numbers a caller read off a transcript such as Fig. 9).
 * Only LRU records a use on a hit.  When evict_set / evict_way are given, the
 * set and way of the first `evict_cap` evictions are written there and the
 * number of evictions to *n_evict.
 *
 * filter (NULL: every access): the cache sees only the accesses t with
 * filter[t] != 0, in order; the others neither hit nor miss (miss_out 0).
 * With filter = the misses of a level above, this is the next level of the
 * hierarchy of Sec. 3 (an L1 miss goes to L2; an L1 hit never reaches it), and
 * with pages for lines (b = page size) it is a TLB level (Sec. 4.4).
 */
int or_cache_sim_ext(uint32_t C, uint32_t b, uint32_t ways, uint32_t T, int policy,
                     uint64_t seed, uint32_t mapping, const uint32_t *trace, uint64_t len,
                     const uint8_t *filter,
                     const uint32_t *victims, uint64_t n_victims,
                     uint8_t *miss_out, uint32_t *final_lines /* T*ways or NULL */,
                     uint32_t *evict_set, uint32_t *evict_way, uint64_t evict_cap,
                     uint64_t *n_evict)
{
    if (!or_geom_ok(C, b, ways, T)) return OR_EINVAL;
    if (policy < OR_LRU || policy > OR_REPLAY) return OR_EINVAL;
    if (policy == OR_WEIGHTED && ways < 3) return OR_EINVAL;
    if (mapping > 16) return OR_EINVAL;
    uint64_t nlines = (uint64_t)T * ways;
    uint64_t *held = (uint64_t *)malloc(nlines * sizeof(uint64_t));
    uint8_t *valid = (uint8_t *)calloc(nlines, 1);
    uint64_t *last_use = (uint64_t *)malloc(nlines * sizeof(uint64_t));
    uint64_t *filled_at = (uint64_t *)malloc(nlines * sizeof(uint64_t));
    uint64_t *evictions = (uint64_t *)calloc(T, sizeof(uint64_t));
    if (!held || !valid || !last_use || !filled_at || !evictions) {
        free(held); free(valid); free(last_use); free(filled_at); free(evictions);
        return OR_ENOMEM;
    }
    uint64_t replay_next = 0, n_ev = 0;
    int rc = OR_OK;
    for (uint64_t t = 0; t < len; t++) {
        if (filter && !filter[t]) {
            /* the access never reaches this cache */
            miss_out[t] = 0;
            continue;
        }
        uint64_t addr = 4ull * trace[t];
        uint64_t line = addr / b;
        uint32_t set = (uint32_t)((line >> mapping) % T);
        uint64_t base = (uint64_t)set * ways;
        int hit_way = -1;
        for (uint32_t w = 0; w < ways; w++) {
            if (valid[base + w] && held[base + w] == line) { hit_way = (int)w; break; }
        }
        if (hit_way >= 0) {
            miss_out[t] = 0;
            if (policy == OR_LRU) last_use[base + hit_way] = t;
            continue;
        }
        miss_out[t] = 1;
        int64_t victim = -1;
        for (uint32_t w = 0; w < ways; w++) {
            if (!valid[base + w]) { victim = w; break; }
        }
        if (victim < 0) {
            if (policy == OR_LRU) {
                victim = 0;
                for (uint32_t w = 1; w < ways; w++)
                    if (last_use[base + w] < last_use[base + victim]) victim = w;
            } else if (policy == OR_FIFO) {
                victim = 0;
                for (uint32_t w = 1; w < ways; w++)
                    if (filled_at[base + w] < filled_at[base + victim]) victim = w;
            } else if (policy == OR_RANDOM) {
                victim = or_random_victim(seed, set, evictions[set], ways);
            } else if (policy == OR_WEIGHTED) {
                victim = or_weighted_victim(seed, set, evictions[set], ways);
            } else {
                if (replay_next >= n_victims) { rc = OR_ERANGE; break; }
                victim = victims[replay_next++];
                if ((uint64_t)victim >= ways) { rc = OR_ERANGE; break; }
            }
            evictions[set]++;
            if (evict_set && evict_way && n_ev < evict_cap) {
                evict_set[n_ev] = set;
                evict_way[n_ev] = (uint32_t)victim;
            }
            n_ev++;
        }
        held[base + victim] = line;
        valid[base + victim] = 1;
        last_use[base + victim] = t;
        filled_at[base + victim] = t;
    }
    if (final_lines) {
        /* line number held by each way, 0xFFFFFFFF for an invalid way */
        for (uint64_t i = 0; i < nlines; i++)
            final_lines[i] = valid[i] ? (uint32_t)held[i] : 0xFFFFFFFFu;
    }
    if (n_evict) *n_evict = n_ev;
    free(held); free(valid); free(last_use); free(filled_at); free(evictions);
    return rc;
}

/* The standard mapping (mapping = 0) without an eviction record. */
int or_cache_sim(uint32_t C, uint32_t b, uint32_t ways, uint32_t T, int policy,
                 uint64_t seed, const uint32_t *trace, uint64_t len,
                 const uint32_t *victims, uint64_t n_victims,
                 uint8_t *miss_out, uint32_t *final_tags /* T*ways or NULL */)
{
    return or_cache_sim_ext(C, b, ways, T, policy, seed, 0, trace, len, NULL, victims,
                            n_victims, miss_out, final_tags, NULL, NULL, 0, NULL);
}

/*
 * A cache with unequal sets: the L2 TLB of Sec. 4.4 (Fig. 9), whose miss
 * count grows set by set as N grows, with one large set of 17 entries and six
 * of 8.  The paper gives the set sizes but not the page-to-set rule.  Reading:
 * the M = T * a + extra lines of capacity are residues of line mod M; residue
 * r < T * a goes to set r mod T, the other `extra` residues to set 0, so set 0
 * holds a + extra lines and the others a.  A chain of n > M lines then
 * overflows set 0 first (n = M + 1) and then sets 1, 2, ... one line at a
 * time, the order Fig. 9's steps show.  With extra = 0 this is set = line mod
 * T.  LRU or FIFO; a miss fills the lowest invalid way of its set, else evicts
 * the oldest use (LRU) or fill (FIFO) among the set's ways.  filter (or NULL)
 * flags the accesses that reach this cache, as in or_cache_sim_ext.
 */
int or_cache_sim_uneq(uint32_t C, uint32_t b, uint32_t ways, uint32_t T, uint32_t extra,
                      int policy, const uint32_t *trace, uint64_t len, const uint8_t *filter,
                      uint8_t *miss_out)
{
    if (b < 4 || (b & (b - 1)) || ways == 0 || T == 0) return OR_EINVAL;
    if (policy != OR_LRU && policy != OR_FIFO) return OR_EINVAL;
    uint64_t M = (uint64_t)T * ways + extra;
    if (M * b != C) return OR_EINVAL;
    uint32_t wmax = ways + extra;
    uint64_t nslots = (uint64_t)T * wmax;
    uint64_t *held = (uint64_t *)malloc(nslots * sizeof(uint64_t));
    uint8_t *valid = (uint8_t *)calloc(nslots, 1);
    uint64_t *stamp = (uint64_t *)malloc(nslots * sizeof(uint64_t));
    if (!held || !valid || !stamp) {
        free(held); free(valid); free(stamp);
        return OR_ENOMEM;
    }
    for (uint64_t t = 0; t < len; t++) {
        if (filter && !filter[t]) {
            /* the access never reaches this cache */
            miss_out[t] = 0;
            continue;
        }
        uint64_t line = 4ull * trace[t] / b;
        uint64_t r = line % M;
        uint32_t set = r < (uint64_t)T * ways ? (uint32_t)(r % T) : 0;
        uint32_t nw = set == 0 ? wmax : ways;
        uint64_t base = (uint64_t)set * wmax;
        int64_t hit_way = -1;
        for (uint32_t w = 0; w < nw; w++)
            if (valid[base + w] && held[base + w] == line) { hit_way = w; break; }
        if (hit_way >= 0) {
            miss_out[t] = 0;
            if (policy == OR_LRU) stamp[base + hit_way] = t;
            continue;
        }
        miss_out[t] = 1;
        int64_t victim = -1;
        for (uint32_t w = 0; w < nw; w++)
            if (!valid[base + w]) { victim = w; break; }
        if (victim < 0) {
            victim = 0;
            for (uint32_t w = 1; w < nw; w++)
                if (stamp[base + w] < stamp[base + victim]) victim = w;
        }
        held[base + victim] = line;
        valid[base + victim] = 1;
        stamp[base + victim] = t;  /* last use (LRU) = fill (FIFO) here */
    }
    free(held); free(valid); free(stamp);
    return OR_OK;
}

/* Miss counts of one replay: total, and after the first `warmup` accesses. */
int or_cache_sim_counts(uint32_t C, uint32_t b, uint32_t ways, uint32_t T, int policy,
                        uint64_t seed, const uint32_t *trace, uint64_t len,
                        uint64_t warmup, uint64_t *total_out, uint64_t *after_out)
{
    uint8_t *m = (uint8_t *)malloc(len ? len : 1);
    if (!m) return OR_ENOMEM;
    int rc = or_cache_sim(C, b, ways, T, policy, seed, trace, len, NULL, 0, m, NULL);
    uint64_t tot = 0, aft = 0;
    for (uint64_t t = 0; t < len; t++) {
        tot += m[t];
        if (t >= warmup) aft += m[t];
    }
    *total_out = tot;
    *after_out = aft;
    free(m);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Latency -> hit/miss                                                       */
/* ------------------------------------------------------------------------ */

static int or_cmp_float(const void *x, const void *y)
{
    float a = *(const float *)x, b = *(const float *)y;
    return (a > b) - (a < b);
}

/*
 * Two-level split of a latency trace into hits and misses.  Sec. 4.2 reads
 * hits and misses off the recorded latencies (t_avg = t0 + t_m * r, Sec. 4.1)
 * but states no rule.  Reading: sort the latencies, set aside the top
 * floor(n/200) values (0.5 %, the spike allowance), find the largest gap
 * between consecutive kept values (the first one on ties) and cut at its
 * midpoint (lo + hi) * 0.5f computed in float; a latency above the cut is a
 * miss.  With no gap (all kept values equal) every access is a hit.
 */
int or_classify(const float *lat, uint64_t n, uint8_t *miss_out, float *thresh_out)
{
    if (n == 0) { if (thresh_out) *thresh_out = 0.0f; return OR_OK; }
    float *v = (float *)malloc(n * sizeof(float));
    if (!v) return OR_ENOMEM;
    memcpy(v, lat, n * sizeof(float));
    qsort(v, n, sizeof(float), or_cmp_float);
    uint64_t keep = n - n / 200;
    float best_gap = 0.0f, thr = 0.0f;
    int found = 0;
    for (uint64_t i = 0; i + 1 < keep; i++) {
        float g = v[i + 1] - v[i];
        if (g > best_gap) { best_gap = g; thr = (v[i] + v[i + 1]) * 0.5f; found = 1; }
    }
    if (!found) thr = v[keep - 1];
    for (uint64_t t = 0; t < n; t++) miss_out[t] = lat[t] > thr ? 1 : 0;
    if (thresh_out) *thresh_out = thr;
    free(v);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Exhaustive matcher                                                        */
/* ------------------------------------------------------------------------ */

/*
 * The two-stage procedure of Fig. 6 (Sec. 4.2) reads C, then b, then T, then
 * the policy off the miss pattern of chosen (N, s) runs.  Its mechanised form:
 * replay every plan trace through every candidate geometry and count the
 * accesses whose simulated outcome differs from the observed one (Hamming
 * distance).  dist_out[g] is that count for candidate g over all traces.
 *
 * cand: n_cand rows of {C, b, ways, T, policy} (uint32) plus seeds[g].
 * traces: all plan traces back to back; offsets[p]..offsets[p+1] is trace p.
 * observed: one byte per access (1 = miss), same layout as traces.
 */
int or_match(const uint32_t *cand, const uint64_t *seeds, uint32_t n_cand,
             const uint32_t *traces, const uint64_t *offsets, uint32_t n_traces,
             const uint8_t *observed, uint64_t *dist_out)
{
    uint64_t maxlen = 0;
    for (uint32_t p = 0; p < n_traces; p++)
        if (offsets[p + 1] - offsets[p] > maxlen) maxlen = offsets[p + 1] - offsets[p];
    uint8_t *m = (uint8_t *)malloc(maxlen ? maxlen : 1);
    if (!m) return OR_ENOMEM;
    int rc = OR_OK;
    for (uint32_t g = 0; g < n_cand && rc == OR_OK; g++) {
        const uint32_t *c = cand + 5 * (uint64_t)g;
        uint64_t d = 0;
        for (uint32_t p = 0; p < n_traces; p++) {
            uint64_t len = offsets[p + 1] - offsets[p];
            rc = or_cache_sim(c[0], c[1], c[2], c[3], (int)c[4], seeds[g],
                              traces + offsets[p], len, NULL, 0, m, NULL);
            if (rc != OR_OK) break;
            for (uint64_t t = 0; t < len; t++) d += (m[t] != observed[offsets[p] + t]);
        }
        dist_out[g] = d;
    }
    free(m);
    return rc;
}

/*
 * Canonical pick among candidates.  Several geometries can give identical
 * outcomes on a plan (on a uniform chain with stride s >= b every line size up
 * to s behaves alike, and LRU and FIFO agree on any uniform chain), so the
 * pick is made in a fixed order: smallest distance, then policy LRU < FIFO <
 * RANDOM, then the largest b, then the fewest ways, then the smallest C.
 * Returns the index of the pick (or n_cand when n_cand is 0) and the number of
 * candidates at the smallest distance in *n_best.
 */
uint32_t or_canonical_pick(const uint32_t *cand, const uint64_t *dist, uint32_t n_cand,
                           uint32_t *n_best)
{
    uint32_t best = n_cand, count = 0;
    for (uint32_t g = 0; g < n_cand; g++) {
        if (best == n_cand) { best = g; count = 1; continue; }
        const uint32_t *x = cand + 5 * (uint64_t)g, *y = cand + 5 * (uint64_t)best;
        if (dist[g] != dist[best]) {
            if (dist[g] < dist[best]) { best = g; count = 1; }
            continue;
        }
        count++;
        int better = 0;
        if (x[4] != y[4]) better = x[4] < y[4];
        else if (x[1] != y[1]) better = x[1] > y[1];
        else if (x[2] != y[2]) better = x[2] < y[2];
        else if (x[0] != y[0]) better = x[0] < y[0];
        if (better) best = g;
    }
    if (n_best) *n_best = count;
    return best;
}

/* ------------------------------------------------------------------------ */
/* Shared-memory banks                                                       */
/* ------------------------------------------------------------------------ */

/*
 * Conflict degree of one warp request (Sec. 6.2, Fig. 14): word w lives in
 * bank w mod n_banks; lanes that read the same word are served together
 * (broadcast, a reading the paper does not state), so the degree is the
 * largest number of distinct words any one bank must deliver.
 */
uint32_t or_bank_degree(const uint32_t *word_addr, uint32_t n_lanes, uint32_t n_banks)
{
    uint32_t best = 0;
    for (uint32_t bank = 0; bank < n_banks; bank++) {
        uint32_t distinct = 0;
        for (uint32_t i = 0; i < n_lanes; i++) {
            if (word_addr[i] % n_banks != bank) continue;
            int seen = 0;
            for (uint32_t j = 0; j < i; j++)
                if (word_addr[j] == word_addr[i]) { seen = 1; break; }
            if (!seen) distinct++;
        }
        if (distinct > best) best = distinct;
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* Mean-latency model                                                        */
/* ------------------------------------------------------------------------ */

/* Sec. 4.1: t_avg = t0 * (1 - r) + (t0 + t_m) * r = t0 + t_m * r. */
double or_mean_latency(double t0, double tm, double r)
{
    return t0 + tm * r;
}
