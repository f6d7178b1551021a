"""Pins for the CPU oracle: the paper's worked examples, closed forms,
special cases and brute force.  None of these calls a GPU."""
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from conftest import golden
from paper_1509_02308_gb300 import workloads as W


def steady_misses_per_pass(C, b, a, T, n_elems, s_elems, passes=3, policy=oracle.LRU):
    per = n_elems // math.gcd(n_elems, s_elems)
    tr = oracle.pchase_trace(n_elems, s_elems, per * passes)
    m = oracle.cache_sim(C, b, a, T, policy, tr)
    return [int(m[p * per:(p + 1) * per].sum()) for p in range(passes)], m, per


# ------------------------------------------------------------------ chain walk
def test_listing1_chain_closed_form():
    # Listing 1 walked from j = 0 visits (t * s) mod N.
    for n, s in [(13, 1), (100, 7), (4096, 32), (96, 64), (1, 1), (5, 5)]:
        tr = oracle.pchase_trace(n, s, 3 * n + 1)
        t = np.arange(tr.size, dtype=np.uint64)
        assert np.array_equal(tr.astype(np.uint64), (t * s) % n)


def test_walk_rejects_chain_outside_array():
    A = np.array([1, 2, 7], dtype=np.uint32)
    with pytest.raises(oracle.OracleError):
        oracle.pchase_walk(A, 10)


# ------------------------------------------------------------------- Fig. 3
def test_fig3_periodic_pattern():
    g = golden("fig3_periodic.json")
    c = g["cache"]
    wb = c["word_bytes"]
    C, b = c["words"] * wb, c["line_words"] * wb
    n = g["array_words"]
    tr = oracle.pchase_trace(n, g["stride_words"], n * 6)
    m = oracle.cache_sim(C, b, c["ways"], c["sets"], oracle.LRU, tr)
    want = np.zeros(n, dtype=np.uint8)
    want[np.array(g["steady_pass_misses_1based_words"]) - 1] = 1
    for p in range(1, 6):
        assert np.array_equal(m[p * n:(p + 1) * n], want), p
    # the pattern repeats with period 13 = the array length
    assert np.array_equal(m[n:2 * n], m[4 * n:5 * n])


# ------------------------------------------------------------------- Fig. 9
def _fig9_trace(g):
    line_elems = 128 // 4
    lines = g["initial_ways"] + g["reads"]
    return np.array([x * line_elems for x in lines], dtype=np.uint32)


def test_fig9_transcript_replay():
    g = golden("fig9_transcript.json")
    tr = _fig9_trace(g)
    victims = np.array(g["replaced_way_per_miss_1based"], dtype=np.uint32) - 1
    m, fin = oracle.cache_sim(4 * 128, 128, 4, 1, oracle.REPLAY, tr, victims=victims,
                              want_final=True)
    k = len(g["initial_ways"])
    assert m[:k].tolist() == [1] * k  # the four fills
    got = "".join("M" if x else "H" for x in m[k:])
    assert got == g["status"]
    assert [int(x) // 1 for x in fin] == g["final_ways"]


def test_fig9_under_lru_everything_misses():
    g = golden("fig9_transcript.json")
    tr = _fig9_trace(g)
    m = oracle.cache_sim(4 * 128, 128, 4, 1, oracle.LRU, tr)
    assert m[len(g["initial_ways"]):].all()


def test_replay_runs_out_of_victims():
    g = golden("fig9_transcript.json")
    with pytest.raises(oracle.OracleError):
        oracle.cache_sim(512, 128, 4, 1, oracle.REPLAY, _fig9_trace(g),
                         victims=np.array([1], dtype=np.uint32))


# ------------------------------------------------------ Eq. (2), config 1
def test_eq2_exact_over_config1():
    g = golden("closed_forms.json")["config1"]
    C, b, a, T = g["C"], g["b"], g["ways"], g["sets"]
    tot_acc = tot_miss = 0
    geo, runs = W.config1()
    assert len(runs) == g["traces"]
    for run in runs:
        nb = run.n_elems * 4
        k = (nb - C) // b
        per, m, pp = steady_misses_per_pass(C, b, a, T, run.n_elems, run.stride, passes=3)
        lines = nb // b
        assert per[0] == lines  # the warm-up pass misses every line once
        want = 0 if k <= 0 else (k * (a + 1) if k <= T else lines)
        assert per[1] == want and per[2] == want, (nb, per)
        tot_acc += m.size
        tot_miss += int(m.sum())
    assert tot_acc == g["accesses"]
    assert tot_miss == g["misses"]


def test_step2_line_size_jump():
    g = golden("closed_forms.json")["step2"]
    C, b, a, T = g["C"], g["b"], g["ways"], g["sets"]
    s = g["stride_bytes"] // 4
    for nb_str, want in g["misses_per_pass"].items():
        per, _, _ = steady_misses_per_pass(C, b, a, T, int(nb_str) // 4, s)
        assert per[1] == want and per[2] == want, (nb_str, per)
    # step 1: C is the largest N at which every access after warm-up hits
    for nb in (C - 4, C):
        per, _, _ = steady_misses_per_pass(C, b, a, T, nb // 4, s)
        assert per[1] == 0 and per[2] == 0


def test_eq1_saavedra_rates():
    C, b, a, T = 1024, 64, 2, 8
    n_bytes = 64 * 1024
    for s_bytes in (4, 8, 16, 32):
        per, _, pp = steady_misses_per_pass(C, b, a, T, n_bytes // 4, s_bytes // 4)
        assert per[2] * b == pp * s_bytes  # rate s / b
    for s_bytes in (64, 128, 1024, 8192, 16384):  # b <= s < N / a
        per, _, pp = steady_misses_per_pass(C, b, a, T, n_bytes // 4, s_bytes // 4)
        assert per[2] == pp
    per, _, pp = steady_misses_per_pass(C, b, a, T, n_bytes // 4, n_bytes // a // 4)
    assert per[2] == 0  # s = N / a: the a visited lines share one set and fit


def test_texture_l1_sweep_fig5_shape():
    # Sec. 4.3: 12 KB, 32 B lines, 4 sets of 96 lines; s = 32 B, N = 12 KB..12.5 KB.
    t4 = golden("table4_geometries.json")["caches"][1]
    C, b, T = t4["C"], t4["b"], t4["T"]
    a = C // (T * b)
    assert a == 96
    prev = None
    for k in range(0, 17):
        nb = C + k * b
        per, _, _ = steady_misses_per_pass(C, b, a, T, nb // 4, b // 4)
        want = 0 if k == 0 else (k * (a + 1) if k <= T else nb // b)
        assert per[2] == want
        if prev is not None:
            assert per[2] >= prev
        prev = per[2]


def test_texture_l1_bits_7_8_mapping_sweep():
    """Sec. 4.3: the texture L1 cache (12 KB, 32 B lines, 4 sets of 96) takes its
    set from address bits 7-8, so each 128-byte block (4 lines) sits in one set
    (mapping = 2 line bits above the offset).  Under LRU a set cycling through
    n > 96 lines misses on every access and any other set hits, so with
    N = 12 KB + d lines (s = 32 B) set i holds 96 + clamp(d - 4i, 0, 4) lines."""
    C, b, T, a = 12 * 1024, 32, 4, 96
    for d in range(0, 17):
        nb = C + d * b
        n_elems = nb // 4
        tr = oracle.pchase_trace(n_elems, b // 4, 3 * (nb // b))
        m = oracle.cache_sim(C, b, a, T, oracle.LRU, tr, mapping=2)
        per = nb // b
        counts = [a + min(max(d - 4 * i, 0), 4) for i in range(T)]
        want = sum(c for c in counts if c > a)
        assert m[2 * per:].sum() == want, d
        # the standard mapping spreads the same lines one per set instead
        ms = oracle.cache_sim(C, b, a, T, oracle.LRU, tr)
        want_std = 0 if d == 0 else (d * (a + 1) if d <= T else per)
        assert ms[2 * per:].sum() == want_std, d
    # read-only / texture cache: above 12.5 KB every access misses (Sec. 4.3)
    for kb in (12.75, 16, 24, 60):
        nb = int(kb * 1024)
        tr = oracle.pchase_trace(nb // 4, b // 4, 3 * (nb // b))
        m = oracle.cache_sim(C, b, a, T, oracle.LRU, tr, mapping=2)
        assert m[nb // b:].all(), kb


def test_mapping_zero_is_the_standard_mapping():
    for g in W.random_small_geoms(30, seed=21, max_lines=32):
        tr = W.random_index_trace(400, g.C // 4 * 3, seed=g.seed % 977)
        a = oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr, seed=g.seed)
        b = oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr, seed=g.seed, mapping=0)
        assert np.array_equal(a, b)


# --------------------------------------------------------------- weighted
def test_weighted_policy_fermi_l1_properties():
    """Sec. 4.5 (Fermi L1 data cache, 16 KB, 128 B lines, 4 ways, 32 sets): way 2
    is replaced once every two misses, and the four ways go with probabilities
    1/6, 1/2, 1/6, 1/6."""
    from scipy.stats import chisquare
    C, b, a, T = 16384, 128, 4, 32
    for seed in (1, 7, 0xFE12):
        n = 129 * b // 4  # 129 lines: one line over, all misses in one set
        tr = oracle.pchase_trace(n, b // 4, 400 * 129)
        m, es, ew = oracle.cache_sim(C, b, a, T, oracle.WEIGHTED, tr, seed=seed,
                                     want_evictions=True)
        assert set(es.tolist()) == {0}  # only the overflowing set evicts
        assert (ew[0::2] == 2).all()    # every other eviction takes way 2
        assert (ew[1::2] != 2).all()
        cnt = np.bincount(ew[1::2], minlength=4)
        assert chisquare(cnt[[0, 1, 3]]).pvalue > 1e-3
        assert abs((ew == 2).mean() - 0.5) <= 1.0 / len(ew)
        # the 129th line sometimes misses and sometimes hits (Fig. 9's text),
        # and the set misses less often than under LRU, where all of its
        # accesses miss
        pos = np.arange(len(tr))
        late = pos >= 2 * 129
        is128 = (tr // (b // 4)) == 128
        assert m[late & is128].any() and not m[late & is128].all()
        ml = oracle.cache_sim(C, b, a, T, oracle.LRU, tr)
        set0 = (tr // (b // 4)) % T == 0
        assert ml[late & set0].all() and m[late & set0].mean() < 1.0


def test_weighted_policy_needs_three_ways():
    tr = np.arange(10, dtype=np.uint32)
    with pytest.raises(oracle.OracleError):
        oracle.cache_sim(64, 32, 2, 1, oracle.WEIGHTED, tr)


# ------------------------------------------------------------ hierarchy
def _lvl(C, b, ways, T, policy=oracle.LRU, seed=0):
    return dict(C=C, b=b, ways=ways, T=T, policy=policy, seed=seed)


def test_filter_all_ones_is_unfiltered_and_all_zeros_sees_nothing():
    for g in W.random_small_geoms(20, seed=31, max_lines=32):
        tr = W.random_index_trace(500, g.C // 4 * 3, seed=g.seed % 911)
        a = oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr, seed=g.seed)
        b = oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr, seed=g.seed,
                             filter=np.ones(tr.size, np.uint8))
        z = oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr, seed=g.seed,
                             filter=np.zeros(tr.size, np.uint8))
        assert np.array_equal(a, b) and not z.any()


def test_filtered_run_is_the_run_of_the_kept_accesses():
    # a lower level sees exactly the subsequence the level above lets through
    rng = np.random.Generator(np.random.PCG64(8))
    for g in W.random_small_geoms(30, seed=32, max_lines=32):
        tr = W.random_index_trace(700, g.C // 4 * 4, seed=g.seed % 977)
        keep = (rng.random(tr.size) < 0.4).astype(np.uint8)
        got = oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr, seed=g.seed, filter=keep)
        sub = oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr[keep == 1], seed=g.seed)
        want = np.zeros(tr.size, np.uint8)
        want[keep == 1] = sub
        assert np.array_equal(got, want)


def test_l2_behind_a_fitting_l1_takes_only_compulsory_misses():
    """N <= C1: the L1 misses each line once; an L2 with lines b2 = f * b1 then
    misses once per L2 line of the array and hits the other f - 1 L1 lines."""
    for (b1, f) in ((32, 1), (32, 2), (64, 4)):
        l1 = _lvl(4096, b1, 4, 4096 // (4 * b1))
        l2 = _lvl(65536, b1 * f, 8, 65536 // (8 * b1 * f))
        for nb in (1024, 3000, 4096):
            n = nb // 4
            tr = oracle.pchase_trace(n, 1, 3 * n)
            m1, m2 = oracle.hierarchy([l1, l2], tr)
            lines1 = -(-nb // b1)
            lines2 = -(-nb // (b1 * f))
            assert m1.sum() == lines1 and m1[n:].sum() == 0
            assert m2.sum() == lines2 and m2[n:].sum() == 0
            assert not (m2 & (1 - m1)).any()  # L2 sees only L1 misses


def test_tlb_cascade_behind_a_thrashing_l1_tlb():
    """Sec. 4.4: the L1 TLB is 16-way fully associative with 2 MB pages.  A
    chain at s = 2 MB over 16 + k pages cycles through more pages than it
    holds, so under LRU every access misses it and the L2 TLB sees the whole
    stream: it then behaves as a lone cache (here 7 sets x 8 ways, LRU: a set
    cycling through more than 8 pages misses on every access)."""
    page = 2 << 20
    l1 = _lvl(16 * page, page, 16, 1)
    l2 = _lvl(56 * page, page, 8, 7)
    for n_pages in (17, 20, 40, 56, 57, 64, 70):
        n = n_pages * page // 4
        tr = oracle.pchase_trace(n, page // 4, 4 * n_pages)
        m1, m2 = oracle.hierarchy([l1, l2], tr)
        assert m1[n_pages:].all()
        lone = oracle.cache_sim(l2["C"], l2["b"], 8, 7, oracle.LRU, tr)
        assert np.array_equal(m2, lone)
        per_set = [len(range(s, n_pages, 7)) for s in range(7)]
        assert m2[n_pages:2 * n_pages].sum() == sum(c for c in per_set if c > 8)
    # 16 pages or fewer: after one pass every access hits the L1 TLB and the
    # L2 TLB sees only the first touches
    for n_pages in (1, 8, 16):
        n = n_pages * page // 4
        tr = oracle.pchase_trace(n, page // 4, 4 * n_pages)
        m1, m2 = oracle.hierarchy([l1, l2], tr)
        assert m1[n_pages:].sum() == 0 and m2.sum() == n_pages


def test_bruteforce_two_level_hierarchy():
    rng = np.random.Generator(np.random.PCG64(99))
    n = 0
    for _ in range(300):
        b1 = int(rng.choice([4, 8]))
        a1, T1 = int(rng.integers(1, 4)), int(rng.integers(1, 4))
        b2 = b1 * int(rng.choice([1, 2]))
        a2, T2 = int(rng.integers(1, 5)), int(rng.integers(1, 5))
        p1, p2 = int(rng.integers(0, 3)), int(rng.integers(0, 3))
        L = int(rng.integers(1, 60))
        tr = rng.integers(0, 4 * a2 * T2 * b2 // 4 + 2, size=L).astype(np.uint32)
        m1, m2 = oracle.hierarchy([_lvl(a1 * T1 * b1, b1, a1, T1, p1, 3),
                                   _lvl(a2 * T2 * b2, b2, a2, T2, p2, 4)], tr)
        w1 = _list_model(a1 * T1 * b1, b1, a1, T1, p1, 3, tr)
        keep = w1 == 1
        w2 = np.zeros(L, np.uint8)
        w2[keep] = _list_model(a2 * T2 * b2, b2, a2, T2, p2, 4, tr[keep])
        assert np.array_equal(m1, w1) and np.array_equal(m2, w2)
        n += 1
    assert n == 300


# --------------------------------------------------------------- invariants
def test_all_hits_after_warmup_when_array_fits():
    for g in W.random_small_geoms(40, seed=11, max_lines=32):
        for s in (1, 2, 3):
            n = g.C // 4  # N = C elements' worth of bytes
            tr = oracle.pchase_trace(n, s, 4 * n)
            m = oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr, seed=g.seed)
            per = n // math.gcd(n, s)
            assert m[per:].sum() == 0, g


def test_lru_equals_fifo_on_uniform_chains():
    for g in W.random_small_geoms(60, seed=5, max_lines=48, policies=(W.LRU,)):
        for nmul, s in ((1.5, 1), (2.0, 3), (1.25, 2), (3.0, 5)):
            n = max(1, int(g.C // 4 * nmul))
            tr = oracle.pchase_trace(n, s, 3 * n)
            a = oracle.cache_sim(g.C, g.b, g.ways, g.sets, oracle.LRU, tr)
            f = oracle.cache_sim(g.C, g.b, g.ways, g.sets, oracle.FIFO, tr)
            assert np.array_equal(a, f)


def test_lru_differs_from_fifo_on_retouch_chain():
    # a hot line re-read between streaming lines stays under LRU, leaves under FIFO
    b = 16
    C, a, T = 4 * b, 4, 1
    hot = 0
    stream = [(i + 1) * (b // 4) for i in range(8)]
    tr = []
    for p in range(4):
        for x in stream:
            tr += [hot, x]
    tr = np.array(tr, dtype=np.uint32)
    ml = oracle.cache_sim(C, b, a, T, oracle.LRU, tr)
    mf = oracle.cache_sim(C, b, a, T, oracle.FIFO, tr)
    assert ml[2::2].sum() == 0  # hot re-reads always hit under LRU
    assert mf[2::2].sum() > 0


def test_direct_mapped_policies_agree():
    for g in W.random_small_geoms(30, seed=9, max_lines=16):
        lines = g.C // g.b
        tr = W.random_index_trace(300, lines * g.b // 4 * 3, seed=g.seed % 1000)
        outs = [oracle.cache_sim(g.C, g.b, 1, lines, p, tr, seed=123) for p in range(3)]
        assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


# ------------------------------------------------------ brute force vs lists
def _list_model(C, b, a, T, policy, seed, trace, mapping=0):
    """Sets as Python lists: LRU keeps recency order, FIFO insertion order,
    RANDOM and WEIGHTED explicit way slots.  Written independently of the
    oracle's stamp-based bookkeeping."""
    sets = [[] for _ in range(T)]
    slots = [[None] * a for _ in range(T)]
    ev = [0] * T
    out = []
    for idx in trace:
        line = (4 * int(idx)) // b
        s = (line >> mapping) % T
        if policy in (oracle.RANDOM, oracle.WEIGHTED):
            if line in slots[s]:
                out.append(0)
                continue
            out.append(1)
            if None in slots[s]:
                slots[s][slots[s].index(None)] = line
            else:
                pick = oracle.random_victim if policy == oracle.RANDOM else oracle.weighted_victim
                slots[s][pick(seed, s, ev[s], a)] = line
                ev[s] += 1
            continue
        lst = sets[s]
        if line in lst:
            out.append(0)
            if policy == oracle.LRU:
                lst.remove(line)
                lst.append(line)
            continue
        out.append(1)
        if len(lst) == a:
            lst.pop(0)
        lst.append(line)
    return np.array(out, dtype=np.uint8)


def test_bruteforce_tiny_caches_random_traces():
    rng = np.random.Generator(np.random.PCG64(2024))
    n_checked = 0
    for b in (4, 8, 16):
        for lines in range(1, 9):
            for a in [d for d in range(1, lines + 1) if lines % d == 0]:
                T = lines // a
                for policy in (oracle.LRU, oracle.FIFO, oracle.RANDOM):
                    for _ in range(12):
                        L = int(rng.integers(1, 40))
                        n_lines = int(rng.integers(1, 2 * lines + 3))
                        tr = rng.integers(0, n_lines * b // 4, size=L).astype(np.uint32)
                        got = oracle.cache_sim(lines * b, b, a, T, policy, tr, seed=77)
                        want = _list_model(lines * b, b, a, T, policy, 77, tr)
                        assert np.array_equal(got, want), (b, lines, a, policy, tr)
                        n_checked += 1
    assert n_checked > 1000


def test_bruteforce_mappings_and_weighted_policy():
    rng = np.random.Generator(np.random.PCG64(77))
    n_checked = 0
    for b in (4, 8):
        for (a, T) in ((1, 4), (2, 2), (3, 2), (4, 1), (4, 3), (2, 6)):
            for mapping in (0, 1, 2, 3):
                for policy in (oracle.LRU, oracle.FIFO, oracle.RANDOM, oracle.WEIGHTED):
                    if policy == oracle.WEIGHTED and a < 3:
                        continue
                    for _ in range(8):
                        L = int(rng.integers(1, 60))
                        n_lines = int(rng.integers(1, 4 * a * T * (1 << mapping) + 2))
                        tr = rng.integers(0, n_lines * b // 4, size=L).astype(np.uint32)
                        got = oracle.cache_sim(a * T * b, b, a, T, policy, tr, seed=5,
                                               mapping=mapping)
                        want = _list_model(a * T * b, b, a, T, policy, 5, tr, mapping)
                        assert np.array_equal(got, want), (b, a, T, mapping, policy, tr)
                        n_checked += 1
    assert n_checked > 1000


def test_bruteforce_every_short_sequence():
    # every sequence of 5 lines drawn from 4 lines, on three small caches
    import itertools
    for (lines, a) in ((2, 2), (4, 2), (3, 3)):
        T = lines // a
        b = 8
        for seq in itertools.product(range(4), repeat=5):
            tr = np.array([x * (b // 4) for x in seq], dtype=np.uint32)
            for policy in (oracle.LRU, oracle.FIFO):
                got = oracle.cache_sim(lines * b, b, a, T, policy, tr)
                want = _list_model(lines * b, b, a, T, policy, 0, tr)
                assert np.array_equal(got, want)


# --------------------------------------------------------------- RANDOM
def test_splitmix64_published_vectors():
    # SplitMix64 seeded with 0: its first two outputs
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_random_victims_uniform_chi2():
    from scipy.stats import chisquare
    for ways in (3, 4, 7, 16, 96):
        n = 200 * ways
        v = [oracle.random_victim(0xABCDEF, 5, k, ways) for k in range(n)]
        cnt = np.bincount(v, minlength=ways)
        assert cnt.size == ways
        assert chisquare(cnt).pvalue > 1e-3


def test_random_policy_depends_only_on_seed():
    g = W.Geom(1024, 32, 4, 8, W.RANDOM, 99)
    tr = oracle.pchase_trace(640, 8, 5000)
    a = oracle.cache_sim(g.C, g.b, g.ways, g.sets, oracle.RANDOM, tr, seed=1)
    b = oracle.cache_sim(g.C, g.b, g.ways, g.sets, oracle.RANDOM, tr, seed=1)
    c = oracle.cache_sim(g.C, g.b, g.ways, g.sets, oracle.RANDOM, tr, seed=2)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


# ----------------------------------------------------------------- banks
def test_bank_degree_is_gcd():
    for s in range(1, 65):
        words = [t * s for t in range(32)]
        assert oracle.bank_degree(words) == math.gcd(s, 32), s


def test_bank_fig14_stride2_and_broadcast():
    words = [t * 2 for t in range(32)]
    assert words[0] % 32 == words[16] % 32 == 0 and words[16] == 32
    assert oracle.bank_degree(words) == 2
    assert oracle.bank_degree([5] * 32) == 1  # same word: broadcast
    assert oracle.bank_degree(list(range(32))) == 1  # odd stride 1
    assert oracle.bank_degree([0, 32, 64, 96]) == 4


# --------------------------------------------------------------- classify
def test_classify_two_levels_with_spikes():
    rng = np.random.Generator(np.random.PCG64(3))
    truth = (rng.random(4000) < 0.3).astype(np.uint8)
    lat = np.where(truth == 1, 400.0, 100.0) * (1 + 0.02 * rng.standard_normal(4000))
    got, thr = oracle.classify(lat.astype(np.float32))
    assert np.array_equal(got, truth) and 100 < thr < 400
    # a few huge spikes on misses move nothing
    lat2 = lat.copy()
    spikes = np.where(truth == 1)[0][:15]
    lat2[spikes] *= 10
    got2, thr2 = oracle.classify(lat2.astype(np.float32))
    assert np.array_equal(got2, truth) and abs(thr2 - thr) < 50


def test_classify_flat_and_empty():
    got, _ = oracle.classify(np.full(100, 7.0, dtype=np.float32))
    assert got.sum() == 0
    got, _ = oracle.classify(np.zeros(0, dtype=np.float32))
    assert got.size == 0


def test_mean_latency_model():
    assert oracle.mean_latency(100.0, 300.0, 0.0) == 100.0
    assert oracle.mean_latency(100.0, 300.0, 1.0) == 400.0
    assert oracle.mean_latency(100.0, 300.0, 0.25) == 175.0


# ------------------------------------------------------------------ matcher
def _small_plan(C0):
    runs = []
    for nb in (C0 // 2, C0 - 4, C0, C0 + 4, C0 + 32, C0 + 36, C0 + 64, C0 + 132, 2 * C0):
        runs.append((nb // 4, 1))
    for nb in (C0 + 64, C0 + 256, 2 * C0, 4 * C0):
        runs.append((nb // 4, 16))
    traces = []
    for n, s in runs:
        per = n // math.gcd(n, s)
        traces.append(oracle.pchase_trace(n, s, 3 * per))
    return traces


def test_match_round_trip_small_grid():
    grid = W.geometry_grid(capacities=(512, 768, 1024), line_sizes=(32, 64),
                           way_choices=(1, 2, 4, 0))
    cands = np.array([(C, b, a, T, p) for (C, b, a, T) in grid for p in (0, 1)],
                     dtype=np.uint32)
    seeds = np.zeros(len(cands), dtype=np.uint64)
    traces = _small_plan(768)
    for truth in ((768, 64, 4, 3, 0), (768, 32, 2, 12, 0), (512, 32, 16, 1, 0)):
        obs = [oracle.cache_sim(*truth[:4], truth[4], t) for t in traces]
        dist = oracle.match(cands, seeds, traces, obs)
        ti = [i for i, c in enumerate(cands.tolist()) if tuple(c) == truth][0]
        assert dist[ti] == 0
        pick, nb = oracle.canonical_pick(cands, dist)
        assert dist[pick] == 0 and nb >= 1
        # the pick is indistinguishable from the truth on this plan
        for t in traces:
            assert np.array_equal(oracle.cache_sim(*cands[pick][:4], int(cands[pick][4]), t),
                                  oracle.cache_sim(*truth[:4], truth[4], t))


def test_canonical_order():
    cands = np.array([(1024, 32, 4, 8, 1), (1024, 64, 4, 4, 0), (1024, 32, 4, 8, 0),
                      (1024, 64, 2, 8, 0), (2048, 64, 2, 16, 0)], dtype=np.uint32)
    dist = np.array([0, 0, 0, 0, 0], dtype=np.uint64)
    assert oracle.canonical_pick(cands, dist) == (3, 5)
    dist = np.array([0, 3, 0, 1, 1], dtype=np.uint64)
    assert oracle.canonical_pick(cands, dist) == (2, 2)


# ------------------------------------------------------- unequal sets (TLB)
def _uneq_list_model(b, a, T, extra, policy, trace):
    """Unequal sets as Python lists (set 0 holds a + extra lines, the others
    a), the residue rule of or_cache_sim_uneq written out per access."""
    M = T * a + extra
    sets = [[] for _ in range(T)]
    out = []
    for idx in trace:
        line = (4 * int(idx)) // b
        r = line % M
        s = r % T if r < T * a else 0
        cap = a + extra if s == 0 else a
        lst = sets[s]
        if line in lst:
            out.append(0)
            if policy == oracle.LRU:
                lst.remove(line)
                lst.append(line)
            continue
        out.append(1)
        if len(lst) == cap:
            lst.pop(0)
        lst.append(line)
    return np.array(out, dtype=np.uint8)


def test_unequal_l2_tlb_fig9_steps():
    """Sec. 4.4, Fig. 9: the L2 TLB (2 MB pages, LRU) holds 65 entries, one
    set of 17 and six of 8, and its misses grow set by set as N passes 130 MB:
    the large set first (at 132 MB), then 8 more entries per 2 MB step up to
    144 MB.  Counted as this model counts Eq. (2)'s steps, an overflowing set
    of w ways misses on all of its w + 1 pages, so a steady pass misses 18 at
    132 MB, 9 more per step to 144 MB, and every access from then on."""
    page = 2 << 20
    C = 65 * page
    steady = {}
    for n_pages in range(60, 80):
        n = n_pages * page // 4
        tr = oracle.pchase_trace(n, page // 4, 3 * n_pages)
        m = oracle.cache_sim_uneq(C, page, 8, 7, 9, oracle.LRU, tr)
        assert m[:n_pages].all()                      # the first pass: cold
        assert np.array_equal(m[n_pages:2 * n_pages], m[2 * n_pages:])  # periodic
        steady[n_pages] = int(m[n_pages:2 * n_pages].sum())
    assert all(steady[k] == 0 for k in range(60, 66))  # up to 130 MB: all held
    assert steady[66] == 17 + 1                        # 132 MB: the large set
    for k in range(67, 73):                            # 134 .. 144 MB
        assert steady[k] - steady[k - 1] == 8 + 1
    assert all(steady[k] == k for k in range(72, 80))  # every set overflows


def test_unequal_sets_with_no_extra_ways_is_the_standard_cache():
    rng = np.random.Generator(np.random.PCG64(65))
    for (b, a, T) in ((4, 2, 3), (8, 4, 7), (32, 8, 7), (64, 1, 5)):
        for policy in (oracle.LRU, oracle.FIFO):
            for _ in range(10):
                tr = rng.integers(0, 3 * a * T * b // 4 + 5, size=400).astype(np.uint32)
                assert np.array_equal(
                    oracle.cache_sim_uneq(a * T * b, b, a, T, 0, policy, tr),
                    oracle.cache_sim(a * T * b, b, a, T, policy, tr))


def test_unequal_sets_hold_any_m_consecutive_lines():
    """Capacity: the M = T*a + extra residues each have a place, so a chain
    over any M consecutive lines misses only on its first pass (LRU, FIFO)."""
    for (a, T, extra) in ((8, 7, 9), (2, 3, 1), (4, 5, 7), (1, 1, 3)):
        M = T * a + extra
        for start in (0, 5, M - 1):
            lines = np.arange(start, start + M, dtype=np.uint32)
            tr = np.tile(lines, 3) * 8          # b = 32 B: 8 elements per line
            for policy in (oracle.LRU, oracle.FIFO):
                m = oracle.cache_sim_uneq(M * 32, 32, a, T, extra, policy, tr)
                assert m[:M].all() and m[M:].sum() == 0
            # one line more than fits, cycled: it shares the set of line
            # `start` (same residue), whose w + 1 lines then miss on every
            # access under LRU while the other sets never do
            tr1 = np.tile(np.arange(start, start + M + 1, dtype=np.uint32), 3) * 8
            m1 = oracle.cache_sim_uneq(M * 32, 32, a, T, extra, oracle.LRU, tr1)
            r0 = start % M
            w = a + extra if (r0 >= T * a or r0 % T == 0) else a
            assert m1[M + 1:2 * (M + 1)].sum() == w + 1
            assert np.array_equal(m1[M + 1:2 * (M + 1)], m1[2 * (M + 1):])


def test_bruteforce_unequal_sets():
    rng = np.random.Generator(np.random.PCG64(17))
    n = 0
    for b in (4, 8):
        for (a, T, extra) in ((1, 1, 1), (1, 3, 2), (2, 3, 1), (3, 2, 4), (2, 7, 5), (8, 7, 9)):
            M = T * a + extra
            for policy in (oracle.LRU, oracle.FIFO):
                for _ in range(10):
                    L = int(rng.integers(1, 80))
                    tr = rng.integers(0, int(rng.integers(1, 3 * M + 3)) * b // 4 + 1,
                                      size=L).astype(np.uint32)
                    got = oracle.cache_sim_uneq(M * b, b, a, T, extra, policy, tr)
                    want = _uneq_list_model(b, a, T, extra, policy, tr)
                    assert np.array_equal(got, want), (b, a, T, extra, policy, tr)
                    n += 1
    assert n == 240


def test_unequal_sets_reject_bad_geometry():
    tr = np.zeros(4, dtype=np.uint32)
    with pytest.raises(Exception):
        oracle.cache_sim_uneq(65 * 32 + 32, 32, 8, 7, 9, oracle.LRU, tr)   # C != M * b
    with pytest.raises(Exception):
        oracle.cache_sim_uneq(65 * 32, 32, 8, 7, 9, oracle.RANDOM, tr)     # LRU / FIFO only


# ------------------------------------------------- LRU stack property (cuts)
def _recent_lines(trace, b, T, a, c0):
    """Per set, the a most recently used distinct lines before access c0,
    read backwards from c0 (the state a time part of an LRU item rebuilds)."""
    held = [[] for _ in range(T)]
    for t in range(c0 - 1, -1, -1):
        line = (4 * int(trace[t])) // b
        s = line % T
        if line not in held[s] and len(held[s]) < a:
            held[s].append(line)
    return held


def test_lru_state_is_the_most_recent_lines_of_each_set():
    """Sec. 3's LRU: the lines a set holds at any access are exactly its a
    most recently used distinct lines, so the state at a cut needs no
    simulation of the accesses before it.  The oracle's held lines after
    every prefix agree; under FIFO they need not (FIFO keeps the a most
    recently inserted lines, which depends on past misses)."""
    rng = np.random.Generator(np.random.PCG64(303))
    fifo_differs = 0
    for _ in range(60):
        b = int(rng.choice([4, 8, 32]))
        a, T = int(rng.integers(1, 6)), int(rng.integers(1, 5))
        n_lines = int(rng.integers(a * T, 4 * a * T + 3))
        L = int(rng.integers(20, 200))
        tr = rng.integers(0, n_lines * b // 4, size=L).astype(np.uint32)
        for c0 in sorted(set(int(x) for x in rng.integers(1, L, size=4))):
            want = _recent_lines(tr, b, T, a, c0)
            for policy in (oracle.LRU, oracle.FIFO):
                _, fin = oracle.cache_sim(a * T * b, b, a, T, policy, tr[:c0], want_final=True)
                fin = fin.reshape(T, a)
                got = [sorted(int(x) for x in row if x != 0xFFFFFFFF) for row in fin]
                same = got == [sorted(h) for h in want]
                if policy == oracle.LRU:
                    assert same, (b, a, T, c0, tr[:c0])
                else:
                    fifo_differs += not same
    assert fifo_differs > 0


def test_fifo_state_after_a_misses_per_set_is_the_most_recent_lines():
    """Sec. 3's FIFO holds each set's a most recently inserted lines.  When
    each set's last accesses before a cut (its last a, or all it had) were all
    misses, every one of them was an insertion, so the set holds exactly its a
    most recently used distinct lines, the state an LRU time part rebuilds: a
    FIFO time part could start from that rebuild once the part before it has
    seen those misses.  And a cyclic stream in which every reuse of a line
    comes after at least a other accesses of its set misses on every access,
    by induction from the cold start."""
    rng = np.random.Generator(np.random.PCG64(404))
    checked = 0
    for _ in range(80):
        b = int(rng.choice([4, 8, 32]))
        a, T = int(rng.integers(1, 6)), int(rng.integers(1, 5))
        n_lines = int(rng.integers(2 * a * T, 6 * a * T + 3))
        L = int(rng.integers(20, 240))
        tr = rng.integers(0, n_lines * b // 4, size=L).astype(np.uint32)
        miss = oracle.cache_sim(a * T * b, b, a, T, oracle.FIFO, tr)
        sets = ((4 * tr.astype(np.int64)) // b) % T
        for c0 in sorted(set(int(x) for x in rng.integers(1, L, size=6))):
            tails_missed = True
            for st in range(T):
                idx = np.nonzero(sets[:c0] == st)[0]
                if not miss[idx[-a:]].all():
                    tails_missed = False
            if not tails_missed:
                continue
            want = _recent_lines(tr, b, T, a, c0)
            _, fin = oracle.cache_sim(a * T * b, b, a, T, oracle.FIFO, tr[:c0], want_final=True)
            got = [sorted(int(x) for x in row if x != 0xFFFFFFFF) for row in fin.reshape(T, a)]
            assert got == [sorted(h) for h in want], (b, a, T, c0)
            checked += 1
    assert checked >= 20
    # cyclic P-chase streams: N / s lines spread so that every set sees more
    # than a distinct lines, each reused a period later
    for (n, s, a, T, b) in ((3072 // 4, 256 // 4, 8, 2, 128), (131328 // 4, 16, 1536, 1, 64),
                            (5632 // 4, 512 // 4, 2, 4, 256), (40000, 37, 4, 8, 32)):
        tr = oracle.pchase_trace(n, s, 3 * n // np.gcd(n, s))
        sets = ((4 * tr.astype(np.int64)) // b) % T
        lines = (4 * tr.astype(np.int64)) // b
        if any(len(np.unique(lines[sets == st])) <= a for st in np.unique(sets)):
            continue
        assert oracle.cache_sim(a * T * b, b, a, T, oracle.FIFO, tr).all(), (n, s, a, T, b)


def test_unequal_l2_tlb_behind_a_thrashing_l1_tlb():
    """Sec. 4.4's path with the measured L2 TLB: past 16 pages the L1 TLB
    (16 entries, LRU) misses on every access of a 2 MB chain, so the
    unequal L2 TLB sees the whole stream and behaves as it does alone
    (Fig. 9's steps); within 16 pages it sees only the first touches."""
    page = 2 << 20
    l1 = dict(C=16 * page, b=page, ways=16, T=1, policy=oracle.LRU)
    l2 = dict(C=65 * page, b=page, ways=8, T=7, policy=oracle.LRU, extra=9)
    for n_pages in (17, 40, 65, 66, 69, 72, 90):
        n = n_pages * page // 4
        tr = oracle.pchase_trace(n, page // 4, 4 * n_pages)
        m1, m2 = oracle.hierarchy([l1, l2], tr)
        assert m1.all()
        assert np.array_equal(m2, oracle.cache_sim_uneq(65 * page, page, 8, 7, 9, oracle.LRU, tr))
    for n_pages in (1, 9, 16):
        n = n_pages * page // 4
        tr = oracle.pchase_trace(n, page // 4, 4 * n_pages)
        m1, m2 = oracle.hierarchy([l1, l2], tr)
        assert m1[n_pages:].sum() == 0 and m2.sum() == n_pages


def test_spectrum_chain_reaches_the_paper_patterns():
    """Sec. 5.2 (Fig. 10, the pattern table of Fig. 11): the non-uniform
    chain's segments land in the patterns they are built for, under the
    cache model with a data cache that holds its lines (256 lines of 128 B,
    fully associative, LRU: with sets taken from the low line bits, lines
    1 MB apart would all share one set), the 16-entry L1 TLB and the unequal
    L2 TLB over 2 MB pages:
    B misses the data cache and the L1 TLB on each new page only; A misses
    both; C hits the data cache, and misses the L1 TLB on its first return
    to each page (A's sweep flushed them); D hits everything after its first
    access."""
    path, labels, n = W.spectrum_chain()
    tr = np.array(path, dtype=np.uint32)
    lab = np.array(labels)
    page = 2 << 20
    data = oracle.cache_sim(256 * 128, 128, 256, 1, oracle.LRU, tr)
    t1, t2 = oracle.hierarchy([dict(C=16 * page, b=page, ways=16, T=1, policy=oracle.LRU),
                               dict(C=65 * page, b=page, ways=8, T=7, policy=oracle.LRU,
                                    extra=9)], tr)
    assert len(path) == 65 + 64 + 65 + 32 and len(set(path)) == len(path)
    assert data[lab == "B_new_page"].all() and data[lab == "B_same_page"].all()
    assert t1[lab == "B_new_page"].all() and not t1[lab == "B_same_page"].any()
    assert data[lab == "A_32MB"].all() and t1[lab == "A_32MB"].all()
    c = np.flatnonzero(lab == "C_revisit")
    c_pages = (4 * tr[c].astype(np.uint64)) // page
    first = np.zeros(c.size, dtype=bool)
    first[np.unique(c_pages, return_index=True)[1]] = True
    assert not data[c].any()
    assert t1[c][first].all()
    d = np.flatnonzero(lab == "D_same_line")
    assert not data[d[1:]].any() and not t1[d[1:]].any()
    # the L2 TLB tells the C accesses apart: their pages were last used
    # before A's 64 new pages went through it
    assert t2[lab == "C_revisit"].sum() > 0


# ------------------------------------------ matcher: every candidate, Table 4
def _canonical(cands, members):
    """The canonical member of a set of candidate indices, by the order the
    C header states: LRU < FIFO < RANDOM (< WEIGHTED), larger b, fewer ways,
    smaller C, lower index."""
    return min(members, key=lambda g: (cands[g].policy, -cands[g].b, cands[g].ways, cands[g].C, g))


def _sim(g, tr):
    return oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr, seed=g.seed, mapping=g.mapping)


def _plan_traces(pts):
    return [t if t is not None else oracle.pchase_trace(r.n_elems, r.stride, r.length)
            for r, t in pts]


def test_match_round_trip_every_candidate_is_the_truth():
    """Sec. 4.2's procedure mechanised, noise-free, with the oracle alone:
    every candidate of a reduced grid (512 B - 1.5 KB, 32 / 64 B lines, 1-8
    ways or full, LRU / FIFO / RANDOM) is the truth in turn.  The candidates
    at distance 0 are exactly the truth's identical-outcome class on the plan,
    and the canonical pick is that class's canonical member."""
    grid = W.geometry_grid(capacities=(512, 768, 1024, 1536), line_sizes=(32, 64),
                           way_choices=(1, 2, 4, 8, 0))
    cands = [W.Geom(C, b, a, T, p, 0x900D + i) for i, (C, b, a, T) in enumerate(grid)
             for p in (0, 1, 2)]
    rows = np.array([(g.C, g.b, g.ways, g.sets, g.policy) for g in cands], dtype=np.uint32)
    seeds = np.array([g.seed for g in cands], dtype=np.uint64)
    traces = _small_plan(768) + [W.hot_retouch_trace(nb, 64) for nb in (1152, 1536, 3072)]
    outcome = [[_sim(g, t) for t in traces] for g in cands]
    keys = [b"".join(np.packbits(o).tobytes() for o in out) for out in outcome]
    assert len(set(keys)) > len(cands) // 3  # the plan separates most of the grid
    for ti in range(len(cands)):
        dist = oracle.match(rows, seeds, traces, outcome[ti])
        cls = [g for g in range(len(cands)) if keys[g] == keys[ti]]
        assert sorted(np.nonzero(dist == 0)[0].tolist()) == cls, ti
        pick, nb = oracle.canonical_pick(rows, dist)
        assert pick == _canonical(cands, cls) and nb == len(cls), (ti, pick, cls)


def test_table4_geometries_recovered_by_the_two_stage_procedure():
    """Table 4's caches (Secs. 4.3-4.5) are recovered exactly by the oracle
    from their own noise-free outcomes: stage 1 of Fig. 6 (s = 1 element over
    the candidate capacities) finds C, stage 2 (two_stage_plan) separates
    line size, sets, mapping and policy among every candidate of that
    capacity (grid and Table 4 additions): the truth is the one candidate at
    distance 0: the 12 KB and 24 KB texture L1 caches (32 B lines, 4 sets, address
    bits 7-8, LRU) and the Fermi L1 data cache (16 KB, 128 B, 32 sets, the
    weighted non-LRU policy)."""
    cands = W.matcher_candidates()
    truths = [g for g in W.table4_candidates() if g.policy == W.LRU and g.mapping == 2]
    truths.append([g for g in W.table4_candidates() if g.policy == W.WEIGHTED][0])
    assert [(g.C, g.b, g.sets) for g in truths] == [(12288, 32, 4), (24576, 32, 4),
                                                    (16384, 128, 32)]
    caps, sweep = W.capacity_sweep()
    for truth in truths:
        steady = []
        for r in sweep:
            m = _sim(truth, oracle.pchase_trace(r.n_elems, r.stride, r.length))
            steady.append(int(m[r.warmup:].sum()))
        C_est = max(c for c, s in zip(caps, steady) if s == 0)
        assert C_est == truth.C
        pool = [i for i, g in enumerate(cands) if g.C == C_est]
        traces = _plan_traces(W.two_stage_plan(C_est))
        obs = [_sim(truth, t) for t in traces]

        def dist(i):
            return sum(int((_sim(cands[i], t) != o).sum()) for t, o in zip(traces, obs))

        with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
            d = dict(zip(pool, ex.map(dist, pool)))
        zero = [i for i in pool if d[i] == 0]
        assert zero == [cands.index(truth)], [cands[i] for i in zero]
