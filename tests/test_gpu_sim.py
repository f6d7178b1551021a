"""Parity of the CUDA path (S1-S3) with the CPU oracle, bit for bit."""
import math

import numpy as np
import pytest

import oracle
from paper_1509_02308_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1509_02308_gb300 import api


def oracle_trace(run: W.Run) -> np.ndarray:
    if run.chain is not None:
        return oracle.pchase_walk(run.chain, run.length)
    return oracle.pchase_trace(run.n_elems, run.stride, run.length)


def oracle_bits(g: W.Geom, tr: np.ndarray) -> np.ndarray:
    return oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr, seed=g.seed)


def gpu_bits(bitmaps, offs, i, n):
    w = bitmaps[int(offs[i]):int(offs[i]) + (n + 31) // 32].cpu().numpy().view(np.uint32)
    return api.unpack_bits(w, n)


def check_items(geoms, runs, pairs, use_idx=True, tag=""):
    """Simulate (geoms x runs via pairs) on the GPU and compare every item."""
    traces, keep = [], []
    for r in runs:
        if use_idx or r.chain is not None:
            t = torch.from_numpy(oracle_trace(r).view(np.int32)).cuda() if r.length else None
            keep.append(t)
            traces.append((t if t is not None else None, r.length, r.warmup, r.n_elems, r.stride))
        else:
            traces.append((None, r.length, r.warmup, r.n_elems, r.stride))
    bitmaps, counts, offs = api.cache_sim_batch(geoms, traces, pairs)
    counts = counts.cpu().numpy()
    for i, (g, t) in enumerate(pairs):
        G, R = geoms[g], runs[t]
        want = oracle_bits(G, oracle_trace(R))
        got = gpu_bits(bitmaps, offs, i, R.length)
        assert np.array_equal(got, want), (tag, i, G, R.n_elems, R.stride, R.length,
                                           int(np.argmax(got != want)))
        assert counts[i, 0] == want.sum()
        assert counts[i, 1] == want[R.warmup:].sum()


# ----------------------------------------------------------------------- S1
def test_build_uniform_matches_listing1():
    for n, s, L in [(13, 1, 100), (4096, 32, 12345), (3072, 7, 1), (5, 5, 17), (100003, 999, 50001),
                    (1 << 20, 1 << 12, 1 << 18)]:
        tr, arr = api.pchase_build(n, s, L, with_array=True)
        assert np.array_equal(tr.cpu().numpy().view(np.uint32), oracle.pchase_trace(n, s, L))
        assert np.array_equal(arr.cpu().numpy().view(np.uint32), oracle.pchase_array(n, s))


def test_build_batch_ragged_offsets():
    runs = [W.Run(n, s, L, 0) for (n, s, L) in
            [(13, 1, 1), (13, 1, 2), (13, 1, 3), (4096, 32, 5), (777, 3, 1000), (64, 64, 7),
             (1 << 16, 5, 70001)]]
    out, offs = api.pchase_build_batch(runs)
    o = out.cpu().numpy().view(np.uint32)
    for i, r in enumerate(runs):
        assert np.array_equal(o[int(offs[i]):int(offs[i + 1])],
                              oracle.pchase_trace(r.n_elems, r.stride, r.length)), i


def test_build_custom_chain_and_out_of_range_chain():
    rng = np.random.Generator(np.random.PCG64(1))
    chain = rng.permutation(1000).astype(np.uint32)
    t = api.pchase_build(1000, 0, 3000, next_chain=torch.from_numpy(chain.view(np.int32)).cuda())
    assert np.array_equal(t.cpu().numpy().view(np.uint32), oracle.pchase_walk(chain, 3000))
    bad = chain.copy()
    bad[oracle.pchase_walk(chain, 10)[5]] = 5000
    st = api.status_word()
    api.pchase_build(1000, 0, 3000, next_chain=torch.from_numpy(bad.view(np.int32)).cuda(),
                     status=st)
    torch.cuda.synchronize()
    assert int(st.item()) & 2


# ------------------------------------------------------------------ config 1
def test_config1_bit_exact_and_closed_form():
    g, runs = W.config1()
    pairs = [(0, t) for t in range(len(runs))]
    check_items([g], runs, pairs, use_idx=True, tag="explicit")
    check_items([g], runs, pairs, use_idx=False, tag="analytic")
    traces = [(None, r.length, r.warmup, r.n_elems, r.stride) for r in runs]
    _, counts, _ = api.cache_sim_batch([g], traces, pairs)
    assert int(counts[:, 0].sum()) == 30544
    assert sum(r.length for r in runs) == 41904


# ------------------------------------------------------- small geometries
def check_host_traces(geoms, host, warmups, n_elems, pairs):
    """Like check_items, for explicit host traces."""
    traces = []
    for t, w, n in zip(host, warmups, n_elems):
        dt = torch.from_numpy(np.ascontiguousarray(t, dtype=np.uint32).view(np.int32)).cuda() \
            if len(t) else None
        traces.append((dt, len(t), w, n, 1))
    bitmaps, counts, offs = api.cache_sim_batch(geoms, traces, pairs)
    counts = counts.cpu().numpy()
    for i, (g, t) in enumerate(pairs):
        want = oracle_bits(geoms[g], host[t])
        got = gpu_bits(bitmaps, offs, i, len(host[t]))
        assert np.array_equal(got, want), (i, geoms[g], n_elems[t], len(host[t]))
        assert counts[i, 0] == want.sum() and counts[i, 1] == want[warmups[t]:].sum()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_small_geometries_ragged_traces(seed):
    """Arbitrary T (not only powers of two), every policy, ragged lengths
    (0, 1, around 32 and 64, several tiles), random and uniform traces."""
    geoms = W.random_small_geoms(48, seed=seed, max_lines=96, line_sizes=(4, 8, 16, 32, 64, 128))
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = [0, 1, 31, 32, 33, 63, 64, 65, 200, 1000, 1025, 4097]
    host, warm, ns = [], [], []
    for i, g in enumerate(geoms):
        L = lens[i % len(lens)]
        n = int(rng.integers(1, 4 * g.C // 4 + 2))
        if i % 3 == 0:
            t = W.random_index_trace(max(L, 1), n, seed=seed * 1000 + i, hot=4)[:L]
        else:
            s = int(rng.integers(1, max(2, n)))
            t = oracle.pchase_trace(n, s, L) if L else np.zeros(0, dtype=np.uint32)
        host.append(t)
        warm.append(min(L, 7))
        ns.append(n)
    check_host_traces(geoms, host, warm, ns, [(i, i) for i in range(len(geoms))])


def test_every_policy_and_way_count_on_uniform_chains():
    geoms, runs, pairs = [], [], []
    for policy in (W.LRU, W.FIFO, W.RANDOM):
        for (C, b, a) in [(1024, 32, 1), (1024, 32, 2), (1024, 32, 4), (1024, 32, 8),
                          (1024, 32, 16), (1024, 32, 32), (3072, 64, 48), (1536, 32, 3),
                          (12288, 32, 96), (6144, 64, 96), (4096, 16, 256), (2048, 4, 5 * 0 + 512),
                          (768, 16, 12), (8192, 256, 32)]:
            if (C // b) % a:
                continue
            geoms.append(W.Geom(C, b, a, C // (a * b), policy, 0xC0FFEE + a))
    for (nb, sb) in [(512, 4), (1020, 8), (1536, 32), (2048, 64), (3200, 128), (12800, 32),
                     (8192, 4), (20000, 4), (16384, 256)]:
        n, s = nb // 4, sb // 4
        per = n // math.gcd(n, s)
        runs.append(W.Run(n, s, 3 * per + 5, per))
    for g in range(len(geoms)):
        for t in range(len(runs)):
            pairs.append((g, t))
    check_items(geoms, runs, pairs, use_idx=False, tag="analytic")
    sub = pairs[::7]
    check_items(geoms, runs, sub, use_idx=True, tag="explicit")


def test_table4_geometries():
    t4 = [(16384, 128, 32), (12288, 32, 4), (24576, 32, 4)]
    geoms = [W.Geom(C, b, C // (T * b), T, p, 5) for (C, b, T) in t4 for p in (0, 1, 2)]
    runs = []
    for C in (12288, 16384, 24576):
        for k in (-2, 0, 1, 3, 8):
            n = (C + k * 32) // 4
            runs.append(W.Run(n, 8, 3 * (n // 8), n // 8))
            runs.append(W.Run(n, 1, 3 * n, n))
    pairs = [(g, t) for g in range(len(geoms)) for t in range(len(runs))]
    check_items(geoms, runs, pairs, use_idx=False, tag="table4")


# ------------------------------------------------------------------ config 2
def test_config2_subsample_bit_exact():
    geoms, runs = W.config2(n_items=96, max_len=1 << 14)
    pairs = [(i, i) for i in range(len(geoms))]
    check_items(geoms, runs, pairs, use_idx=True, tag="cfg2-explicit")
    check_items(geoms, runs, pairs, use_idx=False, tag="cfg2-analytic")


def test_config2_full_size_sampled():
    """All 4096 items at full length in the launch configuration the bench
    times; the oracle checks a sample of items one by one."""
    from paper_1509_02308_gb300.api import SimPlan
    geoms, runs = W.config2()
    flat, offs = api.pchase_build_batch(runs)
    traces = [(flat[int(offs[i]):int(offs[i + 1])], r.length, r.warmup, r.n_elems, r.stride)
              for i, r in enumerate(runs)]
    plan = SimPlan(geoms, traces, pairs=[(i, i) for i in range(len(runs))])
    bitmaps, counts = plan.run()
    torch.cuda.synchronize()
    counts = counts.view(-1, 2).cpu().numpy()
    lens = np.array([r.length for r in runs])
    assert (counts[:, 0] <= lens).all() and (counts[:, 1] <= counts[:, 0]).all()
    # sample: cheap items of every policy and set mode, plus the first and last
    cand = [i for i in range(len(runs)) if runs[i].length <= 60000 and geoms[i].ways <= 512]
    rng = np.random.Generator(np.random.PCG64(7))
    sample = set(rng.choice(cand, size=40, replace=False).tolist())
    # and the longest items of modest associativity (split into set-parts)
    longest = sorted((i for i in range(len(runs)) if geoms[i].ways <= 64),
                     key=lambda i: -runs[i].length)
    sample = sorted(sample | set(longest[:6]))
    for i in sample:
        g, r = geoms[i], runs[i]
        want = oracle_bits(g, oracle.pchase_trace(r.n_elems, r.stride, r.length))
        w0 = int(plan.word_offsets[i])
        got = api.unpack_bits(bitmaps[w0:w0 + (r.length + 31) // 32].cpu().numpy().view(np.uint32),
                              r.length)
        assert np.array_equal(got, want), (i, g, r)
        assert counts[i, 0] == want.sum() and counts[i, 1] == want[r.warmup:].sum()
    # the bitmaps agree with the counts everywhere
    pop = np.unpackbits(bitmaps.cpu().numpy().view(np.uint8)).reshape(-1)
    assert int(pop.sum()) == int(counts[:, 0].sum())


def test_longest_items_split_into_set_parts_full_length():
    """The longest config-2 items of modest associativity at full length,
    planned with forced set splits (up to 8 parts), against the oracle."""
    from paper_1509_02308_gb300.api import SimPlan
    geoms, runs = W.config2()
    idx = sorted((i for i in range(len(runs)) if geoms[i].ways <= 64),
                 key=lambda i: -runs[i].length)[:8]
    g2 = [geoms[i] for i in idx]
    r2 = [runs[i] for i in idx]
    traces = [(None, r.length, r.warmup, r.n_elems, r.stride) for r in r2]
    plan = SimPlan(g2, traces, pairs=[(i, i) for i in range(len(r2))],
                   tune={"max_split": 8, "split_cost_ns": 1})
    assert " split=0 " not in plan.description
    bitmaps, counts = plan.run()
    torch.cuda.synchronize()
    counts = counts.view(-1, 2).cpu().numpy()
    for k, (g, r) in enumerate(zip(g2, r2)):
        want = oracle_bits(g, oracle.pchase_trace(r.n_elems, r.stride, r.length))
        w0 = int(plan.word_offsets[k])
        got = api.unpack_bits(bitmaps[w0:w0 + (r.length + 31) // 32].cpu().numpy().view(np.uint32),
                              r.length)
        assert np.array_equal(got, want), (k, g, r)
        assert counts[k, 0] == want.sum() and counts[k, 1] == want[r.warmup:].sum()


def test_index_out_of_range_is_flagged_not_faulted():
    g = W.Geom(1024, 32, 4, 8)
    t = torch.tensor([1, 2, 3, 5000, 4], dtype=torch.int32, device="cuda")
    from paper_1509_02308_gb300.api import SimPlan
    plan = SimPlan([g], [(t, 5, 0, 100, 1)], pairs=[(0, 0)])
    st = api.status_word()
    plan.run(status=st)
    torch.cuda.synchronize()
    assert int(st.item()) & 1


def test_plan_rerun_is_identical_and_graph_capturable():
    from paper_1509_02308_gb300.api import SimPlan
    geoms, runs = W.config2(n_items=64, max_len=1 << 13)
    traces = [(None, r.length, r.warmup, r.n_elems, r.stride) for r in runs]
    plan = SimPlan(geoms, traces, pairs=[(i, i) for i in range(len(runs))])
    b1, c1 = plan.run()
    b1, c1 = b1.clone(), c1.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b2 = torch.zeros_like(b1)
        c2 = torch.zeros_like(c1)
        plan.run(bitmaps=b2, counts=c2)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    b3 = torch.zeros_like(b1)
    c3 = torch.zeros_like(c1)
    with torch.cuda.graph(g):
        plan.run(bitmaps=b3, counts=c3)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(b1, b2) and torch.equal(c1, c2)
    assert torch.equal(b1, b3) and torch.equal(c1, c3)
