"""Set mappings that take the set from higher line bits (the texture L1 cache
of Sec. 4.3) and the weighted Fermi L1 policy (Sec. 4.5) against the oracle,
bit for bit, in every set mode and with set splits; and the matcher telling
the mappings apart."""
import numpy as np
import pytest

import oracle
from paper_1509_02308_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1509_02308_gb300 import api

TUNES = {
    "default": None,
    "batch_all": {"batch_max_sets": 1 << 30},
    "no_batch_scan8": {"batch_max_sets": 0xFFFFFFFF, "scan_max_ways": 8},
    "no_batch_table": {"batch_max_sets": 0xFFFFFFFF, "scan_max_ways": 1},
    "split_batch": {"max_split": 8, "split_cost_ns": 1, "batch_max_sets": 1 << 30},
    "split_table": {"max_split": 8, "split_cost_ns": 1, "batch_max_sets": 0xFFFFFFFF,
                    "scan_max_ways": 1},
}


def variant_geoms():
    out = []
    # texture L1 (12 KB, 32 B lines, 4 sets of 96, bits 7-8) and smaller relatives
    for (C, b, a, T) in [(12288, 32, 96, 4), (1536, 32, 4, 12), (1024, 16, 8, 8),
                         (768, 32, 3, 8), (2048, 32, 16, 4), (512, 16, 4, 8)]:
        for m in (1, 2, 3):
            for p in (W.LRU, W.FIFO, W.RANDOM, W.WEIGHTED):
                out.append(W.Geom(C, b, a, T, p, 0x7E0 + 13 * m + 3 * p + a, mapping=m))
    # Fermi L1 data cache (16 KB, 128 B, 4 ways, 32 sets) and relatives, weighted
    for (C, b, a, T) in [(16384, 128, 4, 32), (1536, 32, 3, 16), (4096, 64, 8, 8),
                         (1024, 32, 32, 1), (768, 16, 6, 8)]:
        out.append(W.Geom(C, b, a, T, W.WEIGHTED, 0xF3A + a + T))
    return out


def variant_traces(rng):
    tr = []
    for (nb, sb) in [(12288 + 128, 32), (12800, 32), (16512, 128), (2048, 4), (3000, 8),
                     (900, 32), (5000, 64), (1100, 4)]:
        n, s = nb // 4, sb // 4
        tr.append(oracle.pchase_trace(n, s, 3 * (n // s) + 29))
    for m in (3, 7, 17, 40):
        lines = rng.integers(0, 200, size=m) * 8
        tr.append(np.tile(lines, 2500 // m + 1)[:2500].astype(np.uint32))
    for k in range(3):
        tr.append(W.random_index_trace(4000, 2500 * (k + 1), seed=300 + k, hot=5))
    return tr


@pytest.mark.parametrize("tune_name", list(TUNES))
def test_variants_match_oracle(tune_name):
    rng = np.random.Generator(np.random.PCG64(17))
    geoms = variant_geoms()
    host = variant_traces(rng)
    n_el = [int(t.max()) + 1 for t in host]
    dev = [torch.from_numpy(t.view(np.int32)).cuda() for t in host]
    traces = [(d, t.size, min(t.size, 64), n, 1) for d, t, n in zip(dev, host, n_el)]
    plan = api.SimPlan(geoms, traces, tune=TUNES[tune_name])
    if tune_name.startswith("split"):
        assert " split=0 " not in plan.description, plan.description
    bitmaps, counts = plan.run()
    torch.cuda.synchronize()
    b = bitmaps.cpu().numpy().view(np.uint32)
    c = counts.view(-1, 2).cpu().numpy()
    for gi, g in enumerate(geoms):
        for ti, t in enumerate(host):
            i = gi * len(host) + ti
            want = oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, t, seed=g.seed,
                                    mapping=g.mapping)
            got = api.unpack_bits(b[int(plan.word_offsets[i]):], t.size)
            assert np.array_equal(got, want), (tune_name, g, ti, int(np.argmax(got != want)))
            assert c[i, 0] == want.sum() and c[i, 1] == want[64:].sum()


def test_texture_l1_sweep_and_analytic_chains():
    """Sec. 4.3's stage-2 sweep (s = 32 B, N = 12 KB .. 12.5 KB and beyond) as
    analytic chains (no trace array) on the bits-7-8 texture L1 geometry."""
    g = W.Geom(12288, 32, 96, 4, W.LRU, mapping=2)
    sizes = [12288 + 32 * d for d in range(0, 17)] + [16384, 61440]
    traces = [(None, 3 * (nb // 32), nb // 32, nb // 4, 8) for nb in sizes]
    bitmaps, counts, offs = api.cache_sim_batch([g], traces, pairs=[(0, k) for k in range(len(sizes))])
    b = bitmaps.cpu().numpy().view(np.uint32)
    for k, nb in enumerate(sizes):
        tr = oracle.pchase_trace(nb // 4, 8, 3 * (nb // 32))
        want = oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr, mapping=2)
        got = api.unpack_bits(b[int(offs[k]):], tr.size)
        assert np.array_equal(got, want), nb


def test_matcher_tells_mappings_and_weighted_apart():
    """Observed bitmaps of a bits-7-8 texture-L1-like cache and of a weighted
    Fermi-L1-like cache: among candidates that differ only in mapping or
    policy, the matcher's distances equal the oracle's Hamming distances and
    the true candidate is at distance 0."""
    truths = [W.Geom(1536, 32, 12, 4, W.LRU, mapping=2), W.Geom(2048, 64, 4, 8, W.WEIGHTED, 91)]
    for truth in truths:
        cands = [W.Geom(truth.C, truth.b, truth.ways, truth.sets, p, truth.seed, mapping=m)
                 for m in (0, 1, 2, 3) for p in (W.LRU, W.FIFO, W.RANDOM, W.WEIGHTED)]
        runs = []
        for nb in (truth.C - 128, truth.C + 32, truth.C + 128, truth.C + 512, 2 * truth.C):
            runs.append(W.Run(nb // 4, truth.b // 4, 6 * (nb // truth.b), nb // truth.b))
        runs.append(W.Run(truth.C, 1, 3 * truth.C, truth.C))
        host = [oracle.pchase_trace(r.n_elems, r.stride, r.length) for r in runs]
        obs_host = [oracle.cache_sim(truth.C, truth.b, truth.ways, truth.sets, truth.policy, t,
                                     seed=truth.seed, mapping=truth.mapping) for t in host]
        traces = [(torch.from_numpy(t.view(np.int32)).cuda(), r.length, r.warmup, r.n_elems,
                   r.stride) for t, r in zip(host, runs)]
        plan = api.SimPlan(cands, traces)
        words, offs = [], [0]
        for o in obs_host:
            wv = np.packbits(o, bitorder="little")
            wv = np.concatenate([wv, np.zeros((-wv.size) % 4, dtype=np.uint8)]).view(np.uint32)
            words.append(wv)
            offs.append(offs[-1] + wv.size)
        obs = torch.from_numpy(np.concatenate(words).view(np.int32)).cuda()
        owo = torch.tensor(offs[:-1], dtype=torch.int64, device="cuda")
        dist = plan.match(obs, owo).cpu().numpy()
        for ci, g in enumerate(cands):
            want = sum(int((oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, t, seed=g.seed,
                                             mapping=g.mapping) != o).sum())
                       for t, o in zip(host, obs_host))
            assert dist[ci] == want, (truth, g)
        ti = [i for i, g in enumerate(cands) if g == truth][0]
        assert dist[ti] == 0
        assert (dist > 0).sum() >= 4  # other mappings and policies are told apart
