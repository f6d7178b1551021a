"""Unequal sets (the L2 TLB of Sec. 4.4, Fig. 9: one set of 17 entries and
six of 8) against the oracle, bit for bit: alone over the paper's 2 MB
chains and general traces, as the lower level of an L1 TLB -> L2 TLB
cascade (a filtered, queued run), and in the matcher."""
import numpy as np
import pytest

import oracle
from paper_1509_02308_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1509_02308_gb300 import api

PAGE = 2 << 20


def _want(g, tr, flt=None):
    return oracle.cache_sim_uneq(g.C, g.b, g.ways, g.sets, g.extra, g.policy, tr, filter=flt)


def uneq_geoms():
    return [W.Geom(65 * PAGE, PAGE, 8, 7, W.LRU, extra=9),
            W.Geom(65 * PAGE, PAGE, 8, 7, W.FIFO, extra=9),
            W.Geom((3 * 2 + 1) * 32, 32, 2, 3, W.LRU, extra=1),
            W.Geom((5 * 4 + 7) * 64, 64, 4, 5, W.FIFO, extra=7),
            W.Geom((1 * 4 + 3) * 32, 32, 4, 1, W.LRU, extra=3),
            W.Geom((12 * 16 + 40) * 128, 128, 16, 12, W.LRU, extra=40)]


def test_unequal_sets_match_oracle():
    rng = np.random.Generator(np.random.PCG64(9))
    geoms = uneq_geoms()
    host, descs = [], []
    # Fig. 9's sweep: 2 MB strides over 60 .. 80 pages (analytic chains)
    for n_pages in (60, 65, 66, 67, 70, 72, 80):
        n, L = n_pages * PAGE // 4, 5 * n_pages + 3
        host.append(oracle.pchase_trace(n, PAGE // 4, L))
        descs.append((None, L, n_pages, n, PAGE // 4))
    # smaller strides and general traces, explicit
    for (nb, sb, L) in [(4096, 32, 3000), (9000, 64, 7001), (30000, 128, 12000)]:
        t = oracle.pchase_trace(nb // 4, sb // 4, L)
        host.append(t)
        descs.append((torch.from_numpy(t.view(np.int32)).cuda(), L, 0, nb // 4, sb // 4))
    for k, (L, n_el) in enumerate([(5000, 2000), (9000, 40000), (700, 300)]):
        t = W.random_index_trace(L, n_el, seed=40 + k, hot=5)
        host.append(t)
        descs.append((torch.from_numpy(t.view(np.int32)).cuda(), L, 0, n_el, 1))
    lines = rng.integers(0, 300, size=23).astype(np.uint32) * 8
    t = np.tile(lines, 200)
    host.append(t)
    descs.append((torch.from_numpy(t.view(np.int32)).cuda(), t.size, 0, int(t.max()) + 1, 1))
    plan = api.SimPlan(geoms, descs)
    d = dict(kv.split("=", 1) for kv in plan.description.split())
    assert int(d["split"]) == 0 and int(d["time_split"]) == 0
    bitmaps, counts = plan.run()
    torch.cuda.synchronize()
    b = bitmaps.cpu().numpy().view(np.uint32)
    c = counts.view(-1, 2).cpu().numpy()
    for gi, g in enumerate(geoms):
        for ti, (tr, ds) in enumerate(zip(host, descs)):
            i = gi * len(host) + ti
            want = _want(g, tr)
            got = api.unpack_bits(b[int(plan.word_offsets[i]):], tr.size)
            assert np.array_equal(got, want), (g, ti, int(np.argmax(got != want)))
            assert c[i, 0] == want.sum() and c[i, 1] == want[ds[2]:].sum(), (g, ti)


def test_unequal_l2_tlb_behind_the_l1_tlb():
    """Sec. 4.4's TLB path: a 16-entry fully associative L1 TLB in front of
    the unequal L2 TLB (the lower level runs filtered by the L1 misses)."""
    l1 = [W.Geom(16 * PAGE, PAGE, 16, 1, W.LRU)]
    l2 = [W.Geom(65 * PAGE, PAGE, 8, 7, W.LRU, extra=9)]
    host, descs = [], []
    for n_pages in (10, 17, 40, 65, 66, 69, 72, 90):
        n, L = n_pages * PAGE // 4, 4 * n_pages + 1
        host.append(oracle.pchase_trace(n, PAGE // 4, L))
        descs.append((None, L, n_pages, n, PAGE // 4))
    hp = api.HierarchyPlan([l1, l2], descs, pairs=[(0, t) for t in range(len(descs))])
    outs = hp.run()
    torch.cuda.synchronize()
    words = [o[0].cpu().numpy().view(np.uint32) for o in outs]
    for i, tr in enumerate(host):
        lv = [dict(C=g.C, b=g.b, ways=g.ways, T=g.sets, policy=g.policy, extra=g.extra)
              for g in (l1[0], l2[0])]
        want = oracle.hierarchy(lv, tr)
        for k in range(2):
            got = api.unpack_bits(words[k][int(hp.word_offsets[i]):], tr.size)
            assert np.array_equal(got, want[k]), (i, k)


def test_matcher_tells_unequal_sets_apart():
    """Observations of the unequal L2 TLB against candidates with equal
    sets of the same capacity and other splits of it: distances equal the
    oracle's, the truth is at 0 and every other candidate above it."""
    truth = W.Geom(65 * PAGE, PAGE, 8, 7, W.LRU, extra=9)
    cands = [truth, W.Geom(65 * PAGE, PAGE, 8, 7, W.FIFO, extra=9),
             W.Geom(65 * PAGE, PAGE, 5, 13, W.LRU),          # 65 entries, equal sets
             W.Geom(65 * PAGE, PAGE, 65, 1, W.LRU),          # fully associative
             W.Geom(65 * PAGE, PAGE, 9, 7, W.LRU, extra=2),  # another unequal split
             W.Geom(64 * PAGE, PAGE, 8, 8, W.LRU)]
    host, descs = [], []
    for n_pages in range(60, 76, 3):
        n, L = n_pages * PAGE // 4, 4 * n_pages
        host.append(oracle.pchase_trace(n, PAGE // 4, L))
        descs.append((None, L, n_pages, n, PAGE // 4))

    def sim(g, tr):
        if g.extra:
            return _want(g, tr)
        return oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr)

    obs_host = [sim(truth, tr) for tr in host]
    plan = api.SimPlan(cands, descs)
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
        want = sum(int((sim(g, tr) != o).sum()) for tr, o in zip(host, obs_host))
        assert dist[ci] == want, (g, dist[ci], want)
    assert dist[0] == 0 and (dist[2:] > 0).all()
