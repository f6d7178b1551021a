"""Cache and TLB hierarchies (Sec. 3's L1 -> L2 path, Sec. 4.4's L1 -> L2 TLB
path): every level against the oracle's cascade, bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1509_02308_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1509_02308_gb300 import api
    from paper_1509_02308_gb300 import capi as C


def _lv(g):
    return dict(C=g.C, b=g.b, ways=g.ways, T=g.sets, policy=g.policy, seed=g.seed,
                mapping=g.mapping, extra=g.extra)


def _check(levels, traces_host, traces_dev, pairs, tune=None, tag=""):
    hp = api.HierarchyPlan(levels, traces_dev, pairs=pairs, tune=tune)
    outs = hp.run()
    torch.cuda.synchronize()
    words = [o[0].cpu().numpy().view(np.uint32) for o in outs]
    counts = [o[1].view(-1, 2).cpu().numpy() for o in outs]
    for i, (g, t) in enumerate(pairs):
        tr = traces_host[t]
        want = oracle.hierarchy([_lv(lv[g]) for lv in levels], tr)
        for k in range(len(levels)):
            got = api.unpack_bits(words[k][int(hp.word_offsets[i]):], tr.size)
            assert np.array_equal(got, want[k]), (tag, i, k, int(np.argmax(got != want[k])))
            assert counts[k][i, 0] == want[k].sum()


@pytest.mark.parametrize("tune", [None, {"batch_max_sets": 1 << 30},
                                  {"batch_max_sets": 0xFFFFFFFF, "scan_max_ways": 1},
                                  {"max_split": 8, "split_cost_ns": 1}])
def test_two_level_cache_hierarchy_matches_oracle(tune):
    rng = np.random.Generator(np.random.PCG64(4))
    l1 = [W.Geom(1024, 32, 4, 8, W.LRU), W.Geom(2048, 64, 2, 16, W.FIFO),
          W.Geom(1536, 32, 3, 16, W.RANDOM, 71), W.Geom(512, 16, 32, 1, W.LRU),
          W.Geom(1024, 32, 4, 8, W.WEIGHTED, 5), W.Geom(3072, 32, 96, 1, W.LRU, mapping=0)]
    l2 = [W.Geom(16384, 64, 8, 32, W.LRU), W.Geom(32768, 128, 16, 16, W.RANDOM, 9),
          W.Geom(12288, 32, 96, 4, W.LRU, mapping=2), W.Geom(8192, 32, 4, 64, W.FIFO),
          W.Geom(24576, 64, 12, 32, W.WEIGHTED, 13), W.Geom(65536, 256, 16, 16, W.LRU)]
    host = []
    for (nb, sb) in [(900, 4), (1500, 32), (3000, 8), (6000, 64), (20000, 32), (40000, 128),
                     (9000, 4)]:
        n, s = nb // 4, sb // 4
        host.append(oracle.pchase_trace(n, s, 3 * (n // s) + 11))
    for m in (5, 19, 70):
        lines = rng.integers(0, 600, size=m) * 8
        host.append(np.tile(lines, 3000 // m + 1)[:3000].astype(np.uint32))
    host.append(W.random_index_trace(5000, 20000, seed=12, hot=6))
    dev = [(torch.from_numpy(t.view(np.int32)).cuda(), t.size, 0, int(t.max()) + 1, 1)
           for t in host]
    pairs = [(g, t) for g in range(len(l1)) for t in range(len(host))]
    _check([l1, l2], host, dev, pairs, tune=tune, tag=str(tune))


def test_three_levels_and_analytic_chains():
    l1 = [W.Geom(1024, 32, 2, 16, W.LRU)]
    l2 = [W.Geom(8192, 64, 4, 32, W.FIFO)]
    l3 = [W.Geom(65536, 128, 8, 64, W.LRU)]
    sizes = [512, 2048, 6144, 12288, 40000, 100000]
    host, dev = [], []
    for nb in sizes:
        n = nb // 4
        L = 4 * (n // 8) + 5
        host.append(oracle.pchase_trace(n, 8, L))
        dev.append((None, L, 0, n, 8))
    _check([l1, l2, l3], host, dev, [(0, t) for t in range(len(sizes))])


def test_tlb_cascade_two_megabyte_pages():
    """Sec. 4.4: a 16-entry fully associative L1 TLB and a 7 x 8 L2 TLB over
    2 MB pages, driven by s = 2 MB chains of 1 to 70 pages (analytic, no
    trace array), and a 4 KB-page pair (16 entries, 64 x 8) over 4 KB strides."""
    page = 2 << 20
    l1 = [W.Geom(16 * page, page, 16, 1, W.LRU), W.Geom(16 * 4096, 4096, 16, 1, W.LRU)]
    l2 = [W.Geom(56 * page, page, 8, 7, W.LRU), W.Geom(512 * 4096, 4096, 8, 64, W.LRU)]
    host, dev, pairs = [], [], []
    for g, pg, counts in ((0, page, (1, 15, 16, 17, 33, 56, 57, 70)),
                          (1, 4096, (1, 16, 17, 100, 511, 512, 513, 600, 2000))):
        for n_pages in counts:
            n = n_pages * pg // 4
            L = 5 * n_pages
            host.append(oracle.pchase_trace(n, pg // 4, L))
            dev.append((None, L, n_pages, n, pg // 4))
            pairs.append((g, len(host) - 1))
    _check([l1, l2], host, dev, pairs)


def test_filtered_run_needs_a_filtered_plan():
    g = [W.Geom(1024, 32, 4, 8)]
    plan = api.SimPlan(g, [(None, 100, 0, 1000, 1)])
    bm = torch.zeros(8, dtype=torch.int32, device="cuda")
    wo = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(Exception):
        plan.run_filtered(bm, wo)
    L = C.load()
    assert L.pchase_last_error_string()


def test_hierarchy_workload_sample_matches_oracle():
    """A sample of the hierarchy workload the bench times (cache cascade and
    TLB cascade, the unequal L2 TLB over 2 MB pages among them), every level
    against the oracle's cascade."""
    l1, l2, t1, t2, runs = W.hierarchy_config(n_items=48)
    keep = [i for i, r in enumerate(runs) if r.length <= 120000][:24]
    assert any(t2[i].extra for i in keep)
    host = [oracle.pchase_trace(runs[i].n_elems, runs[i].stride, runs[i].length) for i in keep]
    dev = [(None, runs[i].length, runs[i].warmup, runs[i].n_elems, runs[i].stride) for i in keep]
    for levels in ([[l1[i] for i in keep], [l2[i] for i in keep]],
                   [[t1[i] for i in keep], [t2[i] for i in keep]]):
        _check(levels, host, dev, [(k, k) for k in range(len(keep))])
