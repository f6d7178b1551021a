"""Caches whose set state fits no shared-memory arena (the mixed
configuration's large L2 caches, up to 128 MB): whole way-scan units with the
state in global memory, against the oracle bit for bit, alone, as the lower
level of a cache cascade (queued, filtered) and in the matcher."""
import numpy as np
import pytest

import oracle
from paper_1509_02308_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1509_02308_gb300 import api

MB = 1 << 20


def _sim(g, tr):
    return oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr, seed=g.seed)


def test_large_caches_match_oracle():
    geoms = [W.Geom(128 * MB, 128, 16, 65536, W.LRU),       # 1 Mi lines
             W.Geom(8 * MB, 32, 16, 16384, W.FIFO),         # 256 Ki lines
             W.Geom(8 * MB, 32, 16, 16384, W.RANDOM, 11),
             W.Geom(6 * MB, 64, 12, 8192, W.WEIGHTED, 3)]
    host, descs, pairs = [], [], []
    # chains that fit (held) and chains that overflow every set, for each
    for gi, g in enumerate(geoms):
        for f in (0.75, 1.25):
            s = g.b // 4
            n = int(g.C * f) // 4 // s * s
            L = 2 * (n // s) + 77
            host.append(oracle.pchase_trace(n, s, L))
            descs.append((None, L, n // s, n, s))
            pairs.append((gi, len(host) - 1))
    # general traces, explicit
    for k, gi in enumerate((1, 2, 3)):
        t = W.random_index_trace(40000, geoms[gi].C // 4 * 2, seed=70 + k, hot=6)
        host.append(t)
        descs.append((torch.from_numpy(t.view(np.int32)).cuda(), t.size, 0, int(t.max()) + 1, 1))
        pairs.append((gi, len(host) - 1))
    # splits off: every item keeps its whole set state in global memory
    plan = api.SimPlan(geoms, descs, pairs=pairs, tune={"max_split": 1})
    d = dict(kv.split("=", 1) for kv in plan.description.split())
    assert int(d["global_state"]) == len(pairs), plan.description
    # with splits on, the 128 MB cache still does (its parts fit nowhere)
    d2 = dict(kv.split("=", 1) for kv in api.SimPlan(geoms, descs, pairs=pairs).description.split())
    assert int(d2["global_state"]) >= 2
    bitmaps, counts = plan.run()
    torch.cuda.synchronize()
    b = bitmaps.cpu().numpy().view(np.uint32)
    c = counts.view(-1, 2).cpu().numpy()
    for i, (gi, ti) in enumerate(pairs):
        want = _sim(geoms[gi], host[ti])
        got = api.unpack_bits(b[int(plan.word_offsets[i]):], host[ti].size)
        assert np.array_equal(got, want), (geoms[gi], ti, int(np.argmax(got != want)))
        assert c[i, 0] == want.sum() and c[i, 1] == want[descs[ti][2]:].sum()
    # the matcher (candidates x traces, one observation: each unit owns its state)
    cands, tix = [geoms[1], geoms[2], geoms[3]], [2, 3, len(host) - 2]
    mplan = api.SimPlan(cands, [descs[t] for t in tix], tune={"max_split": 1})
    obs_host = [_sim(cands[0], host[t]) for t in tix]
    words, offs = [], [0]
    for o in obs_host:
        wv = np.packbits(o, bitorder="little")
        wv = np.concatenate([wv, np.zeros((-wv.size) % 4, dtype=np.uint8)]).view(np.uint32)
        words.append(wv)
        offs.append(offs[-1] + wv.size)
    obs = torch.from_numpy(np.concatenate(words).view(np.int32)).cuda()
    owo = torch.tensor(offs[:-1], dtype=torch.int64, device="cuda")
    dist = mplan.match(obs, owo).cpu().numpy()
    for ci, g in enumerate(cands):
        want = sum(int((_sim(g, host[t]) != o).sum()) for t, o in zip(tix, obs_host))
        assert dist[ci] == want, (g, dist[ci], want)
    assert dist[0] == 0 and (dist[1:] > 0).all()


def test_large_l2_behind_an_l1():
    l1 = [W.Geom(64 << 10, 64, 4, 256, W.LRU), W.Geom(32 << 10, 32, 8, 128, W.FIFO)]
    l2 = [W.Geom(16 * MB, 64, 16, 16384, W.LRU), W.Geom(12 * MB, 128, 24, 4096, W.RANDOM, 2)]
    host, descs = [], []
    for (nb, sb) in ((20 * MB, 64), (10 * MB, 256), (15 * MB, 128)):
        n, s = nb // 4, sb // 4
        L = 2 * (n // s) + 5
        host.append(oracle.pchase_trace(n, s, L))
        descs.append((None, L, n // s, n, s))
    pairs = [(g, t) for g in range(2) for t in range(len(host))]
    hp = api.HierarchyPlan([l1, l2], descs, pairs=pairs, tune={"max_split": 1})
    assert " global_state=0 " in hp.plans[0].description
    assert " global_state=0 " not in hp.plans[1].description
    outs = hp.run()
    torch.cuda.synchronize()
    words = [o[0].cpu().numpy().view(np.uint32) for o in outs]
    for i, (g, t) in enumerate(pairs):
        lv = [dict(C=x.C, b=x.b, ways=x.ways, T=x.sets, policy=x.policy, seed=x.seed)
              for x in (l1[g], l2[g])]
        want = oracle.hierarchy(lv, host[t])
        for k in range(2):
            got = api.unpack_bits(words[k][int(hp.word_offsets[i]):], host[t].size)
            assert np.array_equal(got, want[k]), (i, k, int(np.argmax(got != want[k])))


def test_batched_inference_refuses_global_state():
    g = [W.Geom(8 * MB, 32, 16, 16384, W.LRU), W.Geom(16 << 10, 64, 4, 64, W.LRU)]
    plan = api.SimPlan(g, [(None, 1000, 0, 1 << 20, 8)], tune={"max_split": 1})
    assert " global_state=1 " in plan.description, plan.description
    lats = torch.zeros(2, 1000, dtype=torch.float32, device="cuda")
    with pytest.raises(Exception):
        api.infer_batch(plan, lats)


def test_pool_regions_are_reused_from_unit_to_unit():
    """Global-state units of 24 large caches (1 Mi and 256 Ki lines, every
    policy) through a pool of only 4 warps, so each warp's region holds one
    unit's state after another (larger and smaller caches in turn): every
    bitmap and count against the oracle."""
    geoms = [W.Geom(128 * MB, 128, 16, 65536, W.LRU), W.Geom(8 * MB, 32, 16, 16384, W.FIFO),
             W.Geom(8 * MB, 32, 16, 16384, W.RANDOM, 11), W.Geom(6 * MB, 64, 12, 8192, W.WEIGHTED, 3),
             W.Geom(64 * MB, 64, 8, 131072, W.FIFO), W.Geom(32 * MB, 128, 32, 8192, W.RANDOM, 5)]
    host, descs, pairs = [], [], []
    for k in range(24):
        gi = k % len(geoms)
        g = geoms[gi]
        if k % 3 == 2:
            t = W.random_index_trace(6000 + 97 * k, g.C // 4 * 2, seed=300 + k, hot=5)
            host.append(t)
            descs.append((torch.from_numpy(t.view(np.int32)).cuda(), t.size, 0, int(t.max()) + 1, 1))
        else:
            s = g.b // 4 * (1 + k % 2)
            n = int(g.C * (0.6 + 0.15 * (k % 5))) // 4 // s * s
            L = 5000 + 131 * k
            host.append(oracle.pchase_trace(n, s, L))
            descs.append((None, L, min(L, n // s), n, s))
        pairs.append((gi, k))
    plan = api.SimPlan(geoms, descs, pairs=pairs, tune={"max_split": 1, "pool_warps": 4})
    d = dict(kv.split("=", 1) for kv in plan.description.split())
    assert int(d["global_state"]) == 24 and d["pool"].startswith("4x"), plan.description
    for _ in range(2):  # a second run reuses the regions the first one left dirty
        bitmaps, counts = plan.run()
        torch.cuda.synchronize()
        b = bitmaps.cpu().numpy().view(np.uint32)
        c = counts.view(-1, 2).cpu().numpy()
        for i, (gi, ti) in enumerate(pairs):
            want = _sim(geoms[gi], host[ti])
            got = api.unpack_bits(b[int(plan.word_offsets[i]):], host[ti].size)
            assert np.array_equal(got, want), (i, geoms[gi], int(np.argmax(got != want)))
            assert c[i, 0] == want.sum() and c[i, 1] == want[descs[ti][2]:].sum()


def test_compact_lines_of_strided_analytic_chains():
    """Analytic chains whose stride is a whole number of lines over arrays far
    larger than any line table (tens of MB) visit only every lstep-th line;
    whole units key their state by line / lstep, so line-table and batch set
    modes fit where before only way scans did.  Single-set and few-set
    streams under LRU (also cut in time), FIFO and RANDOM, every bitmap
    against the oracle."""
    geoms = [W.Geom(16 << 10, 32, 16, 32, W.LRU), W.Geom(16 << 10, 32, 16, 32, W.FIFO),
             W.Geom(16 << 10, 128, 16, 8, W.RANDOM, 9), W.Geom(64 << 10, 64, 8, 128, W.LRU),
             W.Geom(32 << 10, 32, 4, 256, W.FIFO)]
    streams = [(14 * MB, 4096), (57 * MB, 256), (24 * MB, 2048), (9 * MB, 1024)]
    host, descs = [], []
    for nb, sb in streams:
        n, s = nb // 4, sb // 4
        L = 150000
        host.append(oracle.pchase_trace(n, s, L))
        descs.append((None, L, min(L, n // s), n, s))
    pairs = [(g, t) for g in range(len(geoms)) for t in range(len(streams))]
    for tune in (None, {"split_cost_ns": 1, "max_split": 8}):
        plan = api.SimPlan(geoms, descs, pairs=pairs, tune=tune)
        d = dict(kv.split("=", 1) for kv in plan.description.split())
        assert int(d["table"]) + int(d["batch"]) > 0, plan.description
        if tune:
            assert int(d["time_split"]) > 0, plan.description
        bitmaps, counts = plan.run()
        torch.cuda.synchronize()
        b = bitmaps.cpu().numpy().view(np.uint32)
        c = counts.view(-1, 2).cpu().numpy()
        for i, (gi, ti) in enumerate(pairs):
            want = _sim(geoms[gi], host[ti])
            got = api.unpack_bits(b[int(plan.word_offsets[i]):], host[ti].size)
            assert np.array_equal(got, want), (tune, i, geoms[gi], int(np.argmax(got != want)))
            assert c[i, 0] == want.sum() and c[i, 1] == want[descs[ti][2]:].sum()
