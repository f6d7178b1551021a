"""LRU items cut in time: a part that starts at access c0 first rebuilds every
set's recency order from the accesses before c0 (under LRU replacement,
Sec. 3's policy for the caches the P-chase meets, a set holds exactly its a
most recently used distinct lines), then steps on from c0.  Bitmaps, counts
and the matcher's distances against the oracle, bit for bit."""
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
    "forced16": {"split_cost_ns": 1, "max_split": 16},
    "forced3": {"split_cost_ns": 1, "max_split": 3},
}


def lru_geoms():
    return [W.Geom(1024, 32, 32, 1, W.LRU), W.Geom(2048, 64, 32, 1, W.LRU),
            W.Geom(512, 4, 128, 1, W.LRU), W.Geom(16 * 4096, 4096, 16, 1, W.LRU),
            W.Geom(4096, 32, 8, 16, W.LRU), W.Geom(12288, 32, 96, 4, W.LRU, mapping=2),
            W.Geom(2048, 32, 16, 4, W.LRU, mapping=1),
            # not LRU: never cut in time, share the plan
            W.Geom(1024, 32, 32, 1, W.FIFO), W.Geom(1024, 32, 32, 1, W.RANDOM, 77)]


def host_traces(rng):
    """(host trace, device descriptor) pairs: chains that thrash, chains that
    stay resident, a chain over one set of many, repeats of a few lines,
    general index traces; ragged lengths, warm-ups across part bounds."""
    out = []
    for (nb, sb, L, w) in [(1024 + 64, 32, 9000 + 37, 100), (2048 + 256, 64, 20000, 0),
                           (900, 32, 5000, 4500), (3 * 1024, 32, 2100, 0),
                           (40 * 4096, 4096, 4000, 64), (8192 * 4, 512, 12345, 0),
                           (12288 + 256, 32, 16000, 2000), (4096, 4, 30000, 0)]:
        n, s = nb // 4, sb // 4
        out.append((oracle.pchase_trace(n, s, L), (None, L, w, n, s)))
    for m in (7, 40, 300):
        lines = rng.integers(0, 500, size=m).astype(np.uint32) * 8
        t = np.tile(lines, 9000 // m + 1)[:9000 + m].astype(np.uint32)
        out.append((t, t))
    for k, (L, n_el) in enumerate([(6000, 3000), (20000, 40000), (1300, 800)]):
        t = W.random_index_trace(L, n_el, seed=900 + k, hot=4)
        out.append((t, t))
    descs = []
    for t, d in out:
        if isinstance(d, np.ndarray):
            descs.append((torch.from_numpy(d.view(np.int32)).cuda(), d.size, min(d.size, 700),
                           int(d.max()) + 1, 1))
        else:
            descs.append(d)
    return [t for t, _ in out], descs


def _want(g, tr):
    return oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr, seed=g.seed,
                            mapping=g.mapping)


@pytest.mark.parametrize("tune_name", list(TUNES))
def test_time_split_matches_oracle(tune_name):
    rng = np.random.Generator(np.random.PCG64(31))
    geoms = lru_geoms()
    host, descs = host_traces(rng)
    plan = api.SimPlan(geoms, descs, tune=TUNES[tune_name])
    d = dict(kv.split("=", 1) for kv in plan.description.split())
    if tune_name != "default":
        assert int(d["time_split"]) >= 10, plan.description
    bitmaps, counts = plan.run()
    torch.cuda.synchronize()
    b = bitmaps.cpu().numpy().view(np.uint32)
    c = counts.view(-1, 2).cpu().numpy()
    for gi, g in enumerate(geoms):
        for ti, (tr, ds) in enumerate(zip(host, descs)):
            i = gi * len(host) + ti
            want = _want(g, tr)
            got = api.unpack_bits(b[int(plan.word_offsets[i]):], tr.size)
            assert np.array_equal(got, want), (tune_name, g, ti, int(np.argmax(got != want)))
            assert c[i, 0] == want.sum() and c[i, 1] == want[ds[2]:].sum(), (tune_name, g, ti)


def test_time_split_matcher_distances():
    """Observations of one LRU geometry matched against LRU candidates that
    are cut in time: every distance is the oracle's Hamming distance."""
    rng = np.random.Generator(np.random.PCG64(5))
    truth = W.Geom(2048, 32, 64, 1, W.LRU)
    cands = [W.Geom(2048, 32, 64, 1, W.LRU), W.Geom(1024, 32, 32, 1, W.LRU),
             W.Geom(4096, 32, 128, 1, W.LRU), W.Geom(2048, 32, 16, 4, W.LRU),
             W.Geom(2048, 32, 64, 1, W.FIFO), W.Geom(2048, 64, 32, 1, W.LRU)]
    host, descs = [], []
    for nb in (2048 - 64, 2048 + 32, 2048 + 512, 4096 + 96, 8192):
        n, L = nb // 4, 8 * (nb // 32) + 77
        host.append(oracle.pchase_trace(n, 8, L))
        descs.append((None, L, nb // 32, n, 8))
    t = W.random_index_trace(7000, 3000, seed=8, hot=3)
    host.append(t)
    descs.append((torch.from_numpy(t.view(np.int32)).cuda(), t.size, 0, 3000, 1))
    obs_host = [_want(truth, tr) for tr in host]
    plan = api.SimPlan(cands, descs, tune={"split_cost_ns": 1, "max_split": 8})
    assert " time_split=0 " not in plan.description, plan.description
    words, offs = [], [0]
    for o in obs_host:
        wv = np.packbits(o, bitorder="little")
        wv = np.concatenate([wv, np.zeros((-wv.size) % 4, dtype=np.uint8)]).view(np.uint32)
        words.append(wv)
        offs.append(offs[-1] + wv.size)
    obs = torch.from_numpy(np.concatenate(words).view(np.int32)).cuda()
    owo = torch.tensor(offs[:-1], dtype=torch.int64, device="cuda")
    dist = plan.match(obs, owo).cpu().numpy()
    wants = []
    for ci, g in enumerate(cands):
        want = sum(int((_want(g, tr) != o).sum()) for tr, o in zip(host, obs_host))
        wants.append(want)
        assert dist[ci] == want, (g, dist[ci], want)
    assert dist[0] == 0 and (dist[1:] > 0).all()
    # with a bound, distances at or under it stay exact and the others are
    # only known to be above it, whichever time part stopped first
    for bound in (0, min(wants[1:])):
        db = plan.match(obs, owo, stop_above=bound).cpu().numpy()
        for ci, want in enumerate(wants):
            if want <= bound:
                assert db[ci] == want, (bound, ci)
            else:
                assert db[ci] > bound, (bound, ci)
