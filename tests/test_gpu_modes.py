"""Every set mode of the simulator (way scan, line table, whole-step batch)
against the oracle, with each mode forced on items it would not normally
get: tiny and huge associativity, one set and many, lines repeated inside a
32-access step, and random (non-chain) traces."""
import math

import numpy as np
import pytest

import oracle
from paper_1509_02308_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1509_02308_gb300 import api

# split_*: every item whose T has a power-of-two factor is split into as many
# set-parts as that allows (up to 8), each part on its own warp
SPLIT = {"max_split": 8, "split_cost_ns": 1}
TUNES = {
    "batch_all": {"batch_max_sets": 1 << 30},
    "no_batch_scan8": {"batch_max_sets": 0xFFFFFFFF, "scan_max_ways": 8},
    "no_batch_scan32": {"batch_max_sets": 0xFFFFFFFF, "scan_max_ways": 32},
    "no_batch_table": {"batch_max_sets": 0xFFFFFFFF, "scan_max_ways": 1},
    "default": None,
    "split_batch": {**SPLIT, "batch_max_sets": 1 << 30},
    "split_scan": {**SPLIT, "batch_max_sets": 0xFFFFFFFF, "scan_max_ways": 32},
    "split_table": {**SPLIT, "batch_max_sets": 0xFFFFFFFF, "scan_max_ways": 1},
    "split_default": SPLIT,
}


def geoms_under_test():
    out = []
    for policy in (W.LRU, W.FIFO, W.RANDOM):
        for (C, b, a) in [(128, 32, 4), (256, 32, 8), (512, 32, 16), (1024, 32, 32),
                          (1536, 32, 48), (4096, 32, 128), (8192, 16, 512), (32768, 32, 1024),
                          (1024, 32, 1), (1024, 32, 2), (2048, 64, 4), (3072, 32, 24),
                          (6144, 64, 32), (16384, 128, 4), (12288, 32, 96), (192, 16, 3),
                          (960, 16, 6)]:
            lines = C // b
            if lines % a:
                continue
            out.append(W.Geom(C, b, a, lines // a, policy, 0xABC0 + a + 7 * policy))
    return out


def traces_under_test(rng):
    tr = []
    # uniform chains around each capacity scale, 3 passes + a ragged tail
    for (nb, sb) in [(160, 4), (300, 8), (640, 32), (1100, 4), (2100, 64), (5000, 32),
                     (9000, 16), (40000, 32), (20000, 4), (16512, 4), (16640, 128)]:
        n, s = nb // 4, sb // 4
        per = n // math.gcd(n, s)
        tr.append(oracle.pchase_trace(n, s, 3 * per + 17))
    # tiny working sets: the same lines come back inside one 32-access step
    for m in (2, 3, 5, 9, 17, 33):
        lines = rng.integers(0, 64, size=m) * 8
        tr.append(np.tile(lines, 3000 // m + 1)[:3000].astype(np.uint32))
    # random traces with a hot subset
    for k in range(4):
        tr.append(W.random_index_trace(5000, 3000 * (k + 1), seed=100 + k, hot=6))
    return tr


@pytest.mark.parametrize("tune_name", list(TUNES))
def test_modes_match_oracle(tune_name):
    rng = np.random.Generator(np.random.PCG64(42))
    geoms = geoms_under_test()
    host = traces_under_test(rng)
    n_el = [int(t.max()) + 1 for t in host]
    dev = [torch.from_numpy(t.view(np.int32)).cuda() for t in host]
    traces = [(d, t.size, min(t.size, 50), n, 1) for d, t, n in zip(dev, host, n_el)]
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
            want = oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, t, seed=g.seed)
            got = api.unpack_bits(b[int(plan.word_offsets[i]):], t.size)
            assert np.array_equal(got, want), (tune_name, g, ti, int(np.argmax(got != want)))
            assert c[i, 0] == want.sum() and c[i, 1] == want[50:].sum()


def test_batch_mode_long_thrash_and_refill():
    """Long single-set runs that alternate thrashing and fitting phases, so
    the LRU recency ring compacts many times and FIFO/RANDOM wrap often."""
    rng = np.random.Generator(np.random.PCG64(9))
    geoms = [W.Geom(a * 32, 32, a, 1, p, 77 + p) for a in (5, 40, 300) for p in (0, 1, 2)]
    host = []
    for a_scale in (5, 40, 300):
        parts = []
        for ph in range(12):
            m = int(a_scale * (0.5 if ph % 2 else 1.6)) + 1
            base = rng.integers(0, 4 * a_scale) * 8
            seq = (base + np.arange(m) * 8) % (8 * 8 * a_scale)
            parts.append(np.tile(seq, 4).astype(np.uint32))
        host.append(np.concatenate(parts))
    dev = [torch.from_numpy(t.view(np.int32)).cuda() for t in host]
    traces = [(d, t.size, 0, int(t.max()) + 1, 1) for d, t in zip(dev, host)]
    plan = api.SimPlan(geoms, traces, tune={"batch_max_sets": 1 << 30})
    bitmaps, _ = plan.run()
    torch.cuda.synchronize()
    b = bitmaps.cpu().numpy().view(np.uint32)
    for gi, g in enumerate(geoms):
        for ti, t in enumerate(host):
            i = gi * len(host) + ti
            want = oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, t, seed=g.seed)
            got = api.unpack_bits(b[int(plan.word_offsets[i]):], t.size)
            assert np.array_equal(got, want), (g, ti, int(np.argmax(got != want)))


@pytest.mark.parametrize("tune_name", ["batch_all", "default"])
def test_cyclic_periods_around_the_ways(tune_name):
    """Cyclic traces over m lines with m from 1 to 2a+1 and past 32, on 1-3
    sets: steady states that all hit, that all miss with each line coming back
    inside a 32-access step, and that mix; lines touched once or twice in a
    row (dense and half-dense run heads)."""
    geoms = [W.Geom(T * a * 32, 32, a, T, p, 0x5100 + 31 * a + T + 7 * p)
             for T in (1, 2, 3) for a in (1, 2, 3, 4, 7, 8, 12, 16, 31) for p in (0, 1, 2)]
    host = []
    for m in (1, 2, 3, 4, 5, 6, 7, 8, 9, 11, 13, 15, 16, 17, 24, 25, 31, 32, 33, 34, 40, 47,
              63, 64, 65):
        cyc = (np.arange(m) * 8).astype(np.uint32)
        host.append(np.tile(cyc, 4000 // m + 1)[:4000])
        host.append(np.repeat(np.tile(cyc, 2000 // m + 1), 2)[:4000] + 1)
    n_el = [int(t.max()) + 1 for t in host]
    dev = [torch.from_numpy(t.view(np.int32)).cuda() for t in host]
    traces = [(d, t.size, 40, n, 1) for d, t, n in zip(dev, host, n_el)]
    plan = api.SimPlan(geoms, traces, tune=TUNES[tune_name])
    bitmaps, counts = plan.run()
    torch.cuda.synchronize()
    b = bitmaps.cpu().numpy().view(np.uint32)
    c = counts.view(-1, 2).cpu().numpy()
    for gi, g in enumerate(geoms):
        for ti, t in enumerate(host):
            i = gi * len(host) + ti
            want = oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, t, seed=g.seed)
            got = api.unpack_bits(b[int(plan.word_offsets[i]):], t.size)
            assert np.array_equal(got, want), (tune_name, g, ti, int(np.argmax(got != want)))
            assert c[i, 0] == want.sum() and c[i, 1] == want[40:].sum()
