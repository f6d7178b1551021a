"""Parity of S4 (classification), S5 (matcher) and the canonical pick with
the CPU oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1509_02308_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1509_02308_gb300 import api


def synth_latency(miss: np.ndarray, seed: int, t0=100.0, tm=300.0, jitter=0.02, spikes=0.005):
    rng = np.random.Generator(np.random.PCG64(seed))
    lat = (t0 + tm * miss) * (1.0 + jitter * rng.standard_normal(miss.size))
    sp = rng.random(miss.size) < spikes
    lat[sp] *= rng.uniform(2, 10, size=int(sp.sum()))
    return lat.astype(np.float32)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 199, 200, 201, 1000, 4097, 65536, 300001])
def test_classify_matches_oracle(n):
    rng = np.random.Generator(np.random.PCG64(n))
    miss = (rng.random(n) < 0.35).astype(np.uint8)
    lat = synth_latency(miss, n)
    bits, w, thr = api.pchase_classify([torch.from_numpy(lat).cuda()])
    want, wthr = oracle.classify(lat)
    got = api.unpack_bits(bits.cpu().numpy().view(np.uint32), n)
    assert np.float32(thr[0].item()) == np.float32(wthr)
    assert np.array_equal(got, want)


def test_classify_edge_cases_batch():
    cases = [np.full(50, 7.0), np.array([5.0]), np.array([1.0, 2.0]), np.array([-3.0, 4.0, 4.0, -3.0]),
             np.repeat([10.0, 10.0, 50.0], 100), np.arange(1000, dtype=np.float64),
             np.concatenate([np.full(1000, 100.0), np.full(3, 1e6)]),
             np.array([0.0, 1.0, 3.0, 6.0, 10.0, 15.0])]
    lats = [torch.from_numpy(c.astype(np.float32)).cuda() for c in cases]
    bits, w, thr = api.pchase_classify(lats)
    b = bits.cpu().numpy().view(np.uint32)
    for i, c in enumerate(cases):
        want, wthr = oracle.classify(c.astype(np.float32))
        got = api.unpack_bits(b[int(w[i]):], c.size)
        assert np.float32(thr[i].item()) == np.float32(wthr), (i, thr[i].item(), wthr)
        assert np.array_equal(got, want), i


def test_classify_refuses_an_observation_longer_than_max_len():
    """An observation longer than the caller's max_len gets a NaN cut and all-0
    bits and writes no workspace byte outside its own bucket slice; the other
    observations keep the oracle's answer.  A guard region after the
    workspace proves nothing past the last slice is written."""
    from paper_1509_02308_gb300 import capi as C
    L = C.load()
    rng = np.random.Generator(np.random.PCG64(11))
    sizes = [900, 400, 3000]          # max_len below: 1000, so the last one is too long
    max_len = 1000
    lats = []
    for n in sizes:
        miss = (rng.random(n) < 0.4).astype(np.uint8)
        lats.append(synth_latency(miss, n))
    offs = np.zeros(len(sizes) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    words = np.zeros(len(sizes), dtype=np.int64)
    words[1:] = np.cumsum([(n + 31) // 32 for n in sizes])[:-1]
    nwords = sum((n + 31) // 32 for n in sizes)
    flat = torch.from_numpy(np.concatenate(lats)).cuda()
    d_offs, d_w = torch.from_numpy(offs).cuda(), torch.from_numpy(words).cuda()
    bits = torch.full((nwords,), -1, dtype=torch.int32, device="cuda")
    thr = torch.zeros(len(sizes), dtype=torch.float32, device="cuda")
    need = int(L.pchase_classify_workspace_bytes(len(sizes), max_len))
    guard = 1 << 16
    ws = torch.full((need + 256 + guard,), 0xA5, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) & ~255
    lead = base - ws.data_ptr()
    C.check(L.pchase_classify(flat.data_ptr(), d_offs.data_ptr(), len(sizes), max_len,
                              bits.data_ptr(), d_w.data_ptr(), thr.data_ptr(), base, None))
    torch.cuda.synchronize()
    tail = ws[lead + need:].cpu().numpy()
    assert (tail == 0xA5).all(), int(np.argmax(tail != 0xA5))
    b = bits.cpu().numpy().view(np.uint32)
    t = thr.cpu().numpy()
    for i, n in enumerate(sizes):
        got = api.unpack_bits(b[int(words[i]):], n)
        if n > max_len:
            assert np.isnan(t[i])
            assert not got.any()
        else:
            want, wthr = oracle.classify(lats[i])
            assert np.float32(t[i]) == np.float32(wthr)
            assert np.array_equal(got, want)


def small_candidates():
    grid = W.geometry_grid(capacities=(512, 768, 1024, 1536), line_sizes=(32, 64),
                           way_choices=(1, 2, 4, 8, 0))
    return [W.Geom(C, b, a, T, p, 1234 + i) for i, (C, b, a, T) in enumerate(grid)
            for p in (0, 1, 2)]


def small_plan(C0=768):
    runs = []
    for nb in (C0 // 2, C0 - 4, C0, C0 + 4, C0 + 32, C0 + 36, C0 + 64, C0 + 132, 2 * C0):
        n = nb // 4
        runs.append(W.Run(n, 1, 3 * n, n))
    for nb in (C0 + 64, C0 + 256, 2 * C0, 4 * C0):
        n = nb // 4
        runs.append(W.Run(n, 16, 3 * (n // 16), n // 16))
    return runs


def test_match_distances_equal_oracle():
    cands = small_candidates()
    runs = small_plan()
    host = [oracle.pchase_trace(r.n_elems, r.stride, r.length) for r in runs]
    truth = W.Geom(768, 64, 4, 3, W.LRU)
    obs_host = [oracle.cache_sim(truth.C, truth.b, truth.ways, truth.sets, 0, t) for t in host]
    # observed bitmaps with a few flipped bits so distances are not all 0
    rng = np.random.Generator(np.random.PCG64(5))
    for o in obs_host:
        flip = rng.random(o.size) < 0.01
        o[flip] ^= 1
    traces = [(torch.from_numpy(t.view(np.int32)).cuda(), r.length, r.warmup, r.n_elems, r.stride)
              for t, r in zip(host, runs)]
    plan = api.SimPlan(cands, traces)
    # the same candidates with every item split into set-parts
    split = api.SimPlan(cands, traces, tune={"max_split": 4, "split_cost_ns": 1})
    assert " split=0 " not in split.description
    words, offs = [], [0]
    for o in obs_host:
        wv = np.packbits(o, bitorder="little")
        wv = np.concatenate([wv, np.zeros((-wv.size) % 4, dtype=np.uint8)]).view(np.uint32)
        words.append(wv)
        offs.append(offs[-1] + wv.size)
    obs = torch.from_numpy(np.concatenate(words).view(np.int32)).cuda()
    owo = torch.tensor(offs[:-1], dtype=torch.int64, device="cuda")
    dist = plan.match(obs, owo).cpu().numpy().astype(np.uint64)
    rows = np.array([g.row() for g in cands], dtype=np.uint32)
    seeds = np.array([g.seed for g in cands], dtype=np.uint64)
    want = oracle.match(rows, seeds, host, obs_host)
    assert np.array_equal(dist, want)
    assert np.array_equal(split.match(obs, owo).cpu().numpy().astype(np.uint64), want)
    # early stop keeps every candidate at or under the bound exact
    bound = int(np.sort(want)[5])
    d2 = plan.match(obs, owo, stop_above=bound).cpu().numpy().astype(np.uint64)
    assert np.array_equal(d2[want <= bound], want[want <= bound])
    assert (d2[want > bound] > bound).all()
    d3 = split.match(obs, owo, stop_above=bound).cpu().numpy().astype(np.uint64)
    assert np.array_equal(d3[want <= bound], want[want <= bound])
    assert (d3[want > bound] > bound).all()
    # canonical pick
    pick = api.pchase_canonical_pick(cands, torch.from_numpy(want.astype(np.int64)).cuda())
    pi, nb = oracle.canonical_pick(rows, want)
    assert int(pick[0]) == pi and int(pick[1]) == nb


def test_infer_geometry_round_trip():
    cands = small_candidates()
    runs = small_plan()
    host = [oracle.pchase_trace(r.n_elems, r.stride, r.length) for r in runs]
    traces = [(torch.from_numpy(t.view(np.int32)).cuda(), r.length, r.warmup, r.n_elems, r.stride)
              for t, r in zip(host, runs)]
    plan = api.SimPlan(cands, traces)
    rows = np.array([g.row() for g in cands], dtype=np.uint32)
    seeds = np.array([g.seed for g in cands], dtype=np.uint64)
    for ti, truth in enumerate([cands[10], cands[37], cands[len(cands) - 5]]):
        miss = [oracle.cache_sim(truth.C, truth.b, truth.ways, truth.sets, truth.policy, t,
                                 seed=truth.seed) for t in host]
        lat = np.concatenate([synth_latency(m, 100 + ti * 7 + k, spikes=0.0)
                              for k, m in enumerate(miss)])
        dist, pick = plan.infer(torch.from_numpy(lat).cuda())
        torch.cuda.synchronize()
        # oracle: same pooled classification, match, pick
        obits, _ = oracle.classify(lat)
        obs, o = [], 0
        for r in runs:
            obs.append(obits[o:o + r.length])
            o += r.length
        want = oracle.match(rows, seeds, host, obs)
        assert np.array_equal(dist.cpu().numpy().astype(np.uint64), want)
        pi, nb = oracle.canonical_pick(rows, want)
        assert int(pick[0]) == pi and int(pick[1]) == nb
        assert want[pi] == 0
        # the pick is indistinguishable from the truth on this plan
        for t in host:
            g = cands[pi]
            assert np.array_equal(
                oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, t, seed=g.seed),
                oracle.cache_sim(truth.C, truth.b, truth.ways, truth.sets, truth.policy, t,
                                 seed=truth.seed))


def test_batched_inference_equals_one_by_one():
    """infer_geometry_batch over several observations (different truths,
    noise and spikes) returns, per observation, the distances and pick of
    infer_geometry on that observation alone; with a distance bound the
    candidates within it keep exact distances."""
    cands = small_candidates()
    runs = small_plan()
    host = [oracle.pchase_trace(r.n_elems, r.stride, r.length) for r in runs]
    traces = [(torch.from_numpy(t.view(np.int32)).cuda(), r.length, r.warmup, r.n_elems, r.stride)
              for t, r in zip(host, runs)]
    plan = api.SimPlan(cands, traces)
    truths = [cands[i] for i in (3, 10, 37, 58, 90, len(cands) - 5, len(cands) - 1)]
    lats = []
    for ti, truth in enumerate(truths):
        miss = [oracle.cache_sim(truth.C, truth.b, truth.ways, truth.sets, truth.policy, t,
                                 seed=truth.seed) for t in host]
        lats.append(np.concatenate([synth_latency(m, 500 + ti * 11 + k, spikes=0.002 * (ti % 2))
                                    for k, m in enumerate(miss)]))
    lat_t = torch.from_numpy(np.stack(lats)).cuda()
    for stop in (2**64 - 1, 0, 3):
        dist_b, pick_b = api.infer_batch(plan, lat_t, stop_above=stop)
        torch.cuda.synchronize()
        dist_b = dist_b.cpu().numpy().astype(np.uint64)
        pick_b = pick_b.cpu().numpy()
        for o in range(len(truths)):
            d1, p1 = plan.infer(lat_t[o].contiguous(), stop_above=stop)
            d1 = d1.cpu().numpy().astype(np.uint64)
            if stop == 2**64 - 1:
                assert np.array_equal(dist_b[o], d1)
            else:
                keep = d1 <= stop
                assert np.array_equal(dist_b[o][keep], d1[keep])
                assert (dist_b[o][~keep] > stop).all()
            if d1[int(p1[0])] <= stop:
                # an answer within the bound is exact, hence the same pick
                assert int(pick_b[o, 0]) == int(p1[0]) and int(pick_b[o, 1]) == int(p1[1])
            else:
                # nothing within the bound: both say so
                assert dist_b[o][int(pick_b[o, 0])] > stop


# ------------------------------------------- every candidate, Table 4 caches
def _canonical(cands, members):
    """Canonical member of a set of candidate indices, in the order the C
    header states: LRU < FIFO < RANDOM (< WEIGHTED), larger b, fewer ways,
    smaller C, lower index."""
    return min(members, key=lambda g: (cands[g].policy, -cands[g].b, cands[g].ways, cands[g].C, g))


def _plan_tensors(pts):
    traces, keep = [], []
    for r, tr in pts:
        if tr is None:
            traces.append((None, r.length, r.warmup, r.n_elems, r.stride))
        else:
            t = torch.from_numpy(np.ascontiguousarray(tr, dtype=np.uint32).view(np.int32)).cuda()
            keep.append(t)
            traces.append((t, r.length, r.warmup, r.n_elems, 1))
    return traces, keep


def _outcome_rows(plan, n_cand, lens):
    """Per candidate, its miss bits over all plan traces back to back (host
    uint8), from one simulation of the candidates x traces plan."""
    bits, _ = plan.run()
    torch.cuda.synchronize()
    b = bits.cpu().numpy().view(np.uint32)
    rows = []
    k = 0
    for g in range(n_cand):
        row = []
        for n in lens:
            w0 = int(plan.word_offsets[k])
            row.append(api.unpack_bits(b[w0:w0 + (n + 31) // 32], n))
            k += 1
        rows.append(np.concatenate(row))
    return rows


def test_round_trip_every_matcher_candidate_is_the_truth():
    """Every candidate of the matcher (the whole grid under LRU, FIFO and
    RANDOM plus the Table 4 additions: 1321 geometries) is the truth in
    turn, on the one-geometry configuration's plan (97 stride-128 B arrays
    around 16 KB plus an s = 4 B sweep), through infer_geometry_batch with
    distance bound 0.  Noise-free latencies (100 cycles for a hit, 400 for a
    miss) of the truth's own outcome: the pick is the canonical member of the
    truth's identical-outcome class on the plan, and the number of
    candidates at distance 0 is that class's size."""
    from paper_1509_02308_gb300.api import SimPlan, infer_batch
    cands = W.matcher_candidates()
    _, runs = W.config1()
    C0 = 16384
    for nb in (C0 - 4, C0, C0 + 4, C0 + 32, C0 + 36, C0 + 64, C0 + 68, C0 + 128, C0 + 132,
               C0 + 256, C0 + 260):
        n = nb // 4
        runs.append(W.Run(n, 1, 3 * n, n))
    traces = [(None, r.length, r.warmup, r.n_elems, r.stride) for r in runs]
    lens = [r.length for r in runs]
    plan = SimPlan(cands, traces)
    rows = _outcome_rows(plan, len(cands), lens)
    # a sample of the rows against the oracle (the simulator's own parity tests
    # cover the rest)
    for g in list(range(0, len(cands), 97)) + [len(cands) - 1]:
        G = cands[g]
        want = np.concatenate([oracle.cache_sim(G.C, G.b, G.ways, G.sets, G.policy,
                                                oracle.pchase_trace(r.n_elems, r.stride, r.length),
                                                seed=G.seed, mapping=G.mapping) for r in runs])
        assert np.array_equal(rows[g], want), g
    keys = [np.packbits(r).tobytes() for r in rows]
    classes = {}
    for g, k in enumerate(keys):
        classes.setdefault(k, []).append(g)
    assert len(classes) > 100
    step = 512  # observations per call: 512 x 108 plan traces < 65536
    for o0 in range(0, len(cands), step):
        truths = list(range(o0, min(len(cands), o0 + step)))
        lat = torch.from_numpy(np.stack([(100.0 + 300.0 * rows[t]).astype(np.float32)
                                         for t in truths])).cuda()
        st = api.status_word()
        dist, pick = infer_batch(plan, lat, stop_above=0, status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        dist, pick = dist.cpu().numpy(), pick.cpu().numpy()
        for k, t in enumerate(truths):
            cls = classes[keys[t]]
            assert dist[k, t] == 0
            assert int(pick[k, 0]) == _canonical(cands, cls), (t, int(pick[k, 0]), cls)
            assert int(pick[k, 1]) == len(cls), (t, int(pick[k, 1]), cls)
        del lat


def test_table4_geometries_recovered_by_the_two_stage_procedure():
    """Table 4's caches (Secs. 4.3-4.5) recovered on the GPU from their own
    noise-free outcomes: stage 1 of Fig. 6 (s = 1 element over every
    candidate capacity, simulated for the truth) finds C; stage 2 runs
    infer_geometry over every matcher candidate (1321) on the two-stage plan
    for that C; the truth is the only candidate at distance 0 and the pick.
    Truths: the 12 KB and 24 KB texture L1 caches (32 B lines, 4 sets,
    address bits 7-8, LRU) and the Fermi L1 data cache (16 KB, 128 B lines,
    32 sets, the weighted non-LRU policy)."""
    from paper_1509_02308_gb300.api import SimPlan
    cands = W.matcher_candidates()
    truths = [g for g in W.table4_candidates() if g.policy == W.LRU and g.mapping == 2]
    truths.append([g for g in W.table4_candidates() if g.policy == W.WEIGHTED][0])
    caps, sweep = W.capacity_sweep()
    s_traces = [(None, r.length, r.warmup, r.n_elems, r.stride) for r in sweep]
    for truth in truths:
        _, counts, _ = api.cache_sim_batch([truth], s_traces, [(0, i) for i in range(len(sweep))])
        steady = counts[:, 1].cpu().numpy()
        C_est = max(c for c, m in zip(caps, steady) if m == 0)
        assert C_est == truth.C
        pts = W.two_stage_plan(C_est)
        traces, keep = _plan_tensors(pts)
        tb, _, toffs = api.cache_sim_batch([truth], traces, [(0, i) for i in range(len(pts))])
        tbw = tb.cpu().numpy().view(np.uint32)
        miss = np.concatenate([api.unpack_bits(tbw[int(toffs[i]):], r.length)
                               for i, (r, _) in enumerate(pts)])
        plan = SimPlan(cands, traces)
        lat = torch.from_numpy((100.0 + 300.0 * miss).astype(np.float32)).cuda()
        st = api.status_word()
        dist, pick = plan.infer(lat, status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        dist = dist.cpu().numpy()
        ti = cands.index(truth)
        assert np.nonzero(dist == 0)[0].tolist() == [ti], [cands[i] for i in np.nonzero(dist == 0)[0]]
        assert int(pick[0]) == ti and int(pick[1]) == 1
