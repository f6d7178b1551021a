"""The C-ABI library loads, exports every symbol include/pchase.h declares,
and validates its host-side arguments.  No GPU work."""
import ctypes
import os
import re

import pytest

from paper_1509_02308_gb300 import capi as C
from paper_1509_02308_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pchase.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_library_exports_every_declared_symbol():
    L = C.load()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(C.SIGNATURES), set(names) ^ set(C.SIGNATURES)


def test_version_string():
    assert b"sm_103a" in C.load().pchase_version()


def _plan(geoms, traces, pairs=None, tune=None):
    L = C.load()
    ga, ta = C.geom_array(geoms), C.trace_array(traces)
    pa = C.pair_array(pairs) if pairs is not None else None
    tn = C.Tune(*[tune.get(f, 0) for f, _ in C.Tune._fields_]) if tune else None
    h = ctypes.c_void_p()
    rc = L.pchase_sim_plan_create(ctypes.addressof(ga), len(geoms), ctypes.addressof(ta),
                                  len(traces), ctypes.addressof(pa) if pa is not None else None,
                                  len(pairs) if pairs else 0,
                                  ctypes.addressof(tn) if tn is not None else None, ctypes.byref(h))
    return rc, h


def _describe(h) -> dict:
    L = C.load()
    buf = ctypes.create_string_buffer(4096)
    L.pchase_sim_plan_describe(h, buf, len(buf))
    return dict(kv.split("=", 1) for kv in buf.value.decode().split())


@pytest.mark.parametrize("geom,code", [
    (W.Geom(1024, 48, 2, 8), C.EINVAL),       # b not a power of two
    (W.Geom(1024, 32, 2, 8), C.EINVAL),       # T*a*b != C
    (W.Geom(1024, 2, 4, 128), C.EINVAL),      # b < 4
    (W.Geom(1024, 32, 0, 32), C.EINVAL),      # no ways
    (W.Geom(1 << 30, 32, 1 << 25, 1), C.ERANGE),  # 2^25 lines
    (W.Geom(1024, 32, 4, 8, 7), C.EINVAL),    # unknown policy
    (W.Geom(1024, 32, 2, 16, 3), C.EINVAL),   # WEIGHTED needs 3 ways
    (W.Geom(1024, 32, 4, 8, 0, mapping=17), C.EINVAL),  # mapping above 16
    (W.Geom(1 << 20, 4, 1, 1 << 18, 0, mapping=13), C.EINVAL),  # T << mapping above 2^30
])
def test_plan_rejects_bad_geometry(geom, code):
    rc, h = _plan([geom], [(None, 10, 0, 100, 1)])
    assert rc == code
    assert C.load().pchase_last_error_string()


def test_plan_accepts_mapping_and_weighted_policy():
    gs = [W.Geom(12288, 32, 96, 4, 0, mapping=2), W.Geom(16384, 128, 4, 32, 3, 5),
          W.Geom(768, 16, 3, 16, 3, 9, mapping=4)]
    rc, h = _plan(gs, [(None, 1000, 0, 3200, 8)])
    assert rc == C.OK
    d = _describe(h)
    assert int(d["items"]) == 3
    C.load().pchase_sim_plan_destroy(h)


def test_plan_splits_items_too_large_for_one_warp():
    # 2 MB, 64 B lines, 16 ways: 32768 lines of set state, more than one
    # warp's shared memory holds; a stream over every set fits once split
    g = W.Geom(2 << 20, 64, 16, 2048, 0)
    tr = [(None, 200000, 0, (4 << 20) // 4, 16)]
    rc, h = _plan([g], tr)
    assert rc == C.OK
    assert int(_describe(h)["units"]) > 1
    C.load().pchase_sim_plan_destroy(h)
    # with splits off it keeps its set state in global memory instead
    rc, h = _plan([g], tr, tune={"max_split": 1})
    assert rc == C.OK and _describe(h)["global_state"] == "1"
    C.load().pchase_sim_plan_destroy(h)


def test_planner_isolates_the_costliest_units():
    # the batched workload, planned on the host: the costliest units (within
    # 40 % of the longest, at most 12) go to the one-warp launch, beside the
    # units whose arenas are too large for the slot mix
    geoms, runs = W.config2()
    traces = [(None, r.length, r.warmup, r.n_elems, r.stride) for r in runs]
    rc, h = _plan(geoms, traces, pairs=[(i, i) for i in range(len(runs))])
    assert rc == C.OK
    d = _describe(h)
    assert int(d["jumbo"]) >= 8
    crit, target, longest, total = (float(x) for x in d["est_ms"].split(","))
    assert longest <= crit * 1.0001 and total > 64 * longest
    C.load().pchase_sim_plan_destroy(h)
    # a plan of few units (no splits) isolates nothing
    rc, h = _plan(geoms[:32], traces[:32], pairs=[(i, i) for i in range(32)],
                  tune={"max_split": 1})
    assert rc == C.OK and int(_describe(h)["jumbo"]) == 0
    C.load().pchase_sim_plan_destroy(h)


def test_plan_rejects_bad_trace_and_pair():
    g = W.Geom(1024, 32, 4, 8)
    rc, _ = _plan([g], [(None, 10, 0, 0, 1)])
    assert rc == C.EINVAL
    rc, _ = _plan([g], [(None, 1 << 31, 0, 10, 1)])
    assert rc == C.ERANGE
    rc, _ = _plan([g], [(None, 10, 0, 10, 1)], pairs=[(0, 1)])
    assert rc == C.EINVAL


def test_plan_sizes_and_layout():
    L = C.load()
    geoms = [W.Geom(16384, 128, 4, 32), W.Geom(12288, 32, 96, 4, W.FIFO)]
    traces = [(None, 100, 10, 4096, 32), (None, 33, 0, 3072, 1), (None, 0, 0, 5, 1)]
    rc, h = _plan(geoms, traces)
    assert rc == C.OK
    try:
        assert L.pchase_sim_plan_items(h) == 6
        assert L.pchase_sim_plan_bitmap_words(h) == 2 * (4 + 2 + 0)
        assert L.pchase_sim_plan_workspace_bytes(h) >= 256 + 6 * 80
    finally:
        L.pchase_sim_plan_destroy(h)


def test_planner_splits_only_what_can_gain():
    """Host-side split rules: a split part owns a power-of-two share of the
    sets the trace actually visits; fully associative caches and traces whose
    stride keeps them in one set do not split by sets (FIFO: they stay whole;
    LRU: they are cut in time instead); splitting is off at max_split 1."""
    L = C.load()
    n = 1 << 16
    traces = [(None, 1 << 20, 0, n, 16),        # 64 B stride: one line per access, all sets
              (None, 1 << 20, 0, n, 64 * 16)]   # 4 KB stride: 64 lines apart
    force = {"max_split": 8, "split_cost_ns": 1}
    for pol in (W.FIFO, W.LRU):
        geoms = [W.Geom(64 * 8 * 64, 64, 8, 64, pol),   # T = 64
                 W.Geom(8 * 64, 64, 8, 1, pol),          # fully associative
                 W.Geom(96 * 2 * 64, 64, 2, 96, pol)]    # T = 3 * 32
        rc, h = _plan(geoms, traces, tune=force)
        assert rc == C.OK
        try:
            d = _describe(h)
            assert int(d["items"]) == 6
            if pol == W.FIFO:
                # T=64: 8 parts with the dense trace; the 4 KB stride visits set 0
                # only (64 lines apart, T = 64), so it stays whole.  Fully
                # associative: whole.  T=96 with the dense trace: up to 8 parts
                # (K must divide the set groups and be 2^j or 3 * 2^j); with the
                # 4 KB stride the visited sets are the multiples of 32, three set
                # groups, so K = 3.  (How many parts the dense items get depends
                # on the cost model.)
                assert int(d["split"]) == 3 and int(d["time_split"]) == 0
                assert 3 + 3 + 2 + 2 <= int(d["units"]) <= 3 + 3 + 8 + 8
            else:
                # the three items that do not split by sets are cut in time
                # (2 .. 8 parts); the others split by sets or in time, whichever
                # the cost model finds cheaper
                assert int(d["split"]) + int(d["time_split"]) == 6
                assert int(d["time_split"]) >= 3
                assert 6 * 2 <= int(d["units"]) <= 6 * 8
        finally:
            L.pchase_sim_plan_destroy(h)
        rc, h = _plan(geoms, traces, tune={"max_split": 1, "split_cost_ns": 1})
        assert rc == C.OK
        try:
            d = _describe(h)
            assert int(d["split"]) == 0 and int(d["time_split"]) == 0 and int(d["units"]) == 6
        finally:
            L.pchase_sim_plan_destroy(h)


def test_set_state_beyond_shared_memory_goes_to_global_memory():
    """Items whose set state fits no shared-memory arena, even split (a fully
    associative 65535-line cache over a 64 Mi-element array; a 128 MB L2 of
    1 Mi lines), become whole way-scan units with the state in global memory,
    counted in the workspace; batched inference refuses such plans."""
    L = C.load()
    geoms = [W.Geom(65535 * 32, 32, 65535, 1), W.Geom(128 << 20, 128, 16, 65536),
             W.Geom(128 << 20, 128, 16, 65536, W.RANDOM, 5), W.Geom(16 << 10, 64, 4, 64)]
    rc, h = _plan(geoms, [(None, 1 << 12, 0, 1 << 26, 1)])
    assert rc == C.OK
    try:
        d = _describe(h)
        assert d["global_state"] == "3" and d["units"] == "4"
        state = 8 * 65535 + 2 * 8 * (1 << 20) + 4 * 65536
        assert L.pchase_sim_plan_workspace_bytes(h) >= state
    finally:
        L.pchase_sim_plan_destroy(h)


def test_one_shot_reports_workspace_need():
    L = C.load()
    ga = C.geom_array([W.Geom(16384, 128, 4, 32)])
    ta = C.trace_array([(None, 100, 10, 4096, 32)])
    need = ctypes.c_size_t(0)
    rc = L.cache_sim_batch(ctypes.addressof(ga), 1, ctypes.addressof(ta), 1, None, 0, None, None,
                           None, None, None, ctypes.byref(need), None)
    assert rc == C.ERANGE and need.value >= 256


def test_probe_argument_checks():
    L = C.load()
    g = ctypes.c_double()
    assert L.pchase_probe_global_throughput(5, 4, 1, 32, 1, 1, 1, 64, 1, ctypes.byref(g), None) == C.EINVAL
    assert L.pchase_probe_global_throughput(0, 8, 1, 32, 1, 1, 1, 64, 1, ctypes.byref(g), None) == C.EINVAL
    assert L.pchase_probe_global_throughput(0, 4, 1, 33, 1, 1, 1, 64, 1, ctypes.byref(g), None) == C.EINVAL
    assert L.pchase_probe_smem_bank(0, 1, 1, 1, None) == C.EINVAL
    assert L.pchase_probe_smem_bank(65, 1, 1, 1, None) == C.EINVAL
    assert L.pchase_probe_latency(1, 0, 0, 0, 1, 0, 1, 1, 1, 1, None) == C.EINVAL
    assert L.pchase_probe_latency(1, 10, 0, 0, (1 << 24) + 1, 0, 1, 1, 1, 1, None) == C.ERANGE
    assert L.pchase_build(0, 1, None, 10, 1, None, None, None) == C.EINVAL


def test_only_lru_items_are_cut_in_time():
    """Time parts rebuild an LRU set's state from its recency order; FIFO and
    RANDOM states depend on past misses, so those items stay whole."""
    L = C.load()
    geoms = [W.Geom(64 * 32, 32, 64, 1, p, 3) for p in (W.LRU, W.FIFO, W.RANDOM, W.WEIGHTED)]
    traces = [(None, 1 << 18, 0, 1 << 12, 8)]  # 32 B stride over 4096 elements: thrashes
    rc, h = _plan(geoms, traces, tune={"max_split": 16, "split_cost_ns": 1})
    assert rc == C.OK
    try:
        d = _describe(h)
        assert int(d["split"]) == 0 and int(d["time_split"]) == 1
        assert 3 + 2 <= int(d["units"]) <= 3 + 16
    finally:
        L.pchase_sim_plan_destroy(h)


def test_unequal_sets_checks():
    """Unequal sets (mapping bits 8-15): C = (T*a + extra) * b, LRU or FIFO,
    plain mapping; such items run as whole way-scan units."""
    L = C.load()
    page = 2 << 20
    tlb = W.Geom(65 * page, page, 8, 7, W.LRU, extra=9)
    rc, h = _plan([tlb, W.Geom(65 * page, page, 8, 7, W.FIFO, extra=9)],
                  [(None, 1 << 16, 0, 80 * page // 4, page // 4)],
                  tune={"max_split": 16, "split_cost_ns": 1})
    assert rc == C.OK
    try:
        d = _describe(h)
        assert d["units"] == "2" and d["scan"] == "2"
        assert d["split"] == "0" and d["time_split"] == "0"
    finally:
        L.pchase_sim_plan_destroy(h)
    for bad in (W.Geom(64 * page, page, 8, 7, W.LRU, extra=9),        # C != (T*a + extra) * b
                W.Geom(65 * page, page, 8, 7, W.RANDOM, extra=9),     # LRU / FIFO only
                W.Geom(65 * page, page, 8, 7, W.LRU, mapping=1, extra=9)):
        rc, _ = _plan([bad], [(None, 10, 0, 100, 1)])
        assert rc == C.EINVAL, bad


def _units_hold_invariants(h, lens):
    """Every item: one lead unit; its units are one whole unit, K set-parts
    with each residue once, or time parts tiling its steps in whole
    1024-access blocks (so each bitmap word has one writer); a unit with
    global-memory set state fits one region of the plan's pool, and the
    pool (warps x region bytes) fits the workspace."""
    L = C.load()
    units = C.plan_units(h)
    by_item = {}
    for u in units:
        by_item.setdefault(u.item, []).append(u)
    assert sorted(by_item) == list(range(len(lens)))
    pool = _describe(h).get("pool")
    region = int(pool.split("x")[1]) if pool else 0
    pool_bytes = int(pool.split("x")[0]) * region if pool else 0
    for item, us in by_item.items():
        nsteps = (lens[item] + 31) // 32
        assert sum(1 for u in us if u.flags & C.UNIT_LEAD) == 1, item
        tparts = [u for u in us if u.flags & C.UNIT_TIME_PART]
        if tparts:
            assert len(tparts) == len(us) >= 2 and all(u.parts == 1 for u in us)
            spans = sorted((u.first_step, u.end_step) for u in us)
            assert spans[0][0] == 0 and spans[-1][1] == nsteps, (item, spans)
            for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
                assert a1 == b0 and a0 < a1 and b0 % 32 == 0, (item, spans)
            assert all(u.mode == 2 and u.flags & C.UNIT_DIRECT for u in us)
        elif us[0].parts > 1:
            K = us[0].parts
            assert len(us) == K and sorted(u.residue for u in us) == list(range(K))
            assert all(u.first_step == 0 and u.end_step == nsteps for u in us)
        else:
            assert len(us) == 1 and us[0].end_step == nsteps
        for u in us:
            if u.flags & C.UNIT_GLOBAL_STATE:
                assert u.parts == 1 and u.mode == 0 and u.state_bytes > 0
                assert u.state_offset == 0 and u.state_bytes <= region and region % 16 == 0
            else:
                assert u.state_bytes == 0
    # the workspace holds the queues, the whole unit table (112 bytes a unit,
    # the pool's units included) and the pool
    assert L.pchase_sim_plan_workspace_bytes(h) >= 512 + 112 * len(units) + pool_bytes
    if pool_bytes:
        assert pool_bytes <= min(L.pchase_sim_plan_workspace_bytes(h), 16 << 30)
        # the pool's units run last in the unit table, after every size class
        gm = [k for k, u in enumerate(units) if u.flags & C.UNIT_GLOBAL_STATE]
        assert gm == list(range(len(units) - len(gm), len(units)))
    return units


def test_plan_units_tile_items_and_state():
    geoms, runs = W.config2()
    lens = [r.length for r in runs]
    traces = [(None, r.length, r.warmup, r.n_elems, r.stride) for r in runs]
    for tune in (None, {"max_split": 16, "split_cost_ns": 1}, {"max_split": 3, "split_cost_ns": 1}):
        rc, h = _plan(geoms, traces, pairs=[(i, i) for i in range(len(runs))], tune=tune)
        assert rc == C.OK
        try:
            units = _units_hold_invariants(h, lens)
            d = _describe(h)
            assert len(units) == int(d["units"])
            leads = [u for u in units if u.flags & C.UNIT_TIME_PART and u.flags & C.UNIT_LEAD]
            assert len(leads) == int(d["time_split"])
        finally:
            C.load().pchase_sim_plan_destroy(h)
    # large caches (global-memory state) and unequal sets beside ordinary items
    MB, page = 1 << 20, 2 << 20
    geoms = [W.Geom(128 * MB, 128, 16, 65536), W.Geom(8 * MB, 32, 16, 16384, W.RANDOM, 3),
             W.Geom(65 * page, page, 8, 7, W.LRU, extra=9), W.Geom(16 << 10, 64, 4, 64)]
    traces = [(None, 100000, 0, (160 * MB) // 4, 32), (None, 5000, 0, (40 * MB) // 4, 8)]
    lens = [t[1] for _ in geoms for t in traces]
    for tune in (None, {"max_split": 1}):
        rc, h = _plan(geoms, traces, tune=tune)
        assert rc == C.OK
        try:
            units = _units_hold_invariants(h, lens)
            assert sum(1 for u in units if u.flags & C.UNIT_GLOBAL_STATE) >= 2
            assert sum(1 for u in units if u.flags & C.UNIT_UNEQUAL) == 2
        finally:
            C.load().pchase_sim_plan_destroy(h)
