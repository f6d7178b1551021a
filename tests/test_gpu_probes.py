"""Probes on the GPU itself.  Hardware has no oracle, so these check
invariants: the predicted bank degree, latency plateaus, index traces that
equal the chain walk, and throughput below the HBM peak."""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1509_02308_gb300 import api


def test_smem_bank_degree_and_latency_shape():
    cyc, deg = api.pchase_probe_smem_bank(64, repeats=9)
    cyc, deg = cyc.cpu().numpy(), deg.cpu().numpy()
    for s in range(1, 65):
        words = [t * s for t in range(32)]
        assert deg[s - 1] == math.gcd(s, 32) == oracle.bank_degree(words)
    assert (cyc > 0).all()
    by_deg = {d: np.median(cyc[deg == d]) for d in (1, 2, 4, 8, 16, 32)}
    # latency grows with the conflict degree (Table 7's trend)
    assert by_deg[32] > by_deg[8] > by_deg[1]
    assert by_deg[2] >= by_deg[1] * 0.95


def test_pchase_probe_index_trace_and_plateaus():
    # small array: every timed access after the preheat is an L1 hit
    n_small = 1024  # 4 KB
    _, arr = api.pchase_build(n_small, 8, 1, with_array=True)
    lat, idx, ovh, st = api.pchase_probe_latency(arr, n_small, iters=512, warmup=256, cache_mode=0)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    i = idx.cpu().numpy().view(np.uint32)
    walk = oracle.pchase_trace(n_small, 8, 256 + 512)[256:]
    assert np.array_equal(i, walk)
    small = np.median(lat.cpu().numpy().view(np.uint32))
    o = ovh.cpu().numpy()
    assert o[0] > 0 and o[1] > 0
    # large array, 4 KB stride, L2-only loads: every access leaves the SM
    n_big = 64 << 20  # 256 MB
    _, arr2 = api.pchase_build(n_big, 1024, 1, with_array=True)
    lat2, idx2, _, st2 = api.pchase_probe_latency(arr2, n_big, iters=2048, warmup=0, cache_mode=1)
    torch.cuda.synchronize()
    assert int(st2.item()) == 0
    big = np.median(lat2.cpu().numpy().view(np.uint32))
    assert big > 2 * small, (small, big)
    assert np.array_equal(idx2.cpu().numpy().view(np.uint32),
                          (np.arange(2048, dtype=np.uint64) * 1024 % n_big).astype(np.uint32))


def test_pchase_probe_bad_chain_sets_status():
    chain = torch.tensor([1, 2, 100, 0], dtype=torch.int32, device="cuda")
    lat, idx, ovh, st = api.pchase_probe_latency(chain, 4, iters=8)
    torch.cuda.synchronize()
    assert int(st.item()) & 2


def test_global_throughput_is_plausible():
    nbytes = 1 << 30
    a = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    res = {}
    for kind in (0, 1, 2):
        res[kind] = api.pchase_probe_global_throughput(kind, 16, sms * 4, 256, 4, a, b, nbytes, reps=5)
        assert 500.0 < res[kind] < 8000.0 * 1.05, (kind, res[kind])
    small = api.pchase_probe_global_throughput(2, 4, 1, 32, 1, a, b, 1 << 20, reps=3)
    assert 0 < small < res[2]


@pytest.mark.parametrize("threads,per_sm,ilp", [(32, 1, 1), (256, 2, 4), (1024, 1, 8), (128, 6, 6)])
def test_smem_throughput_probe_bounded_by_banks(threads, per_sm, ilp):
    """Sec. 6.1's copy: every SM holds the CTAs asked for, and no SM moves more
    than its 32 banks x 4 bytes per cycle."""
    r = api.pchase_probe_smem_throughput(per_sm, threads, ilp, iters=512)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert r["ctas_per_sm_seen"] == [per_sm, per_sm]
    assert r["sms_measured"] == sms
    assert 0.0 < r["bytes_per_cycle"] <= r["bytes_per_cycle_max"] <= 128.0 * 1.02


def test_smem_throughput_probe_rejects_bad_shapes():
    from paper_1509_02308_gb300 import capi as C
    L = C.load()
    buf = torch.empty(16, dtype=torch.int64, device="cuda")
    p = C.ptr(buf)
    assert L.pchase_probe_smem_throughput(4, 100, 1, 10, p, p, p, None) == C.EINVAL  # not x32
    assert L.pchase_probe_smem_throughput(4, 64, 3, 10, p, p, p, None) == C.EINVAL   # ilp 3
    assert L.pchase_probe_smem_throughput(4, 64, 1, 0, p, p, p, None) == C.EINVAL    # no trips


def test_latency_spectrum_chain_walk():
    """Sec. 5.2's non-uniform chain: the probe walks exactly the constructed
    path (no element repeats), and hits inside one line are faster than the
    32 MB jumps that miss every cache."""
    from paper_1509_02308_gb300 import workloads as W
    path, labels, n = W.spectrum_chain()
    assert len(set(path)) == len(path) and max(path) < n
    arr = torch.zeros(n, dtype=torch.int32, device="cuda")
    arr[torch.tensor(path, dtype=torch.int64, device="cuda")] = torch.tensor(
        path[1:] + path[:1], dtype=torch.int32, device="cuda")
    lab = np.array(labels)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for mode in (0, 1):
        flush.fill_(1)  # the chain's lines out of L2 (the scatter and the last walk put them there)
        lat, vis, _, st = api.pchase_probe_latency(arr, n, iters=len(path), start=path[0],
                                                   cache_mode=mode)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert np.array_equal(vis.cpu().numpy().view(np.uint32), np.array(path, dtype=np.uint32))
        l = lat.cpu().numpy().view(np.uint32)
        assert np.median(l[lab == "D_same_line"]) < np.median(l[lab == "A_32MB"])
    del arr, flush
    torch.cuda.empty_cache()


def test_probe_short_names_are_the_same_calls():
    """probe_pchase, probe_smem_bank and probe_global_throughput (the call
    list's names) through the C ABI: the same index trace and bank degrees as
    the pchase_probe_* calls, host results where the call returns one, and
    the same argument checks."""
    import ctypes

    from paper_1509_02308_gb300 import capi as C
    L = C.load()
    n = 4096
    _, arr = api.pchase_build(n, 16, 1, with_array=True)
    outs = []
    for fn in (L.probe_pchase, L.pchase_probe_latency):
        lat = torch.zeros(300, dtype=torch.int32, device="cuda")
        idx = torch.zeros(300, dtype=torch.int32, device="cuda")
        ovh = torch.zeros(2, dtype=torch.int32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        C.check(fn(arr.data_ptr(), n, 0, 256, 300, 0, lat.data_ptr(), idx.data_ptr(),
                   ovh.data_ptr(), st.data_ptr(), None))
        torch.cuda.synchronize()
        assert int(st.item()) == 0 and (lat.cpu().numpy() >= 0).all()
        outs.append(idx.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0].view(np.uint32), oracle.pchase_trace(n, 16, 556)[256:])
    degs = []
    for fn in (L.probe_smem_bank, L.pchase_probe_smem_bank):
        cyc = torch.zeros(64, dtype=torch.float32, device="cuda")
        deg = torch.zeros(64, dtype=torch.int32, device="cuda")
        C.check(fn(64, 3, cyc.data_ptr(), deg.data_ptr(), None))
        degs.append(deg.cpu().numpy())
    assert np.array_equal(degs[0], degs[1])
    a = torch.zeros(64 << 20, dtype=torch.uint8, device="cuda")
    b = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    g = ctypes.c_double(0)
    C.check(L.probe_global_throughput(2, 16, 152 * 4, 256, 4, a.data_ptr(), b.data_ptr(), 64 << 20,
                                      3, ctypes.byref(g), None))
    assert g.value > 0
    assert torch.equal(a, b)  # a copy copies
    assert L.probe_smem_bank(65, 3, cyc.data_ptr(), deg.data_ptr(), None) == C.EINVAL
    assert L.probe_pchase(arr.data_ptr(), n, 0, 0, (1 << 24) + 1, 0, lat.data_ptr(),
                          idx.data_ptr(), ovh.data_ptr(), st.data_ptr(), None) == C.ERANGE
