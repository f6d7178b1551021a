"""pchase_classify_noalloc: the classifier for callers that cannot allocate
device memory (for instance a loop that classifies probe latencies between
probe runs, where an allocation would synchronise the device and disturb the
timings being taken).  Its scratch is a fixed array inside the library shared
by every call, so this checks it against the workspace form, pchase_classify,
on two different calls in a row: the second must not see the first's data."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1509_02308_gb300 import capi as C  # noqa: E402


def _inputs(seed, sizes):
    rng = np.random.Generator(np.random.PCG64(seed))
    lats = []
    for n in sizes:
        miss = rng.random(n) < rng.uniform(0.1, 0.6)
        lat = np.where(miss, 380.0, 110.0) * (1 + 0.03 * rng.standard_normal(n))
        spikes = rng.random(n) < 0.004
        lat[spikes] *= rng.uniform(2, 8, size=int(spikes.sum()))
        lats.append(lat.astype(np.float32))
    return lats


def _device_layout(lats):
    n = [x.size for x in lats]
    offs = np.zeros(len(n) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(n)
    words = np.zeros(len(n), dtype=np.int64)
    words[1:] = np.cumsum([(k + 31) // 32 for k in n])[:-1]
    flat = torch.from_numpy(np.concatenate(lats)).cuda()
    return (flat, torch.from_numpy(offs).cuda(), torch.from_numpy(words).cuda(), max(n),
            int(sum((k + 31) // 32 for k in n)))


def _classify(lats, noalloc: bool):
    L = C.load()
    flat, offs, words, max_len, nwords = _device_layout(lats)
    bits = torch.full((nwords,), -1, dtype=torch.int32, device="cuda")
    thr = torch.full((len(lats),), -1.0, dtype=torch.float32, device="cuda")
    if noalloc:
        rc = L.pchase_classify_noalloc(flat.data_ptr(), offs.data_ptr(), len(lats), max_len,
                                       bits.data_ptr(), words.data_ptr(), thr.data_ptr(), None)
    else:
        ws = torch.empty(int(L.pchase_classify_workspace_bytes(len(lats), max_len)) + 256,
                         dtype=torch.uint8, device="cuda")
        rc = L.pchase_classify(flat.data_ptr(), offs.data_ptr(), len(lats), max_len,
                               bits.data_ptr(), words.data_ptr(), thr.data_ptr(),
                               (ws.data_ptr() + 255) & ~255, None)
    C.check(rc)
    torch.cuda.synchronize()
    return bits.cpu().numpy(), thr.cpu().numpy()


def test_noalloc_matches_workspace_classifier_twice():
    first = _inputs(1, [5000, 17, 1, 4096, 32, 33, 20000])
    second = _inputs(2, [300, 12000, 7, 999])
    a1 = _classify(first, noalloc=True)
    a2 = _classify(second, noalloc=True)
    b1 = _classify(first, noalloc=False)
    b2 = _classify(second, noalloc=False)
    for (bits_n, thr_n), (bits_w, thr_w) in ((a1, b1), (a2, b2)):
        assert np.array_equal(bits_n, bits_w)
        assert np.array_equal(thr_n.view(np.uint32), thr_w.view(np.uint32))


def test_noalloc_rejects_requests_beyond_its_scratch():
    """The largest request the scratch holds is accepted and agrees with the
    workspace form; one latency more per observation is refused before
    anything is queued.  Both calls get real, consistent device buffers, so a
    regression of the size check shows up as a wrong return code."""
    L = C.load()
    limit = int(L.pchase_classify_noalloc_limit_bytes())
    assert limit == 8 << 20
    # one observation: 256 B of metadata + 16 B per latency of max_len
    fit = (limit - 256) // 16
    assert 256 + 16 * fit == limit
    lat = _inputs(3, [fit])[0]
    got = _classify([lat], noalloc=True)
    want = _classify([lat], noalloc=False)
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[1].view(np.uint32), want[1].view(np.uint32))
    # one more latency does not fit
    flat, offs, words, max_len, nwords = _device_layout(_inputs(4, [fit + 1]))
    bits = torch.zeros(nwords, dtype=torch.int32, device="cuda")
    thr = torch.zeros(1, dtype=torch.float32, device="cuda")
    rc = L.pchase_classify_noalloc(flat.data_ptr(), offs.data_ptr(), 1, max_len, bits.data_ptr(),
                                   words.data_ptr(), thr.data_ptr(), None)
    assert rc == C.ERANGE
    assert b"static scratch" in L.pchase_last_error_string()
    torch.cuda.synchronize()
    assert int(bits.abs().sum()) == 0 and float(thr[0]) == 0.0


def test_noalloc_refuses_an_observation_longer_than_max_len():
    """An observation longer than the max_len the caller passed gets a NaN cut
    and all-0 bits, and writes nothing outside its slice of the shared scratch:
    the call right after it still agrees with the workspace form."""
    L = C.load()
    lats = _inputs(5, [700, 2500])
    flat, offs, words, _, nwords = _device_layout(lats)
    bits = torch.full((nwords,), -1, dtype=torch.int32, device="cuda")
    thr = torch.zeros(2, dtype=torch.float32, device="cuda")
    C.check(L.pchase_classify_noalloc(flat.data_ptr(), offs.data_ptr(), 2, 1000, bits.data_ptr(),
                                      words.data_ptr(), thr.data_ptr(), None))
    torch.cuda.synchronize()
    b = bits.cpu().numpy()
    t = thr.cpu().numpy()
    w1 = int(words[1])
    assert np.isnan(t[1]) and not b[w1:].any()
    short = _classify(lats[:1], noalloc=False)
    assert np.array_equal(b[:w1], short[0]) and t[0] == short[1][0]
    nxt = _inputs(6, [1000, 64])
    assert all(np.array_equal(x, y) for x, y in zip(_classify(nxt, noalloc=True),
                                                   _classify(nxt, noalloc=False)))
