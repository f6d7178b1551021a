"""Learned inverse (S7) on the GPU against the numpy oracle: forward pass,
synthetic traces, least-squares judge, the simulator's miss-rate table, the
gradient of one training step, and learning with fallback."""
import numpy as np
import pytest

import oracle
from oracle import inverse_ref as R
from paper_1509_02308_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1509_02308_gb300 import inverse as INV


def test_forward_matches_oracle():
    net = INV.LearnedInverse(max_batch=64)
    net.init(seed=11)
    rng = np.random.Generator(np.random.PCG64(5))
    x = rng.random((37, R.POINTS)).astype(np.float32)  # 37: ragged against the 128-row tiles
    pred, conf, lg = net.infer(torch.from_numpy(x).cuda(), want_logits=True)
    assert net.status() == 0  # no tensor-core wait gave up
    w = net.weights().cpu().numpy().copy()
    c = R.forward_cache(w, x, round_bf16=True)
    want = c["logits"]
    got = lg.cpu().numpy()
    # per logit: within one bfloat16 unit (2^-8) of the sum of its terms'
    # magnitudes (the inference GELU's hardware tanh errs by about 2^-11,
    # below the bfloat16 rounding of the activation it feeds)
    S = R.logit_scale(c)
    assert (np.abs(got - want) <= 2.0 ** -8 * S).all(), float((np.abs(got - want) / S).max())
    wp, wc = R.predict(want)
    agree = (pred.cpu().numpy() == wp).mean()
    assert agree > 0.97
    # a batch larger than max_batch runs in chunks
    x2 = rng.random((150, R.POINTS)).astype(np.float32)
    _, _, lg2 = net.infer(torch.from_numpy(x2).cuda(), want_logits=True)
    c2 = R.forward_cache(w, x2[130:], round_bf16=True)
    assert (np.abs(lg2.cpu().numpy()[130:] - c2["logits"]) <= 2.0 ** -8 * R.logit_scale(c2)).all()
    assert net.status() == 0


def test_tensor_core_convolution_matches_oracle_layer_by_layer():
    """The tcgen05 convolutions (inference path) against the oracle's
    convolution on the same BF16 operands: layer 2 (fused with layer 1, one
    trace per 128-row tile) and layer 4 (fused with layer 3, two traces per
    layer-3 tile and four per layer-4 tile), with a batch whose last tiles
    are partial."""
    net = INV.LearnedInverse(max_batch=48)
    net.init(seed=21)
    rng = np.random.Generator(np.random.PCG64(12))
    x = rng.random((37, R.POINTS)).astype(np.float32)
    _, _, lg = net.infer(torch.from_numpy(x).cuda(), want_logits=True)
    assert net.status() == 0
    w = net.weights().cpu().numpy().copy()
    layers = R.unpack(w)
    # replay the network layer by layer on the oracle, comparing the device's
    # activations after every convolution (work buffer views)
    acts = net.activations(37)
    # layers 1 and 2 run fused (layer 1 never leaves the SM), and so do
    # layers 3 and 4: each pair's second layer against the oracle's two layers
    # on the BF16 inputs the kernel read, with the first layer of the pair
    # rounded to BF16 as the kernel rounds it
    h = R.bf16(x).reshape(37, R.POINTS, 1)
    for first in (0, 2):
        Wa, ba = layers[first]
        mid = R.bf16(R.gelu(R.conv1d_s2(h, R.bf16(Wa), ba)).astype(np.float32))
        Wl, bl = layers[first + 1]
        want = R.gelu(R.conv1d_s2(mid, R.bf16(Wl), bl))
        got = acts[first + 1].astype(np.float64)
        assert got.shape == want.shape, (first + 1, got.shape, want.shape)
        err = np.abs(got - want)
        # BF16 output rounding (2^-8 relative) plus FP32 accumulation order,
        # and the odd input of the pair's second layer one BF16 unit apart
        # (the hardware tanh in the first layer's GELU)
        assert (err <= 8e-3 * np.abs(want) + 2e-3).all(), (first + 1, float(err.max()))
        h = R.bf16(got.astype(np.float32))


def test_forward_large_batch_sampled_rows():
    """A 3000-trace batch: every elementwise and GEMM launch of the forward
    pass needs several grid-stride rounds or many tiles; sampled rows, the
    last rows included, against the oracle."""
    net = INV.LearnedInverse(max_batch=4096)
    net.init(seed=13)
    rng = np.random.Generator(np.random.PCG64(14))
    x = rng.random((3000, R.POINTS)).astype(np.float32)
    _, _, lg = net.infer(torch.from_numpy(x).cuda(), want_logits=True)
    assert net.status() == 0
    got = lg.cpu().numpy()
    w = net.weights().cpu().numpy().copy()
    rows = np.concatenate([rng.choice(2990, size=10, replace=False), np.arange(2990, 3000)])
    c = R.forward_cache(w, x[rows], round_bf16=True)
    assert (np.abs(got[rows] - c["logits"]) <= 2.0 ** -8 * R.logit_scale(c)).all()


def test_synth_matches_oracle():
    rng = np.random.Generator(np.random.PCG64(6))
    rates = rng.random((7, R.POINTS)).astype(np.float32)
    targets = rng.integers(0, 3, size=(7, 4)).astype(np.int32)
    x, lab, truth = INV.LearnedInverse.synth(torch.from_numpy(rates).cuda(),
                                             torch.from_numpy(targets).cuda(), 20, seed=99, first=1000)
    x, lab, truth = x.cpu().numpy(), lab.cpu().numpy(), truth.cpu().numpy()
    noise = W.latency_noise_params()
    for i in range(20):
        g, y = R.synth_one(rates.astype(np.float64), 7, 99, 1000 + i, noise)
        assert truth[i] == g
        assert (lab[i] == targets[g]).all()
        assert np.abs(x[i] - y).max() < 2e-4, (i, np.abs(x[i] - y).max())


def test_lsq_matches_oracle():
    rng = np.random.Generator(np.random.PCG64(7))
    G = 40
    rates = (rng.random((G, R.POINTS)) < 0.3).astype(np.float32) * rng.random((G, 1)).astype(np.float32)
    rates[5] = rates[4]  # an exact tie: the lower index must win
    targets = np.zeros((G, 4), dtype=np.int32)
    x, _, truth = INV.LearnedInverse.synth(torch.from_numpy(rates).cuda(),
                                           torch.from_numpy(targets).cuda(), 64, seed=5)
    best, res = INV.lsq_match(torch.from_numpy(rates).cuda(), x)
    best, res = best.cpu().numpy(), res.cpu().numpy()
    want = R.lsq_residuals(rates, x.cpu().numpy())
    for i in range(64):
        m = want[i].min()
        assert want[i, best[i]] <= m + 1e-4 * (1 + m), (i, best[i], want[i].argmin())
        assert abs(res[i] - m) <= 1e-3 * (1 + m)
        assert best[i] != 5


def test_rate_table_matches_oracle():
    cands = INV.candidate_table()
    pick = [cands[i] for i in range(0, len(cands), 97)][:12]
    rates, counts = INV.rate_table(pick)
    pts = W.p512_plan()
    rng = np.random.Generator(np.random.PCG64(8))
    for _ in range(40):
        gi = int(rng.integers(0, len(pick)))
        p = int(rng.integers(0, len(pts)))
        g = pick[gi]
        run, tr = pts[p]
        if run.length > 200000:
            continue
        trace = tr if tr is not None else oracle.pchase_trace(run.n_elems, run.stride, run.length)
        tot, aft = oracle.cache_sim_counts(g.C, g.b, g.ways, g.sets, g.policy, trace, run.warmup,
                                           seed=g.seed)
        assert int(counts[gi, p, 0]) == tot and int(counts[gi, p, 1]) == aft
        assert abs(float(rates[gi, p]) - aft / (run.length - run.warmup)) < 1e-6


# BF16 holds 8 significant bits: one rounding moves a value by at most 2^-8
# of itself.  When the device's and the oracle's operands agree up to one such
# rounding each, a sum of products differs by at most about 2^-7 of the sum of
# the terms' magnitudes (plus FP32 accumulation, far smaller).
BF16_TERM_TOL = 2.0 ** -7


@pytest.mark.parametrize("B,step", [(16, 0), (37, 2), (40, 0), (64, 3), (128, 1)])
def test_train_step_matches_oracle_element_by_element(B, step):
    """One pchase_inverse_train_step against the oracle's training step
    (chain-rule backward of every layer, softmax cross-entropy, Adam) on the
    same weights, moments and batch, with bfloat16 rounding where the device
    rounds: every gradient element within 2^-7 of the sum of its terms'
    magnitudes; the loss within 2^-12; the new moments and weights equal to
    Adam applied to the device's own gradient up to FP32 rounding.  Batches
    of 16-128 traces (none a multiple of the 128-row tiles of the dense
    layers), first and later Adam steps with non-zero moments.  37 traces
    leave partial tiles in the convolutions (the last 128-row tile of layers
    3 and 4 holds 1 of its 2 and 1 of its 4 traces) and a batch that is not a
    multiple of 8 for the batch-contiguous weight-gradient operands."""
    net = INV.LearnedInverse(max_batch=128)
    net.init(seed=31 + B)
    rng = np.random.Generator(np.random.PCG64(B))
    n = net.n_params
    m0 = (rng.standard_normal(n) * 1e-3).astype(np.float32) if step else np.zeros(n, np.float32)
    v0 = (rng.random(n) * 1e-5).astype(np.float32) if step else np.zeros(n, np.float32)
    net.param_array(3).copy_(torch.from_numpy(m0))
    net.param_array(4).copy_(torch.from_numpy(v0))
    w0 = net.weights().cpu().numpy().astype(np.float64)
    x = rng.random((B, R.POINTS)).astype(np.float32)
    lab = np.stack([rng.integers(0, k, B) for k in (17, 4, 7, 3)], axis=1).astype(np.int32)
    dx, dl = torch.from_numpy(x).cuda(), torch.from_numpy(lab).cuda()  # alive until synced
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    lr = 1e-3
    INV._check(net.L.pchase_inverse_train_step(net.h, net._p, net._w, dx.data_ptr(),
                                               dl.data_ptr(), B, lr, step, loss.data_ptr(), None))
    torch.cuda.synchronize()
    assert net.status() == 0
    g = net.param_array(2).cpu().numpy().astype(np.float64)
    w1 = net.weights().cpu().numpy().astype(np.float64)
    m1 = net.param_array(3).cpu().numpy().astype(np.float64)
    v1 = net.param_array(4).cpu().numpy().astype(np.float64)
    loss_r, g_r, mag, *_ = R.train_step(w0, m0, v0, x, lab.astype(np.int64), lr, step)
    assert abs(float(loss.item()) - loss_r) <= 2.0 ** -12 * loss_r
    err = np.abs(g - g_r)
    bad = err > BF16_TERM_TOL * mag + 1e-12
    assert not bad.any(), (int(bad.sum()), int(np.argmax(err / np.maximum(mag, 1e-30))))
    # every layer has real signal, and most elements agree far more closely
    offs = np.cumsum([0] + [r * c + r for r, c in R.layer_shapes()])
    for l in range(6):
        seg = slice(offs[l], offs[l + 1])
        assert np.abs(g_r[seg]).max() > 1e-3
        assert np.median(err[seg] / np.maximum(mag[seg], 1e-30)) < 2.0 ** -11
    # Adam on the device's gradient.  The device holds beta1 = 0.9 and
    # beta2 = 0.999 in FP32, where 1 - beta2 is 1.3e-5 of itself away from
    # 0.001, so the moments agree to 2^-15 of their terms; the weights to a
    # few FP32 units of themselves plus 2^-15 of the update's own magnitude and
    # of the magnitude of the first moment's terms (m can cancel to near 0)
    wa, ma, va = R.adam(w0, g, m0, v0, lr, step)
    m_terms = 0.9 * np.abs(m0) + 0.1 * np.abs(g)
    assert (np.abs(m1 - ma) <= 2.0 ** -15 * m_terms + 1e-30).all()
    assert (np.abs(v1 - va) <= 2.0 ** -15 * (0.999 * v0 + 0.001 * g * g) + 1e-30).all()
    t = step + 1
    scale = lr * (m_terms / (1 - 0.9 ** t)) / (np.sqrt(va / (1 - 0.999 ** t)) + 1e-8)
    bound = 2.0 ** -21 * np.abs(w0) + 2.0 ** -15 * (np.abs(wa - w0) + scale)
    assert (np.abs(w1 - wa) <= bound).all(), float((np.abs(w1 - wa) / bound).max())


def test_learns_and_agrees_with_the_exhaustive_judge():
    cands = INV.candidate_table()
    near = [g for g in cands if g.C in (8192, 12288, 16384) and g.b in (64, 128)]
    rates, _ = INV.rate_table(near)
    rep_of, targets, l2c = INV.classes_from_rates(near, rates)
    t_targets = torch.from_numpy(targets.astype(np.int32)).cuda()
    net = INV.LearnedInverse(max_batch=1024)
    net.init(seed=4)
    hist = net.train(rates, t_targets, steps=800, batch=1024, lr=3e-3, log_every=200)
    assert hist[-1][1] < 0.5 * hist[0][1], hist
    x, lab, truth = INV.LearnedInverse.synth(rates, t_targets, 3000, seed=0x5EED1004)
    cand, nf = net.classify(x, torch.from_numpy(l2c.astype(np.int32)).cuda(), rates, 0.9)
    cand, truth = cand.cpu().numpy(), truth.cpu().numpy()
    best, _ = INV.lsq_match(rates, x)
    judge = rep_of[best.cpu().numpy()]
    agree = (rep_of[cand] == judge).mean()
    acc = (rep_of[cand] == rep_of[truth]).mean()
    acc_judge = (judge == rep_of[truth]).mean()
    assert agree >= 0.97, (agree, acc, acc_judge, int(nf.item()))
    assert acc >= acc_judge - 0.02, (acc, acc_judge)


def _single_linkage(r: np.ndarray, tol: float) -> np.ndarray:
    """Lowest index of each row's single-linkage group (rows within tol at
    every point), by union-find on the host."""
    n = r.shape[0]
    parent = np.arange(n)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for i in range(n):
        for j in np.nonzero(np.abs(r[i + 1:] - r[i]).max(axis=1) <= tol)[0] + i + 1:
            a, b = find(i), find(int(j))
            if a != b:
                parent[max(a, b)] = min(a, b)
    return np.array([find(i) for i in range(n)])


def test_answer_classes_equal_host_single_linkage():
    """pchase_answer_classes against union-find on the host: identical rows
    (tol 0), chains that link only through a middle row, and the 0.01
    tolerance; each row is named by the lowest index of its group."""
    from paper_1509_02308_gb300 import capi as C
    rng = np.random.Generator(np.random.PCG64(8))
    G, P = 700, 512
    base = rng.random((40, P)).astype(np.float32)
    r = base[rng.integers(0, 40, G)].copy()
    # small perturbations: some rows within 0.01 of their base, a few chains
    sel = rng.random(G) < 0.3
    r[sel] += (rng.random((int(sel.sum()), P)) * 0.009).astype(np.float32)
    r[5] = r[4] + np.float32(0.008)
    r[6] = r[5] + np.float32(0.008)  # 6 links to 4 only through 5
    L = C.load()
    for tol in (0.0, 0.01, 0.02):
        dr = torch.from_numpy(r).cuda()
        rep = torch.empty(G, dtype=torch.int32, device="cuda")
        work = torch.empty(int(L.pchase_answer_classes_work_bytes(G)) + 256, dtype=torch.uint8,
                           device="cuda")
        C.check(L.pchase_answer_classes(dr.data_ptr(), G, P, tol, rep.data_ptr(),
                                        (work.data_ptr() + 255) & ~255, None))
        want = _single_linkage(r.astype(np.float64), tol)
        assert np.array_equal(rep.cpu().numpy(), want), tol
    assert want[6] == want[4]


def test_miss_rates_from_counts():
    from paper_1509_02308_gb300 import capi as C
    rng = np.random.Generator(np.random.PCG64(9))
    G, P = 37, 512
    meas = rng.integers(0, 1 << 20, P).astype(np.int64)
    meas[3] = 0
    counts = np.zeros((G, P, 2), dtype=np.int64)
    counts[:, :, 1] = (rng.random((G, P)) * meas).astype(np.int64)
    out = torch.empty(G, P, dtype=torch.float32, device="cuda")
    dc, dm = torch.from_numpy(counts).cuda(), torch.from_numpy(meas).cuda()
    C.check(C.load().pchase_miss_rates(dc.data_ptr(), G, P, dm.data_ptr(), out.data_ptr(), None))
    with np.errstate(divide="ignore", invalid="ignore"):
        want = np.where(meas > 0, counts[:, :, 1] / np.maximum(meas, 1), 0.0).astype(np.float32)
    assert np.array_equal(out.cpu().numpy(), want)


def test_loaded_model_classifies_like_the_caller_owned_one():
    """inverse_load from a HOST weights blob (a checkpoint of the FP32
    weights), then inverse_classify, against pchase_inverse_classify on the
    caller-owned parameters the blob came from: the same candidate for every
    trace, the same confidences and fallback count, over 5000 traces (two
    chunks).  A blob of the wrong size is refused; inverse_free(NULL) is a
    no-op."""
    import ctypes

    from paper_1509_02308_gb300 import capi as C
    L = C.load()
    rng = np.random.Generator(np.random.PCG64(17))
    G = 40
    rates = torch.from_numpy(rng.random((G, R.POINTS)).astype(np.float32)).cuda()
    targets = np.stack([rng.integers(0, k, G) for k in (17, 4, 7, 3)], axis=1).astype(np.int32)
    # every label names some geometry, so threshold 0 never falls back
    l2c = (np.arange(17 * 4 * 7 * 3) % G).astype(np.uint32)
    d_l2c = torch.from_numpy(l2c.view(np.int32)).cuda()
    net = INV.LearnedInverse(max_batch=4096)
    net.init(seed=23)
    x, _, _ = INV.LearnedInverse.synth(rates, torch.from_numpy(targets).cuda(), 5000, seed=3)
    blob = net.weights().cpu().numpy().copy()
    h = ctypes.c_void_p()
    assert L.inverse_load(blob.ctypes.data, blob.nbytes - 4, ctypes.byref(h)) == C.EINVAL
    C.check(L.inverse_load(blob.ctypes.data, blob.nbytes, ctypes.byref(h)))
    try:
        # threshold 0: the network answers wherever its labels name a
        # geometry; 0.5: the untrained network is never that sure, so every
        # trace falls back
        for thr in (0.0, 0.5):
            want_cand, want_nf = net.classify(x, d_l2c, rates, thr)
            cand = torch.empty(5000, dtype=torch.int32, device="cuda")
            conf = torch.empty(5000, dtype=torch.float32, device="cuda")
            nf = torch.zeros(1, dtype=torch.int32, device="cuda")
            C.check(L.inverse_classify(h, x.data_ptr(), 5000, d_l2c.data_ptr(), rates.data_ptr(),
                                       G, thr, cand.data_ptr(), conf.data_ptr(), nf.data_ptr(),
                                       None))
            torch.cuda.synchronize()
            assert np.array_equal(cand.cpu().numpy(), want_cand.cpu().numpy()), thr
            assert int(nf.item()) == int(want_nf.item())
            assert int(nf.item()) == (5000 if thr == 0.5 else 0)
            # the FC + heads kernel adds partial logits atomically, so the
            # order of those FP32 additions (and the last bits) vary by run
            _, wconf, _ = net.infer(x)
            assert np.allclose(conf.cpu().numpy(), wconf.cpu().numpy(), rtol=2.0 ** -14, atol=0)
    finally:
        L.inverse_free(h)
    L.inverse_free(None)


def test_classify_captured_in_a_cuda_graph_equals_eager():
    """The learned classification with its fallback (network chunks, routing,
    least-squares matcher over the low-confidence traces) captured in one
    CUDA graph and replayed twice gives the eager call's answers."""
    rng = np.random.Generator(np.random.PCG64(19))
    G = 30
    rates = torch.from_numpy(rng.random((G, R.POINTS)).astype(np.float32)).cuda()
    l2c = torch.from_numpy((np.arange(17 * 4 * 7 * 3) % G).astype(np.int32)).cuda()
    net = INV.LearnedInverse(max_batch=1024)
    net.init(seed=29)
    targets = torch.from_numpy(rng.integers(0, 3, (G, 4)).astype(np.int32)).cuda()
    x, _, _ = INV.LearnedInverse.synth(rates, targets, 5000, seed=8)
    # a threshold in the widest gap between middle confidences, so that the
    # last bits of the confidences (their FC + heads sums are added
    # atomically) cannot move a trace across it
    _, conf, _ = net.infer(x)
    c = np.sort(conf.cpu().numpy().astype(np.float64))
    k = 1250 + int(np.argmax(np.diff(c[1250:3751])))
    thr = float((c[k] + c[k + 1]) / 2)
    want, wnf = net.classify(x, l2c, rates, thr)
    want, wnf = want.cpu().numpy(), int(wnf.item())
    assert 1000 < wnf < 4000
    net.classify(x[:64], l2c, rates, thr)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        cand, nf = net.classify(x, l2c, rates, thr)
    for _ in range(2):
        cand.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(cand.cpu().numpy(), want) and int(nf.item()) == wnf


def test_inference_handle_with_larger_chunks_shares_trained_weights():
    """An inference-only handle (only pchase_inverse_infer_work_bytes of work)
    with 8192-trace chunks over the parameters of a 1024-chunk training handle
    gives the same predictions and, up to the atomic FC sums' last bits, the
    same confidences, over 20,000 traces."""
    rng = np.random.Generator(np.random.PCG64(21))
    net = INV.LearnedInverse(max_batch=1024)
    net.init(seed=31)
    inf = INV.LearnedInverse(max_batch=8192, share_params=net, infer_only=True)
    assert inf.work.numel() < int(inf.L.pchase_inverse_work_bytes(inf.h)) // 2
    x = torch.from_numpy(rng.random((20000, R.POINTS)).astype(np.float32)).cuda()
    p1, c1, l1 = net.infer(x, want_logits=True)
    p2, c2, l2 = inf.infer(x, want_logits=True)
    assert inf.status() == 0
    l1, l2 = l1.cpu().numpy(), l2.cpu().numpy()
    assert np.allclose(l1, l2, rtol=2.0 ** -14, atol=2.0 ** -14 * np.abs(l1).max())
    same = (p1.cpu().numpy() == p2.cpu().numpy()).all(axis=1).mean()
    assert same > 0.999
    assert np.allclose(c1.cpu().numpy(), c2.cpu().numpy(), rtol=2.0 ** -12, atol=0)
