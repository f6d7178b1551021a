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
    want = R.forward(w, x, round_bf16=True)
    got = lg.cpu().numpy()
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 2e-2 * scale + 1e-3, np.abs(got - want).max()
    wp, wc = R.predict(want)
    agree = (pred.cpu().numpy() == wp).mean()
    assert agree > 0.97
    # a batch larger than max_batch runs in chunks
    x2 = rng.random((150, R.POINTS)).astype(np.float32)
    _, _, lg2 = net.infer(torch.from_numpy(x2).cuda(), want_logits=True)
    want2 = R.forward(w, x2[130:], round_bf16=True)
    assert np.abs(lg2.cpu().numpy()[130:] - want2).max() <= 2e-2 * np.abs(want2).max() + 1e-3
    assert net.status() == 0


def test_tensor_core_convolution_matches_oracle_layer_by_layer():
    """The tcgen05 convolution (inference path) against the oracle's
    convolution on the same BF16 operands, for each 64-channel layer shape
    (output positions 128, 64, 32: one, two and four traces per 128-row tile)
    and a batch whose last tile is partial."""
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
    h = R.bf16(x).reshape(37, R.POINTS, 1)
    for l in range(4):
        Wl, bl = layers[l]
        want = R.gelu(R.conv1d_s2(h, R.bf16(Wl), bl))
        got = acts[l].astype(np.float64)
        assert got.shape == want.shape, (l, got.shape, want.shape)
        err = np.abs(got - want)
        # BF16 output rounding (2^-8 relative) plus FP32 accumulation order
        assert (err <= 8e-3 * np.abs(want) + 2e-3).all(), (l, float(err.max()))
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
    want = R.forward(w, x[rows], round_bf16=True)
    scale = np.abs(want).max()
    assert np.abs(got[rows] - want).max() <= 2e-2 * scale + 1e-3, np.abs(got[rows] - want).max()


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


def test_one_step_gradient_signs_match_finite_differences():
    net = INV.LearnedInverse(max_batch=16)
    net.init(seed=3)
    w0 = net.weights().cpu().numpy().copy()
    rng = np.random.Generator(np.random.PCG64(9))
    x = rng.random((16, R.POINTS)).astype(np.float32)
    lab = np.stack([rng.integers(0, 17, 16), rng.integers(0, 4, 16), rng.integers(0, 7, 16),
                    rng.integers(0, 3, 16)], axis=1).astype(np.int32)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    INV._check(net.L.pchase_inverse_train_step(net.h, net._p, net._w,
                                               torch.from_numpy(x).cuda().data_ptr(),
                                               torch.from_numpy(lab).cuda().data_ptr(), 16, 1e-4, 0,
                                               loss.data_ptr(), None))
    torch.cuda.synchronize()
    w1 = net.weights().cpu().numpy()
    step = w1 - w0  # Adam's first step: -lr * sign(g) where |g| >> eps
    assert abs(float(loss.item()) - R.xent(R.forward(w0, x), lab)) < 2e-2
    # finite differences of the oracle's float64 loss on the largest steps of
    # every layer
    offs = np.cumsum([0] + [r * c + r for r, c in R.layer_shapes()])
    agree = total = 0
    for l in range(6):
        seg = np.arange(offs[l], offs[l + 1])
        idx = seg[np.argsort(-np.abs(step[seg]))[:6]]
        for i in idx:
            h = 1e-3 * max(1.0, abs(w0[i]))
            wp, wm = w0.copy(), w0.copy()
            wp[i] += h
            wm[i] -= h
            g = (R.xent(R.forward(wp, x, round_bf16=False), lab) -
                 R.xent(R.forward(wm, x, round_bf16=False), lab)) / (2 * h)
            if abs(g) < 1e-6:
                continue
            total += 1
            agree += np.sign(-step[i]) == np.sign(g)
    assert total >= 20 and agree / total >= 0.9, (agree, total)


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
