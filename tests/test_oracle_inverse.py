"""Pins for the learned-inverse oracle (oracle/inverse_ref.py): textbook
correlation, the erf form of GELU, numpy's least squares, bfloat16 rounding,
the SplitMix64 stream of the C oracle, and the mean-latency model."""
import math

import numpy as np
import pytest

import oracle
from oracle import inverse_ref as R


def test_conv_is_textbook_cross_correlation():
    rng = np.random.Generator(np.random.PCG64(1))
    x = rng.standard_normal((2, 16, 1)).astype(np.float32)
    W = rng.standard_normal((3, 5)).astype(np.float32)
    b = np.zeros(3, dtype=np.float32)
    out = R.conv1d_s2(x, W, b)
    for bi in range(2):
        xp = np.concatenate([np.zeros(2), x[bi, :, 0], np.zeros(2)])
        for co in range(3):
            full = np.correlate(xp, W[co].astype(np.float64), mode="valid")  # positions 0..15
            assert np.allclose(out[bi, :, co], full[::2][:8])


def test_gelu_tanh_form_tracks_erf_form():
    from scipy.special import erf
    x = np.linspace(-6, 6, 2001)
    exact = 0.5 * x * (1 + erf(x / math.sqrt(2)))
    assert np.max(np.abs(R.gelu(x) - exact)) < 1e-3
    assert R.gelu(np.array([0.0]))[0] == 0.0


def test_gelu_sigmoid_form_equals_the_tanh_form():
    """The training kernels compute GELU as x s with s = 1 / (1 + exp(-2u)) and
    its derivative as s + 2 x s (1 - s) k0 (1 + 3 k1 x^2), (1 - s) = exp(-2u) s,
    u = k0 (x + k1 x^3): the oracle's tanh form and its derivative, since
    1 + tanh(u) = 2 / (1 + exp(-2u)) and 1 - tanh(u)^2 = 4 s (1 - s).  In float64
    the two forms agree to rounding over both tails, and the derivative also
    matches central differences of the oracle's GELU."""
    k0, k1 = 0.7978845608028654, 0.044715
    x = np.concatenate([np.linspace(-12, 12, 4801), [-40.0, -1e-6, 0.0, 1e-6, 40.0]])
    u = k0 * (x + k1 * x ** 3)
    e = np.exp(np.minimum(-2.0 * u, 700.0))
    s = 1.0 / (1.0 + e)
    gelu_sig = x * s
    grad_sig = s + 2.0 * x * s * (e * s) * k0 * (1.0 + 3.0 * k1 * x * x)
    ref, dref = R.gelu(x), R.gelu_grad(x)
    assert np.max(np.abs(gelu_sig - ref) - 1e-14 * np.maximum(np.abs(x), 1.0)) <= 0.0
    assert np.max(np.abs(grad_sig - dref)) < 1e-13
    # in the negative tail 1 + tanh(u) cancels in the tanh form (float64 gives 0
    # from about x = -7), while the sigmoid form keeps its relative accuracy:
    # against 60-digit arithmetic it stays within a few ulp
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    for xv in (-3.0, -5.0, -7.5, -10.0, -20.0):
        uu = k0 * (xv + k1 * xv ** 3)
        want = float(mpmath.mpf(xv) / (1 + mpmath.exp(-2 * mpmath.mpf(uu))))
        got = xv / (1.0 + np.exp(-2.0 * uu))
        assert abs(got - want) <= 1e-14 * abs(want), (xv, got, want)
    h = 1e-5
    fd = (R.gelu(x + h) - R.gelu(x - h)) / (2 * h)
    assert np.max(np.abs(grad_sig - fd)) < 1e-8


def test_lsq_matches_numpy_lstsq():
    rng = np.random.Generator(np.random.PCG64(2))
    G, n = 6, 4
    rates = rng.random((G, R.POINTS))
    y = rng.random((n, R.POINTS))
    y[0] = 0.3 + 0.5 * rates[2] + 0.01 * rng.standard_normal(R.POINTS)
    got = R.lsq_residuals(rates, y)
    for i in range(n):
        thr = np.sort(y[i])[R.KEEP - 1]
        m = y[i] <= thr
        for g in range(G):
            A = np.stack([np.ones(m.sum()), rates[g][m]], axis=1)
            coef, *_ = np.linalg.lstsq(A, y[i][m], rcond=None)
            res = ((A @ coef - y[i][m]) ** 2).sum()
            if coef[1] > 0:
                assert abs(got[i, g] - res) < 1e-9 * max(1.0, res) + 1e-9
            else:
                yy = y[i][m]
                assert abs(got[i, g] - ((yy - yy.mean()) ** 2).sum()) < 1e-9
    assert got[0].argmin() == 2


def test_bf16_rounding():
    v = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 65280.0, 1e-3], dtype=np.float32)
    r = R.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0  # tie to even
    assert r[2] == np.float32(1 + 2 ** -6)  # 1 + 3/256 rounds up to 1 + 4/256
    assert r[3] == -2.5
    assert np.all(r.view(np.uint32) & 0xFFFF == 0)


def test_splitmix_agrees_with_c_oracle():
    for x in (0, 1, 0x5EED, 0xDEADBEEFCAFEBABE):
        assert R.splitmix64(x) == oracle.splitmix64(x)


def test_synth_is_affine_in_the_miss_rate_without_noise():
    rng = np.random.Generator(np.random.PCG64(3))
    rates = rng.random((5, R.POINTS))
    noise = {"t0_lo": 20.0, "t0_hi": 400.0, "rho_lo": 1.1, "rho_hi": 30.0, "sigma": 0.0,
             "spike_p": 0.0, "spike_lo": 2.0, "spike_hi": 10.0}
    for k in range(6):
        g, y = R.synth_one(rates, 5, 77, k, noise)
        assert 0 <= g < 5
        assert abs(y.min()) < 1e-12 and abs(y.max() - 1) < 1e-12
        r = rates[g]
        assert np.allclose(y, (r - r.min()) / (r.max() - r.min()), atol=1e-9)


def test_cross_entropy_of_flat_logits():
    z = np.zeros((3, R.LOGITS))
    lab = np.array([[0, 0, 0, 0], [16, 3, 6, 2], [5, 1, 2, 1]])
    want = (math.log(17) + math.log(4) + math.log(7) + math.log(3)) / 4
    assert abs(R.xent(z, lab) - want) < 1e-12
    pred, conf = R.predict(z)
    assert (pred == 0).all() and np.allclose(conf, 1 / (17 * 4 * 7 * 3))


# ----------------------------------------------------------- training step
TINY = R.Spec(points=32, ch=3, hidden=6)


def _tiny_net(seed, B=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal(R.param_count(TINY)) * 0.7
    x = rng.random((B, TINY.points))
    lab = np.stack([rng.integers(0, n, size=B) for n in (17, 4, 7, 3)], axis=1)
    return w, x, lab


def test_backward_equals_finite_differences_on_every_parameter():
    """The chain-rule gradient of the mean cross-entropy against central
    differences of the float64 loss, on every parameter of a tiny network
    (32 points, 3 channels, hidden 6: all four convolutions, the dense layer,
    the heads and every bias)."""
    for seed in (1, 2):
        w, x, lab = _tiny_net(seed)
        g, mag = R.backward(R.forward_cache(w, x, round_bf16=False, spec=TINY), lab)
        assert g.size == w.size == R.param_count(TINY) and (mag >= np.abs(g) - 1e-15).all()
        h = 1e-6
        fd = np.empty_like(g)
        for i in range(w.size):
            wp, wm = w.copy(), w.copy()
            wp[i] += h
            wm[i] -= h
            fd[i] = (R.xent(R.forward(wp, x, False, TINY), lab) -
                     R.xent(R.forward(wm, x, False, TINY), lab)) / (2 * h)
        err = np.abs(g - fd)
        assert (err <= 1e-7 + 1e-5 * np.abs(fd)).all(), (int(err.argmax()), err.max())
        # every layer's weights and biases carry signal
        o = 0
        for r, c in R.layer_shapes(TINY):
            assert np.abs(g[o:o + r * c]).max() > 1e-4
            o += r * c + r


def test_flatten_is_position_major_by_brute_force():
    """The oracle's forward pass against plain loops over (trace, position,
    channel) that write the dense layer's input feature p * ch + c (the
    layout the C header states), on the tiny network."""
    w, x, _ = _tiny_net(3, B=2)
    layers = R.unpack(w, TINY)
    h = [[[x[b, p]] for p in range(TINY.points)] for b in range(2)]
    cin = 1
    for l in range(4):
        W, bias = layers[l]
        L = len(h[0])
        out = [[[0.0] * TINY.ch for _ in range(L // 2)] for _ in range(2)]
        for b in range(2):
            for lo in range(L // 2):
                for co in range(TINY.ch):
                    acc = bias[co]
                    for kk in range(R.K):
                        li = 2 * lo + kk - 2
                        if 0 <= li < L:
                            for ci in range(cin):
                                acc += W[co, kk * cin + ci] * h[b][li][ci]
                    out[b][lo][co] = R.gelu(np.array(acc))
        h, cin = out, TINY.ch
    W4, b4 = layers[4]
    W5, b5 = layers[5]
    for b in range(2):
        feat = np.zeros(TINY.flat)
        for p in range(len(h[b])):
            for c in range(TINY.ch):
                feat[p * TINY.ch + c] = h[b][p][c]
        hid = R.gelu(W4 @ feat + b4)
        want = W5 @ hid + b5
        got = R.forward(w, x[b:b + 1], round_bf16=False, spec=TINY)[0]
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


def test_adam_closed_forms():
    """Kingma & Ba's bias corrections make the first step, and every step of
    a constant gradient, move each weight by lr * g / (|g| + eps); a zero
    gradient from zero moments moves nothing."""
    rng = np.random.Generator(np.random.PCG64(4))
    w = rng.standard_normal(50)
    g = rng.standard_normal(50) * np.logspace(-6, 2, 50)
    lr = 1e-3
    w1, m1, v1 = R.adam(w, g, np.zeros(50), np.zeros(50), lr, 0)
    assert np.allclose(w - w1, lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
    wt, mt, vt = w, np.zeros(50), np.zeros(50)
    for t in range(6):
        w_prev = wt
        wt, mt, vt = R.adam(wt, g, mt, vt, lr, t)
        assert np.allclose(w_prev - wt, lr * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=0), t
    w0, m0, v0 = R.adam(w, np.zeros(50), np.zeros(50), np.zeros(50), lr, 3)
    assert np.array_equal(w0, w) and not m0.any() and not v0.any()


def test_train_step_with_bfloat16_rounding_tracks_the_exact_step():
    """The rounded step (operands rounded to bfloat16, 8 significant bits,
    where the device rounds them) stays within a few bfloat16 units of the
    exact float64 step, in the norm of the whole gradient, on the tiny
    network; and the step's loss is the oracle's cross-entropy."""
    for seed in (5, 6, 7):
        w, x, lab = _tiny_net(seed)
        z = np.zeros_like(w)
        loss, g, _, w1, m1, v1 = R.train_step(w, z, z, x, lab, 1e-3, 0, round_bf16=True, spec=TINY)
        _, g64, *_ = R.train_step(w, z, z, x, lab, 1e-3, 0, round_bf16=False, spec=TINY)
        assert np.linalg.norm(g - g64) <= 2 ** -5 * np.linalg.norm(g64)
        assert loss == R.xent(R.forward(w, x, True, TINY), lab)
        assert np.allclose((w1, m1, v1), R.adam(w, g, z, z, 1e-3, 0))


def test_predict_two_rows_by_hand():
    """Argmax per head (the first on ties) and confidence = product of the
    heads' top softmax probabilities, worked out by hand."""
    z = np.zeros((2, R.LOGITS))
    z[0, 5] = np.log(3.0)            # capacity head: top 3 / (16 + 3)
    z[0, 17] = np.log(2.0)           # line-size head: top 2 / (3 + 2)
    z[0, 21 + 6] = np.log(4.0)       # ways head: top 4 / (6 + 4)
    #                                  policy head flat: 1 / 3, first index
    z[1, 2] = z[1, 9] = np.log(4.0)  # tie: index 2 wins, 4 / (15 + 8)
    z[1, 20] = 1.0                   # last of the line-size head
    z[1, 21:28] = -5.0               # flat ways head: 1 / 7
    z[1, 29] = 7.0                   # policy head: e^7 / (2 + e^7)
    pred, conf = R.predict(z)
    assert pred.tolist() == [[5, 0, 6, 0], [2, 3, 0, 1]]
    assert abs(conf[0] - (3 / 19) * (2 / 5) * (4 / 10) * (1 / 3)) < 1e-15
    e = math.e
    want1 = (4 / 23) * (e / (3 + e)) * (1 / 7) * (e ** 7 / (2 + e ** 7))
    assert abs(conf[1] - want1) < 1e-15


def test_cross_entropy_head_boundaries():
    """A dominant logit at index 17, the first of the line-size head, makes
    only that head's loss vanish: the heads are 17, 4, 7 and 3 logits in
    that order."""
    z = np.zeros((1, R.LOGITS))
    z[0, 17] = 60.0
    lab = np.zeros((1, 4), dtype=np.int64)
    want = (math.log(17) + 0.0 + math.log(7) + math.log(3)) / 4
    assert abs(R.xent(z, lab) - want) < 1e-12
    g = R.xent_grad(z, lab)
    assert abs(g[0, 17]) < 1e-20 and abs(g[0, 0] - (1 / 17 - 1) / 4) < 1e-12
