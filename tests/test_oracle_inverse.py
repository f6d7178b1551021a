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
