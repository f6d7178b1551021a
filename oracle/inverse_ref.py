"""CPU oracle for the learned inverse and its least-squares judge.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): imported by
tests and the bench's CPU baseline, never by the product library.  Plain
numpy, written from the definitions:

* the network: 1-D convolution (kernel 5, stride 2, zero padding 2) as the
  textbook cross-correlation sum, GELU in its tanh form (Hendrycks & Gimpel
  2016), dense layers, softmax cross-entropy;
* the mean-latency model of Sec. 4.1, t = t0 + t_m r, with the jitter and
  spike recipe of the synthetic traces, drawn from SplitMix64 (Steele, Lea &
  Flood 2014) keyed exactly as the device draws them;
* least squares y ~ alpha + beta r over the kept points of a trace.
"""
from __future__ import annotations

import numpy as np

POINTS = 512
CH = 64
K = 5
HIDDEN = 256
LOGITS = 31
HEADS = (0, 17, 21, 28, 31)
M64 = (1 << 64) - 1


def layer_shapes():
    """(weight rows, weight cols) per layer in parameter order."""
    sh = []
    cin = 1
    for _ in range(4):
        sh.append((CH, K * cin))
        cin = CH
    sh.append((HIDDEN, 32 * CH))
    sh.append((LOGITS, HIDDEN))
    return sh


def unpack(w: np.ndarray):
    """Flat FP32 weights -> [(W, b)] in layer order."""
    out, o = [], 0
    for r, c in layer_shapes():
        W = w[o:o + r * c].reshape(r, c)
        o += r * c
        b = w[o:o + r]
        o += r
        out.append((W, b))
    assert o == w.size
    return out


def bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (nearest, ties to even), returned as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(0.7978845608028654 * (x + 0.044715 * x ** 3)))


def conv1d_s2(x, W, b):
    """x [B, L, Cin] -> [B, L/2, Cout]; out[lo] = b + sum_kk W[:, kk*Cin:(kk+1)*Cin] . x[2 lo + kk - 2]."""
    B, L, cin = x.shape
    lo_n = L // 2
    out = np.zeros((B, lo_n, W.shape[0]), dtype=np.float64)
    for kk in range(K):
        Wk = W[:, kk * cin:(kk + 1) * cin].astype(np.float64)  # [Cout, Cin]
        for lo in range(lo_n):
            li = 2 * lo + kk - 2
            if 0 <= li < L:
                out[:, lo, :] += x[:, li, :].astype(np.float64) @ Wk.T
    return out + b.astype(np.float64)


def forward(w: np.ndarray, x: np.ndarray, round_bf16: bool = True) -> np.ndarray:
    """Logits [B, 31].  With round_bf16 the operands of every product are
    rounded to bfloat16 where the device rounds them (inputs, weights and the
    activations fed to the next layer); sums are float64."""
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float32))
    layers = unpack(np.asarray(w, dtype=np.float32))
    h = r(x.astype(np.float32)).reshape(x.shape[0], POINTS, 1)
    for l in range(4):
        W, b = layers[l]
        h = r(gelu(conv1d_s2(h, r(W), b)).astype(np.float32))
    f = h.reshape(x.shape[0], -1).astype(np.float64)
    W, b = layers[4]
    z = f @ r(W).astype(np.float64).T + b
    h4 = r(gelu(z).astype(np.float32)).astype(np.float64)
    W, b = layers[5]
    return h4 @ r(W).astype(np.float64).T + b


def xent(logits: np.ndarray, labels: np.ndarray) -> float:
    """Mean over batch and the four heads of softmax cross-entropy."""
    tot = 0.0
    for h in range(4):
        z = logits[:, HEADS[h]:HEADS[h + 1]]
        m = z.max(axis=1, keepdims=True)
        lse = np.log(np.exp(z - m).sum(axis=1)) + m[:, 0]
        tot += (lse - z[np.arange(z.shape[0]), labels[:, h]]).sum()
    return tot / (4 * logits.shape[0])


def predict(logits: np.ndarray):
    pred = np.zeros((logits.shape[0], 4), dtype=np.int64)
    conf = np.ones(logits.shape[0])
    for h in range(4):
        z = logits[:, HEADS[h]:HEADS[h + 1]]
        pred[:, h] = z.argmax(axis=1)
        p = np.exp(z - z.max(axis=1, keepdims=True))
        conf *= 1.0 / p.sum(axis=1)
    return pred, conf


# ------------------------------------------------------------------ judge
KEEP = POINTS - 5


def lsq_residuals(rates: np.ndarray, y: np.ndarray) -> np.ndarray:
    """[n, G] residual of the best y ~ alpha + beta r_g fit (beta > 0) over the
    points of y at or below its KEEP-th smallest value; the plain variance of
    y when the slope would not be positive."""
    y = np.asarray(y, dtype=np.float64)
    R = np.asarray(rates, dtype=np.float64)
    out = np.zeros((y.shape[0], R.shape[0]))
    for i in range(y.shape[0]):
        thr = np.sort(y[i])[KEEP - 1]
        m = y[i] <= thr
        yy = y[i][m]
        n = m.sum()
        var_y = (yy * yy).sum() - yy.sum() ** 2 / n
        Rm = R[:, m]
        sr = Rm.sum(axis=1)
        cov = Rm @ yy - yy.sum() * sr / n
        var_r = (Rm * Rm).sum(axis=1) - sr * sr / n
        ok = (var_r > 1e-12) & (cov > 0)
        res = np.where(ok, var_y - np.where(ok, cov * cov / np.where(ok, var_r, 1.0), 0.0), var_y)
        out[i] = np.maximum(res, 0.0)
    return out


# ---------------------------------------------------------------- synthesis
def splitmix64(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def unit(h: int) -> float:
    return float(h >> 40) / 16777216.0


def synth_one(rates: np.ndarray, n_geoms: int, seed: int, number: int, noise: dict):
    """One synthetic trace: (geometry index, normalised float64 trace)."""
    base = splitmix64(seed ^ ((number * 0xD1B54A32D192ED03) & M64))
    g = ((splitmix64(base ^ 1) >> 32) * n_geoms) >> 32
    t0 = noise["t0_lo"] + (noise["t0_hi"] - noise["t0_lo"]) * unit(splitmix64(base ^ 2))
    lr_lo, lr_hi = np.log(noise["rho_lo"]), np.log(noise["rho_hi"])
    rho = np.exp(lr_lo + (lr_hi - lr_lo) * unit(splitmix64(base ^ 3)))
    tm = t0 * (rho - 1.0)
    y = np.zeros(POINTS)
    for p in range(POINTS):
        hp = splitmix64(base ^ ((p + 16) << 20))
        u1 = max(unit(splitmix64(hp ^ 1)), 1e-7)
        u2 = unit(splitmix64(hp ^ 2))
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        v = (t0 + tm * rates[g, p]) * (1.0 + noise["sigma"] * z)
        if unit(splitmix64(hp ^ 3)) < noise["spike_p"]:
            v *= noise["spike_lo"] + (noise["spike_hi"] - noise["spike_lo"]) * unit(splitmix64(hp ^ 4))
        y[p] = v
    mn, mx = y.min(), y.max()
    return int(g), (y - mn) / (mx - mn) if mx > mn else np.zeros(POINTS)
