"""CPU oracle for the learned inverse and its least-squares judge.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): imported by
tests and the bench's CPU baseline, never by the product library.  Plain
numpy, written from the definitions:

* the network: 1-D convolution (kernel 5, stride 2, zero padding 2) as the
  textbook cross-correlation sum, GELU in its tanh form (Hendrycks & Gimpel
  2016), dense layers, softmax cross-entropy;
* its training step: the backward pass of every layer by the chain rule
  (convolution, GELU, dense, softmax cross-entropy) and one Adam update
  (Kingma & Ba 2015, Algorithm 1), with bfloat16 rounding at the points where
  the device rounds; every function also takes a smaller network size, so a
  tiny network can be checked by finite differences on every parameter;
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


class Spec:
    """Network size: trace points (a multiple of 16), convolution channels,
    hidden width.  The heads are always 17 + 4 + 7 + 3 logits."""

    def __init__(self, points: int = POINTS, ch: int = CH, hidden: int = HIDDEN):
        assert points % 16 == 0
        self.points, self.ch, self.hidden = points, ch, hidden
        self.flat = (points // 16) * ch


FULL = Spec()


def layer_shapes(spec: Spec = FULL):
    """(weight rows, weight cols) per layer in parameter order."""
    sh = []
    cin = 1
    for _ in range(4):
        sh.append((spec.ch, K * cin))
        cin = spec.ch
    sh.append((spec.hidden, spec.flat))
    sh.append((LOGITS, spec.hidden))
    return sh


def param_count(spec: Spec = FULL) -> int:
    return sum(r * c + r for r, c in layer_shapes(spec))


def unpack(w: np.ndarray, spec: Spec = FULL):
    """Flat FP32 weights -> [(W, b)] in layer order."""
    out, o = [], 0
    for r, c in layer_shapes(spec):
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


def forward(w: np.ndarray, x: np.ndarray, round_bf16: bool = True,
            spec: Spec = FULL) -> np.ndarray:
    """Logits [B, 31].  With round_bf16 the operands of every product are
    rounded to bfloat16 where the device rounds them (inputs, weights and the
    activations fed to the next layer); sums are float64.  Without it the
    whole pass is float64."""
    return forward_cache(w, x, round_bf16, spec)["logits"]


def _rounder(round_bf16: bool):
    if round_bf16:
        return lambda a: bf16(np.asarray(a, dtype=np.float32)).astype(np.float64)
    return lambda a: np.asarray(a, dtype=np.float64)


def forward_cache(w: np.ndarray, x: np.ndarray, round_bf16: bool = True,
                  spec: Spec = FULL) -> dict:
    """The forward pass keeping what the backward pass needs: each layer's
    input (as rounded), pre-activation and output.  The flatten before the
    dense layer is position-major: feature p * ch + c holds channel c of
    position p."""
    r = _rounder(round_bf16)
    wd = np.asarray(w, dtype=np.float32 if round_bf16 else np.float64)
    layers = unpack(wd, spec)
    B = x.shape[0]
    h = r(x).reshape(B, spec.points, 1)
    ins, pres = [], []
    for l in range(4):
        W, b = layers[l]
        ins.append(h)
        z = conv1d_s2(h, r(W), b)
        pres.append(z)
        h = r(gelu(z))
    f = h.reshape(B, -1)
    W, b = layers[4]
    z4 = f @ r(W).T + b
    h4 = r(gelu(z4))
    W, b = layers[5]
    logits = h4 @ r(W).T + b
    return {"ins": ins, "pres": pres, "flat": f, "pre4": z4, "h4": h4, "logits": logits,
            "layers": layers, "spec": spec, "round": round_bf16}


def xent(logits: np.ndarray, labels: np.ndarray) -> float:
    """Mean over batch and the four heads of softmax cross-entropy."""
    tot = 0.0
    for h in range(4):
        z = logits[:, HEADS[h]:HEADS[h + 1]]
        m = z.max(axis=1, keepdims=True)
        lse = np.log(np.exp(z - m).sum(axis=1)) + m[:, 0]
        tot += (lse - z[np.arange(z.shape[0]), labels[:, h]]).sum()
    return tot / (4 * logits.shape[0])


def logit_scale(cache: dict) -> np.ndarray:
    """Per logit, the sum of the magnitudes of the terms it adds (|h4| . |W5|
    + |b5|): the scale of its rounding error when the operands agree up to
    their bfloat16 rounding."""
    r = _rounder(cache["round"])
    W5, b5 = cache["layers"][5]
    return np.abs(cache["h4"]) @ np.abs(r(W5)).T + np.abs(np.asarray(b5, dtype=np.float64))


def gelu_grad(x):
    """Derivative of the tanh form of GELU."""
    k0, k1 = 0.7978845608028654, 0.044715
    t = np.tanh(k0 * (x + k1 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * k0 * (1.0 + 3.0 * k1 * x * x)


def xent_grad(logits: np.ndarray, labels: np.ndarray) -> np.ndarray:
    """d xent / d logits: per head, (softmax - one-hot) / (4 B)."""
    B = logits.shape[0]
    d = np.zeros_like(logits, dtype=np.float64)
    for h in range(4):
        z = np.asarray(logits[:, HEADS[h]:HEADS[h + 1]], dtype=np.float64)
        p = np.exp(z - z.max(axis=1, keepdims=True))
        p /= p.sum(axis=1, keepdims=True)
        p[np.arange(B), labels[:, h]] -= 1.0
        d[:, HEADS[h]:HEADS[h + 1]] = p / (4.0 * B)
    return d


def conv1d_s2_back(dz: np.ndarray, x: np.ndarray, W: np.ndarray):
    """Backward of conv1d_s2 by the chain rule: out[b, lo, co] depends on
    x[b, 2 lo + kk - 2, ci] through W[co, kk * Cin + ci].  Returns (dx, dW,
    db) and the magnitudes |dz|^T |x| of dW's terms."""
    B, L, cin = x.shape
    lo_n = L // 2
    dx = np.zeros((B, L, cin))
    dW = np.zeros(W.shape)
    dWabs = np.zeros(W.shape)
    for kk in range(K):
        Wk = W[:, kk * cin:(kk + 1) * cin]
        for lo in range(lo_n):
            li = 2 * lo + kk - 2
            if 0 <= li < L:
                dW[:, kk * cin:(kk + 1) * cin] += dz[:, lo, :].T @ x[:, li, :]
                dWabs[:, kk * cin:(kk + 1) * cin] += np.abs(dz[:, lo, :]).T @ np.abs(x[:, li, :])
                dx[:, li, :] += dz[:, lo, :] @ Wk
    return dx, dW, dz.sum(axis=(0, 1)), dWabs


def backward(cache: dict, labels: np.ndarray):
    """Gradient of the mean cross-entropy (xent) with respect to every
    parameter, flat in parameter order, and for each gradient element the sum
    of the magnitudes of the terms it adds (the scale of its rounding error).
    With bfloat16 rounding, the backward pass rounds where the device does:
    the upstream gradient entering each weight product (the logits' gradient
    and each GELU output gradient) goes to bfloat16, the weights are the
    bfloat16 copies; sums and bias gradients stay wide."""
    r = _rounder(cache["round"])
    spec, layers = cache["spec"], cache["layers"]
    B = cache["logits"].shape[0]
    grads, mags = [None] * 6, [None] * 6
    dlog = xent_grad(cache["logits"], labels)
    dlb = r(dlog)
    W5, _ = layers[5]
    grads[5] = (dlb.T @ cache["h4"], dlog.sum(axis=0))
    mags[5] = (np.abs(dlb).T @ np.abs(cache["h4"]), np.abs(dlog).sum(axis=0))
    dh = dlb @ r(W5)
    dz = dh * gelu_grad(cache["pre4"])
    dzb = r(dz)
    W4, _ = layers[4]
    grads[4] = (dzb.T @ cache["flat"], dz.sum(axis=0))
    mags[4] = (np.abs(dzb).T @ np.abs(cache["flat"]), np.abs(dz).sum(axis=0))
    dact = (dzb @ r(W4)).reshape(B, spec.points // 16, spec.ch)
    for l in range(3, -1, -1):
        W, _ = layers[l]
        dz = dact * gelu_grad(cache["pres"][l])
        dzb = r(dz)
        dx, dW, _, dWabs = conv1d_s2_back(dzb, cache["ins"][l], r(W))
        grads[l] = (dW, dz.sum(axis=(0, 1)))
        mags[l] = (dWabs, np.abs(dz).sum(axis=(0, 1)))
        dact = dx
    flat = np.concatenate([np.concatenate([g.reshape(-1), b]) for g, b in grads])
    mag = np.concatenate([np.concatenate([g.reshape(-1), b]) for g, b in mags])
    return flat, mag


def adam(w, g, m, v, lr: float, step: int, b1: float = 0.9, b2: float = 0.999,
         eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) with the bias
    corrections of step t = step + 1: returns (w', m', v')."""
    w, g, m, v = (np.asarray(a, dtype=np.float64) for a in (w, g, m, v))
    m2 = b1 * m + (1.0 - b1) * g
    v2 = b2 * v + (1.0 - b2) * g * g
    t = step + 1
    mh = m2 / (1.0 - b1 ** t)
    vh = v2 / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m2, v2


def train_step(w, m, v, x, labels, lr: float, step: int, round_bf16: bool = True,
               spec: Spec = FULL):
    """One training step on a batch: (loss, gradient, gradient term scale,
    w', m', v')."""
    c = forward_cache(w, x, round_bf16, spec)
    g, mag = backward(c, labels)
    w2, m2, v2 = adam(w, g, m, v, lr, step)
    return xent(c["logits"], labels), g, mag, w2, m2, v2


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
