"""Learned inverse (S7) driver: argument marshalling and the training loop's
sequencing over the C ABI.  Every computation (simulation, synthesis, the
network, the least-squares matcher) runs in the CUDA library."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import capi as C
from . import workloads as W
from .api import SimPlan

DEV = "cuda"
N_LABELS = 17 * 4 * 7 * 3


def _check(rc):
    if rc != C.OK:
        L = C.load()
        raise C.PchaseError(rc, L.pchase_inverse_last_error().decode() or
                            L.pchase_last_error_string().decode())


def canonical_key(g: W.Geom):
    """Identifiability order (policy LRU < FIFO < RANDOM, larger b, fewer ways,
    smaller C) used to pick one representative of geometries a plan cannot
    separate."""
    return (g.policy, -g.b, g.ways, g.C)


def candidate_table(seed_base: int = 0x5EED):
    """Every grid geometry under every policy, in canonical order."""
    cands = [W.Geom(C_, b, a, T, p, seed_base + i)
             for i, (C_, b, a, T) in enumerate(W.geometry_grid()) for p in (0, 1, 2)]
    return sorted(cands, key=canonical_key)


def plan_traces():
    """The 512 plan points as simulator trace descriptors (explicit traces on
    the device for the hot re-touch points)."""
    pts = W.p512_plan()
    traces, keep = _traces_of(pts)
    return pts, traces, keep


def rate_table(cands, tune=None, pts=None):
    """Miss rate after warm-up of every candidate at every plan point
    (FP32 [G, points]), by one simulator plan over candidates x points and
    pchase_miss_rates."""
    if pts is None:
        pts, traces, keep = plan_traces()
    else:
        traces, keep = _traces_of(pts)
    plan = SimPlan(cands, traces, tune=tune)
    _, counts = plan.run(want_bitmaps=False)
    meas = torch.tensor([r.length - r.warmup for r, _ in pts], dtype=torch.int64, device=DEV)
    rates = torch.empty(len(cands), len(pts), dtype=torch.float32, device=DEV)
    _check(C.load().pchase_miss_rates(C.ptr(counts), len(cands), len(pts), C.ptr(meas),
                                      C.ptr(rates), C.stream_handle()))
    torch.cuda.synchronize()
    return rates, counts.view(len(cands), len(pts), 2)


def _traces_of(pts):
    traces, keep = [], []
    for run, tr in pts:
        if tr is None:
            traces.append((None, run.length, run.warmup, run.n_elems, run.stride))
        else:
            t = torch.from_numpy(np.ascontiguousarray(tr, dtype=np.uint32).view(np.int32)).to(DEV)
            keep.append(t)
            traces.append((t, run.length, run.warmup, run.n_elems, 1))
    return traces, keep


# Two geometries whose miss rates differ by at most this much at every plan
# point are one answer class.  0: identical rows, the plan's identifiability
# classes (no observation of the plan separates their members).  The plan's
# hot/stream chains separate LRU from FIFO, so no two distinct rows are within
# 0.01 of each other everywhere and a wider tolerance would merge nothing.
CLASS_TOLERANCE = 0.0


def classes_from_rates(cands, rates: torch.Tensor, tol: float = CLASS_TOLERANCE):
    """Answer classes of the candidates under the plan (pchase_answer_classes:
    single-linkage groups of rate rows within `tol` of each other at every
    point; tol = 0: identical rows).  Returns per candidate its class
    representative (the first member in canonical order), the targets (labels
    of the representative) and the label -> candidate table."""
    L = C.load()
    n = len(cands)
    rep = torch.empty(max(1, n), dtype=torch.int32, device=DEV)
    work = torch.empty(int(L.pchase_answer_classes_work_bytes(n)) + 256, dtype=torch.uint8,
                       device=DEV)
    _check(L.pchase_answer_classes(C.ptr(rates), n, rates.shape[1], float(tol), C.ptr(rep),
                                   (C.ptr(work) + 255) & ~255, C.stream_handle()))
    rep_of = rep[:n].cpu().numpy().astype(np.int64)
    targets = np.array([W.geometry_label(cands[rep_of[i]]) for i in range(n)], dtype=np.uint32)
    l2c = np.full(N_LABELS, 0xFFFFFFFF, dtype=np.uint32)
    for i, g in enumerate(cands):
        c, b, w, p = W.geometry_label(g)
        l2c[((c * 4 + b) * 7 + w) * 3 + p] = rep_of[i]
    return rep_of, targets, l2c


class LearnedInverse:
    def __init__(self, max_batch: int = 4096, share_params: "LearnedInverse | None" = None,
                 infer_only: bool = False):
        """max_batch: the training batch and the inference chunk.  share_params:
        another model whose parameter buffer this one uses (an inference handle
        with larger chunks over trained weights); infer_only: allocate only the
        work buffers inference needs."""
        self.L = C.load()
        h = ctypes.c_void_p()
        _check(self.L.pchase_inverse_create(max_batch, ctypes.byref(h)))
        self.h = h
        self.max_batch = max_batch
        self.n_params = int(self.L.pchase_inverse_param_count(h))
        if share_params is not None:
            self.params = share_params.params
            self._p = share_params._p
        else:
            self.params = torch.empty(int(self.L.pchase_inverse_param_bytes(h)) + 256,
                                      dtype=torch.uint8, device=DEV)
            self._p = (C.ptr(self.params) + 255) & ~255
        wb = (self.L.pchase_inverse_infer_work_bytes(h) if infer_only
              else self.L.pchase_inverse_work_bytes(h))
        self.work = torch.empty(int(wb) + 256, dtype=torch.uint8, device=DEV)
        self._w = (C.ptr(self.work) + 255) & ~255

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.L.pchase_inverse_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def weights(self) -> torch.Tensor:
        """FP32 master weights (a view into the parameter buffer)."""
        return self.param_array(0)

    def param_array(self, which: int) -> torch.Tensor:
        """A view of one parameter array: 0 FP32 weights, 1 BF16 copies, 2 the
        last train step's FP32 gradient, 3 / 4 the Adam moments."""
        off = (self._p - C.ptr(self.params)) + int(self.L.pchase_inverse_param_offset(self.h, which))
        if which == 1:
            return self.params[off:off + 2 * self.n_params].view(torch.bfloat16)
        return self.params[off:off + 4 * self.n_params].view(torch.float32)

    def status(self) -> int:
        """Device status word (PCHASE_DEV_* bits) of the last infer, classify
        or train call; reading it synchronises with the device."""
        off = (self._w - C.ptr(self.work)) + int(self.L.pchase_inverse_status_offset(self.h))
        return int(self.work[off:off + 4].view(torch.int32).item())

    def activations(self, B: int):
        """Host copies of the four convolution outputs of the last forward
        chunk (B traces): float32 [B, positions, 64] per layer."""
        out = []
        for l in range(4):
            off = (self._w - C.ptr(self.work)) + int(
                self.L.pchase_inverse_activation_offset(self.h, l))
            n = B * (W.PLAN_POINTS >> (l + 1)) * 64
            a = self.work[off:off + 2 * n].view(torch.bfloat16).float().cpu().numpy()
            out.append(a.reshape(B, W.PLAN_POINTS >> (l + 1), 64))
        return out

    def init(self, seed: int = 1):
        _check(self.L.pchase_inverse_init(self.h, self._p, seed, C.stream_handle()))

    @staticmethod
    def synth(rates: torch.Tensor, targets: torch.Tensor, n: int, seed: int, first: int = 0,
              noise: dict | None = None):
        L = C.load()
        nz = noise or W.latency_noise_params()
        arr = (ctypes.c_float * 8)(nz["t0_lo"], nz["t0_hi"], nz["rho_lo"], nz["rho_hi"],
                                   nz["sigma"], nz["spike_p"], nz["spike_lo"], nz["spike_hi"])
        x = torch.empty(n, W.PLAN_POINTS, dtype=torch.float32, device=DEV)
        lab = torch.empty(n, 4, dtype=torch.int32, device=DEV)
        truth = torch.empty(max(1, n), dtype=torch.int32, device=DEV)
        _check(L.pchase_inverse_synth(C.ptr(rates), C.ptr(targets), rates.shape[0], seed, first, n,
                                      ctypes.addressof(arr), C.ptr(x), C.ptr(lab), C.ptr(truth),
                                      C.stream_handle()))
        return x, lab, truth[:n]

    def train(self, rates, targets, steps: int, batch: int, lr: float = 2e-3, seed: int = 0x5EED0004,
              log_every: int = 0):
        """Adam with a cosine schedule on freshly synthesised batches."""
        loss = torch.zeros(1, dtype=torch.float32, device=DEV)
        hist = []
        for s in range(steps):
            x, lab, _ = self.synth(rates, targets, batch, seed, first=s * batch)
            lr_s = lr * 0.5 * (1.0 + np.cos(np.pi * s / max(1, steps)))
            loss.zero_()
            _check(self.L.pchase_inverse_train_step(self.h, self._p, self._w, C.ptr(x), C.ptr(lab),
                                                    batch, lr_s, s, C.ptr(loss),
                                                    C.stream_handle()))
            if log_every and (s % log_every == 0 or s == steps - 1):
                hist.append((s, float(loss.item())))
        return hist

    def infer(self, x: torch.Tensor, want_logits: bool = False):
        n = x.shape[0]
        pred = torch.empty(max(1, n), 4, dtype=torch.int32, device=DEV)
        conf = torch.empty(max(1, n), dtype=torch.float32, device=DEV)
        lg = torch.empty(max(1, n), 31, dtype=torch.float32, device=DEV) if want_logits else None
        _check(self.L.pchase_inverse_infer(self.h, self._p, self._w, C.ptr(x), n, C.ptr(pred),
                                           C.ptr(conf), C.ptr(lg), C.stream_handle()))
        return pred[:n], conf[:n], (lg[:n] if lg is not None else None)

    def classify(self, x: torch.Tensor, l2c: torch.Tensor, rates: torch.Tensor,
                 conf_thresh: float = 0.9):
        """Learned answer with least-squares fallback: (candidate index per
        trace, number of fallbacks)."""
        n = x.shape[0]
        pred = torch.empty(max(1, n), 4, dtype=torch.int32, device=DEV)
        conf = torch.empty(max(1, n), dtype=torch.float32, device=DEV)
        cand = torch.empty(max(1, n), dtype=torch.int32, device=DEV)
        fl = torch.empty(max(1, n), dtype=torch.int32, device=DEV)
        nf = torch.zeros(1, dtype=torch.int32, device=DEV)
        rows = torch.empty(max(1, n), W.PLAN_POINTS, dtype=torch.float32, device=DEV)
        idx = torch.empty(max(1, n), dtype=torch.int32, device=DEV)
        lw = torch.empty(int(self.L.pchase_lsq_work_bytes(n)) + 256, dtype=torch.uint8, device=DEV)
        _check(self.L.pchase_inverse_classify(self.h, self._p, self._w, C.ptr(x), n, C.ptr(l2c),
                                              C.ptr(rates), rates.shape[0], conf_thresh,
                                              C.ptr(pred), C.ptr(conf), C.ptr(cand), C.ptr(fl),
                                              C.ptr(nf), C.ptr(rows), C.ptr(idx),
                                              (C.ptr(lw) + 255) & ~255, C.stream_handle()))
        return cand[:n], nf


def lsq_match(rates: torch.Tensor, y: torch.Tensor):
    """Exhaustive least-squares matcher: (best candidate index, residual)."""
    L = C.load()
    n = y.shape[0]
    best = torch.empty(max(1, n), dtype=torch.int32, device=DEV)
    res = torch.empty(max(1, n), dtype=torch.float32, device=DEV)
    lw = torch.empty(int(L.pchase_lsq_work_bytes(n)) + 256, dtype=torch.uint8, device=DEV)
    _check(L.pchase_lsq_match(C.ptr(rates), rates.shape[0], C.ptr(y), n, C.ptr(best), C.ptr(res),
                              (C.ptr(lw) + 255) & ~255, C.stream_handle()))
    return best[:n], res[:n]


def _train_timing(batch: int, steps: int, warmup: int, seed: int):
    """CUDA-event time of `steps` training steps (after `warmup`) on one batch
    of random traces and labels."""
    g = torch.Generator(device=DEV).manual_seed(seed)
    x = torch.rand(batch, W.PLAN_POINTS, device=DEV, generator=g)
    lab = torch.stack([torch.randint(0, k, (batch,), device=DEV, generator=g) for k in (17, 4, 7, 3)],
                      1).to(torch.int32).contiguous()
    net = LearnedInverse(max_batch=batch)
    net.init(seed=seed)
    loss = torch.zeros(1, dtype=torch.float32, device=DEV)

    def step(s):
        _check(net.L.pchase_inverse_train_step(net.h, net._p, net._w, C.ptr(x), C.ptr(lab), batch,
                                               1e-3, s, C.ptr(loss), C.stream_handle()))
    for s in range(warmup):
        step(s)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for s in range(steps):
        step(warmup + s)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / max(1, steps)
    print(f"train step: {ms:.3f} ms per {batch} traces ({batch / ms / 1e3:.2f} M traces/s)")
    _check(net.status())


def _main():
    """Inference timing on random traces with freshly initialised weights:
    ``python -m paper_1509_02308_gb300.inverse --traces N --passes P`` runs P
    passes of the network over N traces in one inference-only handle and
    prints the CUDA-event time of each.  ``--train-steps K`` times K training
    steps of ``--batch`` traces instead (after ``--warmup`` steps)."""
    import argparse

    p = argparse.ArgumentParser()
    p.add_argument("--traces", type=int, default=65536)
    p.add_argument("--passes", type=int, default=3)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--train-steps", type=int, default=0)
    p.add_argument("--batch", type=int, default=4096)
    p.add_argument("--warmup", type=int, default=3)
    a = p.parse_args()
    if a.train_steps:
        _train_timing(a.batch, a.train_steps, a.warmup, a.seed)
        return
    g = torch.Generator(device=DEV).manual_seed(a.seed)
    x = torch.rand(a.traces, W.PLAN_POINTS, device=DEV, generator=g)
    net = LearnedInverse(max_batch=a.traces, infer_only=True)
    net.init(seed=a.seed)
    for i in range(a.passes):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        net.infer(x)
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        print(f"pass {i}: {ms:.3f} ms, {a.traces / ms / 1e3:.2f} M traces/s")
    _check(net.status())


if __name__ == "__main__":
    _main()
