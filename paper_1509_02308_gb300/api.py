"""Python-facing helpers over the C ABI: allocate torch outputs, marshal
descriptors, call the library.  No computation happens here."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import capi as C
from .workloads import Geom, Run

DEV = "cuda"


def _u32(n, device=DEV):
    return torch.empty(int(n), dtype=torch.int32, device=device)


def status_word(device=DEV) -> torch.Tensor:
    return torch.zeros(1, dtype=torch.int32, device=device)


# --------------------------------------------------------------------- S1
def pchase_build(n_elems: int, stride: int, length: int, next_chain: torch.Tensor | None = None,
                 with_array: bool = False, status: torch.Tensor | None = None, stream=None):
    """Trace of `length` accesses of the chain from j = 0 (int32 tensor, uint32
    bit patterns), and optionally the uniform Listing-1 array."""
    L = C.load()
    trace = _u32(length)
    arr = _u32(n_elems) if with_array else None
    if next_chain is not None and status is None:
        status = status_word()
    C.check(L.pchase_build(n_elems, stride, C.ptr(next_chain), length, C.ptr(trace), C.ptr(arr),
                           C.ptr(status), C.stream_handle(stream)))
    return (trace, arr) if with_array else trace


def pchase_build_batch(runs: list[Run], stream=None):
    """All uniform runs' traces back to back: (flat int32 tensor, offsets)."""
    L = C.load()
    offs = np.zeros(len(runs) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([r.length for r in runs])
    out = _u32(max(1, int(offs[-1])))
    descs = C.trace_array((None, r.length, r.warmup, r.n_elems, r.stride) for r in runs)
    o = C.u64_array(offs[:-1])
    C.check(L.pchase_build_batch(ctypes.addressof(descs), len(runs), C.ptr(out),
                                 o.ctypes.data, C.stream_handle(stream)))
    return out, offs


# --------------------------------------------------------- S2, S3, S5, S6
class SimPlan:
    """A planned batch: create once, upload once, run many times.

    traces: list of (idx tensor or None, length, warmup, n_elems, stride);
    idx tensors are kept alive by the plan."""

    def __init__(self, geoms: list[Geom], traces, pairs=None, tune: dict | None = None,
                 stream=None):
        self.L = C.load()
        self.geoms = list(geoms)
        self.traces = list(traces)
        self._keep = [t[0] for t in self.traces]
        self.cross = pairs is None
        ga = C.geom_array(self.geoms)
        ta = C.trace_array(self.traces)
        pa = C.pair_array(pairs) if pairs is not None else None
        tn = None
        if tune:
            tn = C.Tune(tune.get("scan_max_ways", 0), tune.get("smem_budget_bytes", 0),
                        tune.get("max_warps_per_cta", 0), tune.get("ctas_per_sm_cap", 0),
                        tune.get("batch_max_sets", 0), tune.get("max_split", 0),
                        tune.get("split_cost_ns", 0), tune.get("filtered", 0),
                        tune.get("pool_warps", 0), tune.get("big_slots", 0),
                        tune.get("kind_affinity", 0), tune.get("head_streams", 0))
        h = ctypes.c_void_p()
        C.check(self.L.pchase_sim_plan_create(
            ctypes.addressof(ga), len(self.geoms), ctypes.addressof(ta), len(self.traces),
            ctypes.addressof(pa) if pa is not None else None,
            len(pairs) if pairs is not None else 0,
            ctypes.addressof(tn) if tn is not None else None, ctypes.byref(h)))
        self.h = h
        self.n_items = int(self.L.pchase_sim_plan_items(h))
        self.bitmap_words = int(self.L.pchase_sim_plan_bitmap_words(h))
        self.ws_bytes = int(self.L.pchase_sim_plan_workspace_bytes(h))
        self.launches = int(self.L.pchase_sim_plan_launches(h))
        buf = ctypes.create_string_buffer(4096)
        self.L.pchase_sim_plan_describe(h, buf, 4096)
        self.description = buf.value.decode()
        self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=DEV)
        self._ws = (C.ptr(self.workspace) + 255) & ~255
        C.check(self.L.pchase_sim_plan_upload(h, self._ws, self.ws_bytes, C.stream_handle(stream)))
        # default bitmap layout: items in the caller's order, back to back
        if self.cross:
            lens = [self.traces[i % len(self.traces)][1] for i in range(self.n_items)]
        else:
            lens = [self.traces[t][1] for (_, t) in pairs]
        w = np.array([(x + 31) // 32 for x in lens], dtype=np.uint64)
        self.word_offsets = np.zeros(self.n_items + 1, dtype=np.uint64)
        self.word_offsets[1:] = np.cumsum(w)
        self.lens = lens

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.L.pchase_sim_plan_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def run(self, bitmaps: torch.Tensor | None = None, counts: torch.Tensor | None = None,
            status: torch.Tensor | None = None, want_bitmaps: bool = True, stream=None):
        if want_bitmaps and bitmaps is None:
            bitmaps = _u32(max(1, self.bitmap_words))
        if counts is None:
            counts = torch.empty(2 * max(1, self.n_items), dtype=torch.int64, device=DEV)
        C.check(self.L.pchase_sim_run(self.h, self._ws, C.ptr(bitmaps) if want_bitmaps else None,
                                      None, C.ptr(counts), C.ptr(status), C.stream_handle(stream)))
        return bitmaps, counts

    def run_filtered(self, filter_bitmaps: torch.Tensor, filter_word_offsets: torch.Tensor,
                     bitmaps: torch.Tensor | None = None, counts: torch.Tensor | None = None,
                     status: torch.Tensor | None = None, stream=None):
        """A lower level of a hierarchy (plan made with tune filtered=1): item
        i sees only the accesses set in filter_bitmaps + filter_word_offsets[i]."""
        if bitmaps is None:
            bitmaps = _u32(max(1, self.bitmap_words))
        if counts is None:
            counts = torch.empty(2 * max(1, self.n_items), dtype=torch.int64, device=DEV)
        C.check(self.L.pchase_sim_run_filtered(self.h, self._ws, C.ptr(filter_bitmaps),
                                               C.ptr(filter_word_offsets), C.ptr(bitmaps), None,
                                               C.ptr(counts), C.ptr(status),
                                               C.stream_handle(stream)))
        return bitmaps, counts

    def run_profiled(self, stream=None):
        """run() that also returns the per-item timeline (int64 [items, 4]:
        start ns, end ns, SM id, warp slot)."""
        bitmaps = _u32(max(1, self.bitmap_words))
        counts = torch.empty(2 * max(1, self.n_items), dtype=torch.int64, device=DEV)
        tl = torch.zeros(4 * max(1, self.n_items), dtype=torch.int64, device=DEV)
        C.check(self.L.pchase_sim_run_profiled(self.h, self._ws, C.ptr(bitmaps), None, C.ptr(counts),
                                               None, C.ptr(tl), C.stream_handle(stream)))
        return bitmaps, counts, tl.view(-1, 4)

    def match(self, observed: torch.Tensor, obs_word_offsets: torch.Tensor,
              stop_above: int = 2**64 - 1, status=None, stream=None) -> torch.Tensor:
        dist = torch.empty(max(1, len(self.geoms)), dtype=torch.int64, device=DEV)
        C.check(self.L.pchase_match_run(self.h, self._ws, C.ptr(observed), C.ptr(obs_word_offsets),
                                        stop_above, C.ptr(dist), C.ptr(status),
                                        C.stream_handle(stream)))
        return dist

    def infer(self, lat: torch.Tensor, stop_above: int = 2**64 - 1, status=None, stream=None):
        scratch_b = int(self.L.pchase_infer_scratch_bytes(self.h))
        if getattr(self, "_scratch", None) is None or self._scratch.numel() < scratch_b + 256:
            self._scratch = torch.empty(scratch_b + 256, dtype=torch.uint8, device=DEV)
        sp = (C.ptr(self._scratch) + 255) & ~255
        dist = torch.empty(max(1, len(self.geoms)), dtype=torch.int64, device=DEV)
        pick = torch.empty(2, dtype=torch.int32, device=DEV)
        C.check(self.L.infer_geometry(self.h, self._ws, C.ptr(lat), sp, stop_above, C.ptr(dist),
                                      C.ptr(pick), C.ptr(status), C.stream_handle(stream)))
        return dist, pick


def infer_batch(plan: "SimPlan", lats: torch.Tensor, stop_above: int = 2**64 - 1, status=None,
                stream=None):
    """Batched inference: lats [n_obs, L] FP32 (each row one observation of
    every plan trace) -> (dist [n_obs, n_candidates], pick [n_obs, 2])."""
    L = plan.L
    n_obs = int(lats.shape[0])
    scratch_b = int(L.pchase_infer_batch_scratch_bytes(plan.h, n_obs))
    scratch = torch.empty(scratch_b + 256, dtype=torch.uint8, device=DEV)
    sp = (C.ptr(scratch) + 255) & ~255
    dist = torch.empty(n_obs, max(1, len(plan.geoms)), dtype=torch.int64, device=DEV)
    pick = torch.empty(n_obs, 2, dtype=torch.int32, device=DEV)
    C.check(L.infer_geometry_batch(plan.h, plan._ws, C.ptr(lats), n_obs, sp, stop_above,
                                   C.ptr(dist), C.ptr(pick), C.ptr(status),
                                   C.stream_handle(stream)))
    return dist, pick


class HierarchyPlan:
    """A cascade of cache (or TLB) levels over the same traces: level 0 sees
    every access, level k only the misses of level k-1 (Sec. 3's L1 -> L2
    path; page-sized lines give Sec. 4.4's L1 -> L2 TLB path).  levels: one
    list of geometries per level, item i of every level pairing geometry
    levels[k][pairs[i][0]] with trace pairs[i][1] (all x all when None)."""

    def __init__(self, levels: list[list[Geom]], traces, pairs=None, tune: dict | None = None):
        self.plans = []
        for k, geoms in enumerate(levels):
            tn = dict(tune or {})
            if k > 0:
                tn["filtered"] = 1
            self.plans.append(SimPlan(geoms, traces, pairs=pairs, tune=tn or None))
        self.word_offsets = self.plans[0].word_offsets
        self._wo = torch.from_numpy(self.word_offsets[:-1].astype(np.int64)).to(DEV)

    def run(self, stream=None):
        """(bitmaps, counts) per level; an access's level is the sum of its bits."""
        out = [self.plans[0].run(stream=stream)]
        for p in self.plans[1:]:
            out.append(p.run_filtered(out[-1][0], self._wo, stream=stream))
        return out


def cache_sim_batch(geoms: list[Geom], traces, pairs=None, stream=None):
    """One-shot simulation: (bitmaps int32 tensor, counts int64 [items, 2],
    word offsets numpy)."""
    L = C.load()
    ga = C.geom_array(geoms)
    ta = C.trace_array(traces)
    pa = C.pair_array(pairs) if pairs is not None else None
    n_items = len(pairs) if pairs is not None else len(geoms) * len(traces)
    lens = ([traces[t][1] for (_, t) in pairs] if pairs is not None
            else [traces[i % len(traces)][1] for i in range(n_items)])
    offs = np.zeros(n_items + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([(x + 31) // 32 for x in lens])
    bitmaps = _u32(max(1, int(offs[-1])))
    counts = torch.empty(2 * max(1, n_items), dtype=torch.int64, device=DEV)
    d_offs = torch.from_numpy(offs[:-1].astype(np.int64)).to(DEV)
    need = ctypes.c_size_t(0)
    args = (ctypes.addressof(ga), len(geoms), ctypes.addressof(ta), len(traces),
            ctypes.addressof(pa) if pa is not None else None, len(pairs) if pairs is not None else 0,
            C.ptr(bitmaps), C.ptr(d_offs), C.ptr(counts), None)
    rc = L.cache_sim_batch(*args, None, ctypes.byref(need), C.stream_handle(stream))
    if rc != C.ERANGE:
        C.check(rc)
    ws = torch.empty(need.value + 256, dtype=torch.uint8, device=DEV)
    wp = (C.ptr(ws) + 255) & ~255
    have = ctypes.c_size_t(need.value)
    C.check(L.cache_sim_batch(*args, wp, ctypes.byref(have), C.stream_handle(stream)))
    torch.cuda.current_stream().synchronize()
    return bitmaps, counts.view(-1, 2)[:n_items], offs


# --------------------------------------------------------------------- S4
def pchase_classify(lats: list[torch.Tensor], stream=None):
    """Per-observation classification: (bits int32, word offsets, thresholds)."""
    L = C.load()
    n = [int(x.numel()) for x in lats]
    offs = np.zeros(len(lats) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(n)
    w = np.zeros(len(lats), dtype=np.int64)
    w[1:] = np.cumsum([(x + 31) // 32 for x in n])[:-1]
    flat = torch.cat([x.float().reshape(-1) for x in lats]) if lats else torch.zeros(1, device=DEV)
    max_len = max(n) if n else 0
    d_offs = torch.from_numpy(offs).to(DEV)
    d_w = torch.from_numpy(w).to(DEV)
    nwords = int(sum((x + 31) // 32 for x in n))
    bits = _u32(max(1, nwords))
    thr = torch.empty(max(1, len(lats)), dtype=torch.float32, device=DEV)
    ws = torch.empty(int(L.pchase_classify_workspace_bytes(len(lats), max_len)) + 256,
                     dtype=torch.uint8, device=DEV)
    wp = (C.ptr(ws) + 255) & ~255
    C.check(L.pchase_classify(C.ptr(flat), C.ptr(d_offs), len(lats), max_len, C.ptr(bits),
                              C.ptr(d_w), C.ptr(thr), wp, C.stream_handle(stream)))
    return bits, w, thr


def pchase_canonical_pick(geoms: list[Geom], dist: torch.Tensor, stream=None):
    L = C.load()
    ga = C.geom_array(geoms)
    dg = torch.frombuffer(bytearray(ga), dtype=torch.uint8).to(DEV)
    pick = torch.empty(2, dtype=torch.int32, device=DEV)
    C.check(L.pchase_canonical_pick(C.ptr(dg), C.ptr(dist), len(geoms), C.ptr(pick),
                                    C.stream_handle(stream)))
    return pick


# --------------------------------------------------------------- probes
def pchase_probe_latency(array: torch.Tensor, n_elems: int, iters: int, warmup: int = 0,
                         start: int = 0, cache_mode: int = 0, stream=None):
    L = C.load()
    lat, idx = _u32(max(1, iters)), _u32(max(1, iters))
    ovh = _u32(2)
    st = status_word()
    C.check(L.pchase_probe_latency(C.ptr(array), n_elems, start, warmup, iters, cache_mode,
                                   C.ptr(lat), C.ptr(idx), C.ptr(ovh), C.ptr(st),
                                   C.stream_handle(stream)))
    return lat, idx, ovh, st


def pchase_probe_smem_bank(max_stride: int = 64, repeats: int = 9, stream=None):
    L = C.load()
    cyc = torch.empty(max_stride, dtype=torch.float32, device=DEV)
    deg = _u32(max_stride)
    C.check(L.pchase_probe_smem_bank(max_stride, repeats, C.ptr(cyc), C.ptr(deg),
                                     C.stream_handle(stream)))
    return cyc, deg


def pchase_probe_smem_throughput(ctas_per_sm: int, threads: int, ilp: int, iters: int = 4096,
                                 stream=None) -> dict:
    """Sec. 6.1's shared-memory copy on every SM: bytes per SM cycle (mean and
    best over SMs that held exactly ctas_per_sm CTAs), and CTAs seen per SM."""
    L = C.load()
    sms = torch.cuda.get_device_properties(DEV).multi_processor_count
    ctas = sms * ctas_per_sm
    t0 = torch.empty(ctas, dtype=torch.int64, device=DEV)
    t1 = torch.empty(ctas, dtype=torch.int64, device=DEV)
    sid = torch.empty(ctas, dtype=torch.int32, device=DEV)
    C.check(L.pchase_probe_smem_throughput(ctas, threads, ilp, iters, C.ptr(t0), C.ptr(t1),
                                           C.ptr(sid), C.stream_handle(stream)))
    torch.cuda.current_stream().synchronize()
    a, b, s = t0.cpu().numpy(), t1.cpu().numpy(), sid.cpu().numpy().astype(np.int64)
    per = []
    count = np.bincount(s, minlength=sms)
    for sm in np.nonzero(count == ctas_per_sm)[0]:
        m = s == sm
        span = int(b[m].max() - a[m].min())
        per.append(8.0 * ilp * threads * iters * int(m.sum()) / max(1, span))
    return {"bytes_per_cycle": float(np.mean(per)) if per else 0.0,
            "bytes_per_cycle_max": float(np.max(per)) if per else 0.0,
            "sms_measured": len(per), "ctas_per_sm_seen": [int(count.min()), int(count.max())]}


def pchase_probe_global_throughput(kind: int, vec_bytes: int, ctas: int, threads: int, ilp: int,
                                   src: torch.Tensor | None, dst: torch.Tensor, nbytes: int,
                                   reps: int = 5, stream=None) -> float:
    L = C.load()
    g = ctypes.c_double(0)
    C.check(L.pchase_probe_global_throughput(kind, vec_bytes, ctas, threads, ilp, C.ptr(src),
                                             C.ptr(dst), nbytes, reps, ctypes.byref(g),
                                             C.stream_handle(stream)))
    return g.value


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    """LSB-first packed uint32 words -> uint8 flags (test helper)."""
    b = np.unpackbits(np.ascontiguousarray(words).view(np.uint8), bitorder="little")
    return b[:n]
