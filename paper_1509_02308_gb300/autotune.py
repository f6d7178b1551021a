"""Autotuner for the simulator plan (S6): picks the set-mode thresholds and
the CTA shape by timing the caller's own workload on the device.

Coordinate descent over the knobs of pchase_tune: for each knob in turn every
candidate value is timed (median of `reps` CUDA-event-timed runs of the whole
planned batch, bitmaps and counts written) with the other knobs at their best so far; two sweeps.  The
winner is cached as JSON, keyed by the device name and a signature of the
workload (geometry and trace shapes), so later runs reuse it.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics

import torch

from .api import SimPlan

KNOBS = {
    "batch_max_sets": [0xFFFFFFFF, 2, 4, 8, 16, 32, 64, 1 << 30],
    "scan_max_ways": [4, 8, 16, 32],
    "max_warps_per_cta": [8, 12, 16],
    "smem_budget_bytes": [64 * 1024, 96 * 1024, 128 * 1024, 160 * 1024, 200 * 1024, 220 * 1024],
    "max_split": [1, 8, 32],
}
DEFAULT = {"batch_max_sets": 64, "scan_max_ways": 4, "max_warps_per_cta": 16,
           "smem_budget_bytes": 220 * 1024, "max_split": 32}
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def signature(geoms, traces, pairs) -> str:
    h = hashlib.sha1()
    for g in geoms:
        h.update(f"{g.C},{g.b},{g.ways},{g.sets},{g.policy};".encode())
    for t in traces:
        h.update(f"{t[1]},{t[2]},{t[3]},{t[4]},{t[0] is None};".encode())
    h.update(str(len(pairs) if pairs is not None else -1).encode())
    return h.hexdigest()[:16]


def _time(geoms, traces, pairs, tune, reps):
    plan = SimPlan(geoms, traces, pairs=pairs, tune=tune)
    bitmaps, counts = plan.run()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        plan.run(bitmaps=bitmaps, counts=counts)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def tune(geoms, traces, pairs=None, reps: int = 3, sweeps: int = 2, cache: str | None = CACHE,
         log=None) -> dict:
    """Best pchase_tune settings (dict) for this workload on this device."""
    dev = torch.cuda.get_device_name()
    sig = signature(geoms, traces, pairs)
    key = f"{dev}|{sig}"
    db = {}
    if cache and os.path.exists(cache):
        try:
            with open(cache) as f:
                db = json.load(f)
        except Exception:
            db = {}
        if key in db:
            return dict(db[key]["tune"])
    best = dict(DEFAULT)
    best_ms = _time(geoms, traces, pairs, best, reps)
    trials = [(dict(best), best_ms)]
    for _ in range(sweeps):
        improved = False
        for knob, values in KNOBS.items():
            for v in values:
                if v == best[knob]:
                    continue
                t = dict(best)
                t[knob] = v
                ms = _time(geoms, traces, pairs, t, reps)
                trials.append((t, ms))
                if log:
                    log(f"{knob}={v}: {ms:.2f} ms (best {best_ms:.2f})")
                if ms < best_ms * 0.98:
                    best, best_ms, improved = t, ms, True
        if not improved:
            break
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        db[key] = {"tune": best, "ms": best_ms, "default_ms": trials[0][1], "trials": len(trials)}
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1)
        os.replace(tmp, cache)
    return best
