"""Autotuner for the simulator plan (S6): picks the set-mode thresholds and
the CTA shape by timing the caller's own workload on the device.

Coordinate descent over the knobs of pchase_tune: for each knob in turn every
candidate value is timed (median of `reps` CUDA-event-timed runs of the whole
planned batch, bitmaps and counts written) with the other knobs at their
best so far; two sweeps.  The winner is cached as JSON, keyed by the device
name and a signature of the workload (geometry and trace shapes), so later
runs reuse it.

``tuned.json`` beside this file ships the knobs the tuner chose on a GB300
for the workloads this package benchmarks (same key).  They are looked up
first, so a benchmark times, and a test replays, one fixed plan rather than
whatever a noisy tuning run picks; ``tune(fresh=True)`` ignores them.
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
    "big_slots": [1, 2, 3],
    "kind_affinity": [1, 0xFFFFFFFF],
}
DEFAULT = {"batch_max_sets": 64, "scan_max_ways": 4, "max_warps_per_cta": 16,
           "smem_budget_bytes": 220 * 1024, "max_split": 32, "big_slots": 1, "kind_affinity": 1}
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def signature(geoms, traces, pairs) -> str:
    h = hashlib.sha1()
    for g in geoms:
        h.update(f"{g.C},{g.b},{g.ways},{g.sets},{g.policy};".encode())
    for t in traces:
        h.update(f"{t[1]},{t[2]},{t[3]},{t[4]},{t[0] is None};".encode())
    h.update(str(len(pairs) if pairs is not None else -1).encode())
    return h.hexdigest()[:16]


def key(geoms, traces, pairs, device: str | None = None) -> str:
    dev = device if device is not None else torch.cuda.get_device_name()
    return f"{dev}|{signature(geoms, traces, pairs)}"


def lookup(geoms, traces, pairs=None, device: str | None = None) -> dict | None:
    """The shipped knobs for this workload on this device, or None."""
    if not os.path.exists(SHIPPED):
        return None
    with open(SHIPPED) as f:
        db = json.load(f)
    e = db.get(key(geoms, traces, pairs, device))
    return dict(e["tune"]) if e else None


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
         log=None, fresh: bool = False) -> dict:
    """Best pchase_tune settings (dict) for this workload on this device:
    the shipped knobs, else the cached ones, else a tuning run (fresh=True:
    always a tuning run, whose result is then cached)."""
    k = key(geoms, traces, pairs)
    if not fresh:
        shipped = lookup(geoms, traces, pairs)
        if shipped is not None:
            return shipped
    db = {}
    if cache and os.path.exists(cache) and not fresh:
        try:
            with open(cache) as f:
                db = json.load(f)
        except Exception:
            db = {}
        if k in db:
            return dict(db[k]["tune"])
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
                    # run-to-run spread is a few percent: a winner must stay
                    # ahead when both are timed again, more times
                    ms = _time(geoms, traces, pairs, t, 2 * reps + 1)
                    again = _time(geoms, traces, pairs, best, 2 * reps + 1)
                    if log:
                        log(f"  confirm {knob}={v}: {ms:.2f} ms vs {again:.2f}")
                    if ms < again * 0.98:
                        best, best_ms, improved = t, ms, True
                    else:
                        best_ms = again
        if not improved:
            break
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        if fresh and os.path.exists(cache):
            try:
                with open(cache) as f:
                    db = json.load(f)
            except Exception:
                db = {}
        db[k] = {"tune": best, "ms": best_ms, "default_ms": trials[0][1], "trials": len(trials)}
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1)
        os.replace(tmp, cache)
    return best


def _main():
    """Tunes the batched-simulation benchmark workload (4096 items) on this
    device and writes its entry into the shipped table (or --out)."""
    import argparse

    from . import api, workloads as W
    p = argparse.ArgumentParser()
    p.add_argument("--out", default=SHIPPED)
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--sweeps", type=int, default=2)
    a = p.parse_args()
    geoms, runs = W.config2()
    flat, offs = api.pchase_build_batch(runs)
    traces = [(flat[int(offs[i]):int(offs[i + 1])], r.length, r.warmup, r.n_elems, r.stride)
              for i, r in enumerate(runs)]
    pairs = [(i, i) for i in range(len(runs))]
    torch.cuda.synchronize()
    log = []
    best = tune(geoms, traces, pairs=pairs, reps=a.reps, sweeps=a.sweeps, cache=None,
                log=log.append, fresh=True)
    # the shipped pick: the tuned knobs only if they stay ahead of the defaults
    # over interleaved re-timings
    tb, td = [], []
    for _ in range(5):
        tb.append(_time(geoms, traces, pairs, best, 3))
        td.append(_time(geoms, traces, pairs, dict(DEFAULT), 3))
    ms_best, ms_default = statistics.median(tb), statistics.median(td)
    if not ms_best < 0.99 * ms_default:
        best, ms_best = dict(DEFAULT), ms_default
    db = {}
    if os.path.exists(a.out):
        with open(a.out) as f:
            db = json.load(f)
    db[key(geoms, traces, pairs)] = {
        "workload": "batched simulation, 4096 items (workloads.config2 defaults)",
        "tune": best, "ms": round(ms_best, 3), "default_ms": round(ms_default, 3),
        "trials": len(log) + 1}
    with open(a.out, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
        f.write("\n")
    print("\n".join(log))
    print(json.dumps(db[key(geoms, traces, pairs)]))


if __name__ == "__main__":
    _main()
