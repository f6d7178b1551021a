#!/usr/bin/env python3
"""Benchmark of the P-chase hot path on GB300.

Step (one pass of the hot path over one batch): the batched-simulation
workload of 4096 seeded (geometry, P-chase run) items - capacities 1 KB to
256 KB (2^k and 3*2^k), lines 32-256 B, 1..32-way or fully associative,
LRU / FIFO / RANDOM, strides 4 B - 4 KB, arrays C/2..2C, lengths 1K-1M
accesses (about 0.64 G accesses).  Each step builds every trace into HBM
(S1, pchase_build_batch) and replays all items in one planned launch set
(S2/S3 with the persistent per-class queues of S6), both captured in one
CUDA graph.  The metric is simulated accesses per second.

Also reported: the end-to-end rate through the one-shot C ABI call with host
descriptors in and host bitmaps out, the simulator's roofline (trace
streaming: 4 B read + 1/8 B written per access, against measured HBM copy
bandwidth), traces inferred per second by the exhaustive matcher on the
one-geometry configuration, and the CPU oracle on a bounded sample of the
same workload.

Multi-GPU (torchrun): each rank simulates its own batch (seeds offset by
rank), no collective on the data path; value = all ranks' accesses / the
slowest rank's time (weak scaling).

--impl reference runs the CPU oracle (the slow reference this repository
keeps for parity) on a bounded sample per step, on the host's cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "simulated accesses/s (batched cache simulation, 4096 geometries x P-chase traces)"
UNIT = "accesses/s"
WORKLOAD = ("batched simulation: 4096 seeded geometries (C 1-256 KB, b 32-256 B, 1-32 ways or "
            "full, LRU/FIFO/RANDOM), strides 4 B-4 KB, N in C/2..2C, lengths 1K-1M, one launch set")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--items", type=int, default=4096)
    p.add_argument("--max-len", type=int, default=1 << 20,
                   help="longest trace of the batch (smaller for profiler captures)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-infer", action="store_true")
    p.add_argument("--no-graph", action="store_true",
                   help="launch each step directly instead of replaying a CUDA graph "
                        "(for profilers that cannot follow stream capture)")
    p.add_argument("--cpu-sample", type=int, default=512, help="items in the oracle sample")
    p.add_argument("--no-tune", action="store_true", help="skip the autotuner (default knobs)")
    p.add_argument("--retune", action="store_true",
                   help="run the autotuner afresh instead of using the shipped knobs")
    p.add_argument("--no-learned", action="store_true", help="skip the learned-inverse section")
    p.add_argument("--no-probes", action="store_true", help="skip the on-device probe section")
    p.add_argument("--no-hierarchy", action="store_true",
                   help="skip the cache / TLB hierarchy section")
    p.add_argument("--no-mixed", action="store_true",
                   help="skip the large mixed batch (65,536 cache and TLB hierarchies)")
    p.add_argument("--no-variants", action="store_true",
                   help="skip the set-mapping / weighted-policy section")
    p.add_argument("--inverse-steps", type=int, default=2442,
                   help="training steps of 4096 synthetic traces for the learned inverse")
    p.add_argument("--inverse-eval", type=int, default=100000)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------ multi-GPU
def rank_workload(rank: int, items: int, max_len: int):
    """Rank r's own batch: the same recipe with its own seed range (items
    r*items .. (r+1)*items - 1 of the seed sequence), so ranks share no item."""
    from paper_1509_02308_gb300 import workloads as W
    return W.config2(n_items=items, seed_base=0x5EED0002 + rank * items, max_len=max_len)


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's time (all_reduce MAX); the value itself when alone."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# From one ncu capture (three single-pass counters) of the current sim_kernel
# on the full batched workload, 644,096,746 accesses: the slot-mix launch and
# the one-warp launch of one run, summed.
SIM_DRAM_BYTES_PER_ACCESS = (2790.483456e6 + 62.115584e6 + 24.692736e6) / 644096746
SIM_WARP_INST_PER_ACCESS = (3408117654 + 47543930) / 644096746
# Algorithmic work of one simulated access in the warp-per-set mapping: the
# decode (line, set and tag by shift and multiply-high), one warp-wide tag
# compare (ballot / match), the replacement-state update and the miss bit,
# about 4-6 warp instructions; the middle of that range.
ALG_WARP_INST_PER_ACCESS = 5.0
# multiply-adds x 2 of one trace through the learned inverse: four k5 s2
# convolutions to 64 channels (256 x 64 x 5, then 128, 64 and 32 positions x
# 64 x 320), FC 2048 -> 256, heads 256 -> 31
INVERSE_FLOP_PER_TRACE = 2 * (256 * 64 * 5 + (128 + 64 + 32) * 64 * 320 + 2048 * 256 + 256 * 31)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------- CPU oracle
def oracle_sample(geoms, runs, n_items, seed=0xC0DE):
    rng = np.random.Generator(np.random.PCG64(seed))
    return sorted(rng.choice(len(runs), size=min(n_items, len(runs)), replace=False).tolist())


def run_oracle(geoms, runs, idx, threads):
    """The oracle's full output (per-access miss flags) for items idx, one item
    per thread; returns (accesses, wall seconds, flags per item)."""
    import oracle

    def one(i):
        g, r = geoms[i], runs[i]
        tr = oracle.pchase_trace(r.n_elems, r.stride, r.length)
        return oracle.cache_sim(g.C, g.b, g.ways, g.sets, g.policy, tr, seed=g.seed)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(one, idx))
    dt = time.perf_counter() - t0
    acc = sum(runs[i].length for i in idx)
    return acc, dt, res


def cpu_baseline(geoms, runs, n_items):
    """The oracle on a fixed seeded sample of the batch (all host cores, one
    item per thread), and on one core over the same items.  Also returns the
    sample and its flags for the parity check."""
    idx = oracle_sample(geoms, runs, n_items)
    cores = os.cpu_count() or 1
    acc, dt, flags = run_oracle(geoms, runs, idx, cores)
    # one core over the same items: the few fully associative items of
    # thousands of ways take most of the oracle's time, so a smaller sample
    # would not have their mix
    idx1 = idx
    acc1, dt1, _ = run_oracle(geoms, runs, idx1, 1)
    return {"value": acc / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(idx)} seeded items of the 4096-item batch at full length "
                      f"({acc} accesses, {dt:.1f} s wall, one item per thread, per-access "
                      f"miss flags out)",
            "single_thread": {"value": acc1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"the same {len(idx1)} items on one core "
                                        f"({acc1} accesses, {dt1:.1f} s)"}}, idx, flags


def parity_check(bitmaps_host, counts_host, word_offsets, runs, idx, flags) -> dict:
    """Bit-exact comparison of the timed run's outputs (bitmaps and both miss
    counts) with the oracle's flags for the sampled items."""
    bad = []
    acc = 0
    for i, want in zip(idx, flags):
        n = runs[i].length
        w0 = int(word_offsets[i])
        got = np.unpackbits(bitmaps_host[w0:w0 + (n + 31) // 32].view(np.uint8),
                            bitorder="little")[:n]
        acc += n
        if (not np.array_equal(got, want) or int(counts_host[i, 0]) != int(want.sum())
                or int(counts_host[i, 1]) != int(want[runs[i].warmup:].sum())):
            bad.append(int(i))
    return {"parity_ok": not bad, "parity_items_checked": len(idx),
            "parity_accesses_checked": acc, "parity_mismatched_items": bad[:16]}


# ------------------------------------------------------------- our arm
def ours(args):
    import torch

    from paper_1509_02308_gb300 import api, workloads as W

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    geoms, runs = rank_workload(rank, args.items, args.max_len)
    total_acc = W.total_accesses(runs)
    offs = np.zeros(len(runs) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([r.length for r in runs])
    flat = torch.empty(int(offs[-1]), dtype=torch.int32, device=dev)
    traces = [(flat[int(offs[i]):int(offs[i + 1])], r.length, r.warmup, r.n_elems, r.stride)
              for i, r in enumerate(runs)]
    pairs = [(i, i) for i in range(len(runs))]
    tune = None
    tune_note = "defaults"
    shipped = None
    if not args.no_tune and not args.retune:
        from paper_1509_02308_gb300 import autotune
        shipped = autotune.lookup(geoms, traces, pairs)
    if shipped is not None:
        tune = shipped
        tune_note = ("autotuned on a GB300 (coordinate descent on this workload), knobs shipped "
                     "in the package's tuned.json")
    elif not args.no_tune:
        from paper_1509_02308_gb300 import autotune
        # the traces must exist before candidate plans are timed: build them once
        from paper_1509_02308_gb300 import capi as _C
        import ctypes as _ct
        _d = _C.trace_array((None, r.length, r.warmup, r.n_elems, r.stride) for r in runs)
        _o = _C.u64_array(offs[:-1])
        _C.check(_C.load().pchase_build_batch(_ct.addressof(_d), len(runs), _C.ptr(flat),
                                              _o.ctypes.data, _C.stream_handle()))
        torch.cuda.synchronize()
        tune = autotune.tune(geoms, traces, pairs=pairs, reps=2, sweeps=1, fresh=args.retune)
        tune_note = "autotuned in this run (coordinate descent on this workload)"
    plan = api.SimPlan(geoms, traces, pairs=pairs, tune=tune)
    bitmaps = torch.empty(max(1, plan.bitmap_words), dtype=torch.int32, device=dev)
    counts = torch.empty(2 * len(runs), dtype=torch.int64, device=dev)

    from paper_1509_02308_gb300 import capi as C
    descs = C.trace_array((None, r.length, r.warmup, r.n_elems, r.stride) for r in runs)
    d_offs = C.u64_array(offs[:-1])
    L = C.load()
    import ctypes

    def build(stream):
        C.check(L.pchase_build_batch(ctypes.addressof(descs), len(runs), C.ptr(flat),
                                     d_offs.ctypes.data, C.stream_handle(stream)))

    def step(stream):
        build(stream)
        plan.run(bitmaps=bitmaps, counts=counts, stream=stream)

    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step(s)  # first run creates the plan's streams and events
    torch.cuda.synchronize()
    if args.no_graph:
        class _Direct:
            def replay(self):
                with torch.cuda.stream(s):
                    step(s)
                torch.cuda.current_stream().wait_stream(s)
        graph = _Direct()
    else:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            step(s)
    launches_per_step = math.ceil(len(runs) / 1024) + plan.launches

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()

    vis = [x for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip().isdigit()]
    clocks = ClockSampler(int(vis[local]) if local < len(vis) else local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    cur = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for _ in range(args.steps):
        graph.replay()
    e1.record(cur)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    # the dominant kernel set (S3) timed alone, each launch bracketed by events
    # on the stream it is launched from
    sim_ms = []
    for _ in range(max(3, args.steps // 2)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            a.record(s)
            plan.run(bitmaps=bitmaps, counts=counts, stream=s)
            b.record(s)
        torch.cuda.synchronize()
        sim_ms.append(a.elapsed_time(b))
    build_ms = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            a.record(s)
            build(s)
            b.record(s)
        torch.cuda.synchronize()
        build_ms.append(a.elapsed_time(b))
    clk = clocks.stop()
    # outputs of the last run of the timed plan, for the parity check below
    bits_host = bitmaps.cpu().numpy().view(np.uint32)
    counts_host = counts.view(-1, 2).cpu().numpy()

    # max over ranks
    t_step = max_over_ranks(ms / args.steps, world, dev)
    value = total_acc * world / (t_step * 1e-3)

    peaks, peak_kind = measured_peaks()
    sim_avg = statistics.mean(sim_ms)
    alg_bytes = total_acc * 4.0 + total_acc / 8.0
    achieved = alg_bytes / (sim_avg * 1e-3) / 1e9
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # DRAM bytes per access of sim_kernel from one ncu capture of the same
    # kernel on this workload with items capped at 64 K accesses (273.2 MB for
    # 65,559,830 accesses), scaled to this launch set by its accesses
    traffic = SIM_DRAM_BYTES_PER_ACCESS * total_acc
    # The simulator is bound by integer / shared-memory instruction issue, not
    # by HBM or tensor cores: its roofline is the SMs' warp-instruction issue
    # rate (SMs x 4 schedulers x 1 warp instruction per cycle x the maximum SM
    # clock) against ALG_WARP_INST_PER_ACCESS algorithmic warp instructions per
    # access; HBM (trace streaming) is the secondary bound.
    f_max = peaks.get("sm_max_mhz", 2070.0)
    issue_peak = sms * 4 * f_max * 1e6 / 1e9  # G warp instructions / s
    alg_inst = total_acc * ALG_WARP_INST_PER_ACCESS
    achieved_inst = alg_inst / (sim_avg * 1e-3) / 1e9
    roof = {"bound": "alu", "achieved": achieved_inst, "peak": issue_peak,
            "unit": "G warp-instructions/s", "frac": achieved_inst / issue_peak,
            "traffic": traffic,
            "peak_kind": (f"{sms} SMs x 4 warp schedulers x {f_max:.0f} MHz (maximum SM clock, "
                          f"{peak_kind} peaks file)"),
            "algorithmic_warp_inst_per_access": ALG_WARP_INST_PER_ACCESS,
            "algorithmic_warp_inst_per_launch": alg_inst,
            "measured_warp_inst_per_access": SIM_WARP_INST_PER_ACCESS,
            "measured_issue_frac": (total_acc * SIM_WARP_INST_PER_ACCESS / (sim_avg * 1e-3) / 1e9
                                    / issue_peak),
            "hbm": {"achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"],
                    "algorithmic_bytes_per_launch": alg_bytes,
                    "peak_kind": f"{peak_kind} HBM copy bandwidth",
                    "nominal_8TBs_frac": achieved / 8000.0},
            "kernel": "sim_kernel (all size classes of one pchase_sim_run)",
            "kernel_ms": sim_avg}
    torch.cuda.synchronize()

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "items_per_gpu": len(runs),
                   "accesses_per_gpu_step": total_acc,
                   "l2": "inputs larger than L2 (traces %.2f GB per step)" % (total_acc * 4 / 1e9),
                   "parallelism": f"replicas x{world} (independent batches)",
                   "plan": plan.description, "tune": tune or {}, "tune_source": tune_note},
        "clocks": clk, "gpu_launches": launches_per_step * args.steps,
        "roofline": roof,
        "phases_ms": {"build_S1": statistics.mean(build_ms), "simulate_S3": sim_avg},
    }

    # ------------------------------------------------ end to end through the C ABI
    if not args.no_e2e:
        result["e2e"] = e2e_run(args, geoms, runs, dev, world)

    # ------------------------------------------------ traces inferred per second
    if not args.no_infer and rank == 0:
        try:
            result["inference"] = infer_bench(dev)
        except Exception as ex:  # reported, never hidden
            result["inference"] = {"error": repr(ex)}

    if not args.no_probes and rank == 0:
        try:
            result["probes"] = probe_bench(dev)
        except Exception as ex:  # report, never mask the main number
            result["probes"] = {"error": repr(ex)}
    if not args.no_hierarchy and rank == 0:
        try:
            result["hierarchy"] = hierarchy_bench(dev)
        except Exception as ex:  # noqa: BLE001
            result["hierarchy"] = {"error": repr(ex)}
    if not args.no_mixed and rank == 0:
        try:
            result["mixed"] = mixed_bench(dev)
        except Exception as ex:  # noqa: BLE001
            result["mixed"] = {"error": repr(ex)}
        import torch as _t
        _t.cuda.empty_cache()
    if not args.no_variants and rank == 0:
        try:
            result["variants"] = variants_bench(dev)
        except Exception as ex:  # noqa: BLE001
            result["variants"] = {"error": repr(ex)}
    if not args.no_learned and rank == 0:
        try:
            result["learned_inverse"] = learned_bench(args, dev)
        except Exception as ex:  # reported, never hidden
            result["learned_inverse"] = {"error": repr(ex)}

    li, inf = result.get("learned_inverse", {}), result.get("inference", {})
    if li.get("at_99pct", {}).get("threshold") is not None and "batched" in inf:
        # against the per-access simulate-and-compare matcher (S5): a
        # DIFFERENT observation of a cache (per-access latencies of the 108
        # traces of the one-geometry plan, not a 512-point mean-latency
        # vector), so context only; the like-for-like comparisons are
        # speedup_vs_judge and speedup_vs_exhaustive_with_simulation
        a = li["at_99pct"]
        a["ratio_to_per_access_matcher_other_observation"] = {
            "single_unbounded": a["traces_per_s"] / inf["traces_inferred_per_s"],
            "batched_bound0": a["traces_per_s"] / inf["batched"]["stop0"]["traces_inferred_per_s"]}
    if rank == 0 and not args.no_cpu:
        result["cpu_baseline"], sample, flags = cpu_baseline(geoms, runs, args.cpu_sample)
        # the outputs of the last timed-plan run, checked against the oracle
        result.update(parity_check(bits_host, counts_host, plan.word_offsets, runs, sample,
                                   flags))
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def e2e_run(args, geoms, runs, dev, world):
    """Host descriptors in, host bitmaps and counts out, one-shot C ABI calls."""
    import ctypes

    import torch

    from paper_1509_02308_gb300 import capi as C
    L = C.load()
    n = len(runs)
    offs = np.zeros(n + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([r.length for r in runs])
    words = np.zeros(n + 1, dtype=np.uint64)
    words[1:] = np.cumsum([(r.length + 31) // 32 for r in runs])
    flat = torch.empty(int(offs[-1]), dtype=torch.int32, device=dev)
    # two device result buffers too: step i + 1's kernels write one while step
    # i's copy to the host reads the other on a copy stream
    d_bits = [torch.empty(int(words[-1]), dtype=torch.int32, device=dev) for _ in range(2)]
    d_counts = [torch.empty(2 * n, dtype=torch.int64, device=dev) for _ in range(2)]
    d_words = torch.from_numpy(words[:-1].astype(np.int64)).to(dev)
    # two pinned result buffers: step i's copies land in buffer i % 2, and the
    # host reads a step's result once its copies are done (before that buffer
    # is reused two steps later), so step i + 1's host planning overlaps step
    # i's device work, as a caller streaming batches through the C ABI would
    h_bits = [torch.empty(int(words[-1]), dtype=torch.int32, pin_memory=True) for _ in range(2)]
    h_counts = [torch.empty(2 * n, dtype=torch.int64, pin_memory=True) for _ in range(2)]
    done = [None, None]
    ga = C.geom_array(geoms)
    pa = C.pair_array((i, i) for i in range(n))
    bdescs = C.trace_array((None, r.length, r.warmup, r.n_elems, r.stride) for r in runs)
    b_offs = C.u64_array(offs[:-1])
    base = int(flat.data_ptr())
    tdescs = C.trace_array(((None, r.length, r.warmup, r.n_elems, r.stride) for r in runs))
    for i in range(n):
        tdescs[i].idx = base + 4 * int(offs[i])
    need = ctypes.c_size_t(0)
    def sim_args(b):
        return (ctypes.addressof(ga), n, ctypes.addressof(tdescs), n, ctypes.addressof(pa), n,
                C.ptr(d_bits[b]), C.ptr(d_words), C.ptr(d_counts[b]), None)
    L.cache_sim_batch(*sim_args(0), None, ctypes.byref(need), None)
    # what one call copies to the device: the plan's tables (cache_sim_batch
    # plans with the default knobs, as this plan does)
    hp = ctypes.c_void_p()
    C.check(L.pchase_sim_plan_create(ctypes.addressof(ga), n, ctypes.addressof(tdescs), n,
                                     ctypes.addressof(pa), n, None, ctypes.byref(hp)))
    upload = int(L.pchase_sim_plan_upload_bytes(hp))
    L.pchase_sim_plan_destroy(hp)
    ws = torch.empty(need.value + 256, dtype=torch.uint8, device=dev)
    wp = (C.ptr(ws) + 255) & ~255
    st = torch.cuda.current_stream()
    cs = torch.cuda.Stream()
    copied = [None, None]  # device buffer b free again (its copy is done)
    misses = []

    def read(b):
        # the host's read of a finished step's result (its total miss count)
        if done[b] is not None:
            done[b].synchronize()
            misses.append(int(h_counts[b][1::2].sum()))
            done[b] = None

    def one(i):
        b = i & 1
        read(b)
        C.check(L.pchase_build_batch(ctypes.addressof(bdescs), n, C.ptr(flat), b_offs.ctypes.data,
                                     C.stream_handle(st)))
        if copied[b] is not None:
            st.wait_event(copied[b])
        have = ctypes.c_size_t(need.value)
        C.check(L.cache_sim_batch(*sim_args(b), wp, ctypes.byref(have), C.stream_handle(st)))
        ran = torch.cuda.Event()
        ran.record(st)
        cs.wait_event(ran)
        with torch.cuda.stream(cs):
            h_bits[b].copy_(d_bits[b], non_blocking=True)
            h_counts[b].copy_(d_counts[b], non_blocking=True)
        done[b] = torch.cuda.Event()
        done[b].record(cs)
        copied[b] = done[b]

    def drain():
        read(0)
        read(1)

    for i in range(max(1, min(args.warmup, 2))):
        one(i)
    drain()
    k = max(2, min(args.steps, 5))
    t0 = time.perf_counter()
    for i in range(k):
        one(i)
    drain()
    dt = (time.perf_counter() - t0) / k
    assert len(set(misses)) == 1, misses  # every step computed the same batch
    total = int(offs[-1])
    h2d = upload + n * 24
    d2h = int(words[-1]) * 4 + 2 * n * 8
    return {"value": total * world / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3,
            "path": "pchase_build_batch + cache_sim_batch (plan, upload, run) + bitmaps/counts "
                    "to pinned host memory, read on the host; two result buffers on the device "
                    "and the host, the copies on a second stream: a step's host planning and "
                    "the previous step's copies overlap this step's device work"}


def infer_bench(dev):
    """Exhaustive inference on the one-geometry configuration: candidates are
    the whole grid x {LRU, FIFO, RANDOM}; the plan is the 97 stride-128 B runs
    plus 11 stride-4 B runs around C; each observation is a fresh noisy latency
    trace of the true cache (16 KB, 128 B, 4-way, LRU)."""
    import torch

    from paper_1509_02308_gb300 import api, workloads as W

    truth, runs = W.config1()
    C0 = truth.C
    for nb in (C0 - 4, C0, C0 + 4, C0 + 32, C0 + 36, C0 + 64, C0 + 68, C0 + 128, C0 + 132,
               C0 + 256, C0 + 260):
        n = nb // 4
        runs.append(W.Run(n, 1, 3 * n, n))
    cands = [W.Geom(C, b, a, T, p, 0x5EED + i)
             for i, (C, b, a, T) in enumerate(W.geometry_grid()) for p in (0, 1, 2)]
    offs = np.zeros(len(runs) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([r.length for r in runs])
    flat_built, _ = api.pchase_build_batch(runs)
    traces = [(flat_built[int(offs[i]):int(offs[i + 1])], r.length, r.warmup, r.n_elems, r.stride)
              for i, r in enumerate(runs)]
    plan = api.SimPlan(cands, traces)
    # observations: latencies synthesised from the truth's miss pattern, which
    # the library simulates (the tests hold it bit-exact to the oracle)
    tb, _, toffs = api.cache_sim_batch([truth], traces, pairs=[(0, i) for i in range(len(runs))])
    tbw = tb.cpu().numpy().view(np.uint32)
    miss = np.concatenate([api.unpack_bits(tbw[int(toffs[i]):], r.length)
                           for i, r in enumerate(runs)]).astype(np.float64)
    rng = np.random.Generator(np.random.PCG64(0x5EED1001))
    n_obs = 8
    lats = []
    for _ in range(n_obs):
        lat = (100.0 + 300.0 * miss) * (1.0 + 0.02 * rng.standard_normal(miss.size))
        lats.append(torch.from_numpy(lat.astype(np.float32)).to(dev))
    rows = [c for c in cands]
    truth_idx = [i for i, c in enumerate(rows) if (c.C, c.b, c.ways, c.policy) ==
                 (truth.C, truth.b, truth.ways, 0)][0]
    # exact-recovery reference: the canonical class of the truth on this plan
    plan.infer(lats[0])
    torch.cuda.synchronize()
    res = []
    for stop in (2**64 - 1, 0):
        picks = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for lat in lats:
            d, p = plan.infer(lat, stop_above=stop)
            picks.append(p)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / n_obs
        picks = [int(p[0]) for p in picks]
        res.append((stop, dt, picks))
    full_dt, full_picks = res[0][1], res[0][2]
    fast_dt, fast_picks = res[1][1], res[1][2]
    exact = sum(1 for p in full_picks if p == truth_idx) / n_obs
    exact_fast = sum(1 for p in fast_picks if p == truth_idx) / n_obs
    sim_acc = len(cands) * int(offs[-1])
    # batched: many observations per call, each with its own noise
    n_batch = 256
    lat_b = torch.from_numpy(np.stack([
        ((100.0 + 300.0 * miss) * (1.0 + 0.02 * rng.standard_normal(miss.size))).astype(np.float32)
        for _ in range(n_batch)])).to(dev)
    batch = {}
    for stop, name in ((2**64 - 1, "unbounded"), (0, "stop0")):
        api.infer_batch(plan, lat_b[:8], stop_above=stop)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, pk = api.infer_batch(plan, lat_b, stop_above=stop)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        pk = pk.cpu().numpy()
        batch[name] = {"traces_inferred_per_s": n_batch / dt,
                       "exact_recovery": float((pk[:, 0] == truth_idx).mean()),
                       "observations_per_call": n_batch}
    return {"traces_inferred_per_s": 1.0 / full_dt, "exact_recovery": exact,
            "traces_inferred_per_s_stop0": 1.0 / fast_dt, "exact_recovery_stop0": exact_fast,
            "batched": batch,
            "candidates": len(cands), "plan_traces": len(runs), "plan_accesses": int(offs[-1]),
            "simulated_accesses_per_inference": sim_acc,
            "matcher_accesses_per_s": sim_acc / full_dt,
            "note": "one observation = latencies of all plan traces (2% jitter); stop0 = "
                    "distance bound 0, exact whenever a candidate matches perfectly; batched = "
                    "infer_geometry_batch over 256 observations per call"}


def probe_bench(dev):
    """The sm_103a probes on this GPU (S8-S10): P-chase latency plateaus,
    the shared-memory bank sweep, and global read/write/copy throughput over
    1 GB against the measured HBM copy bandwidth, swept over CTAs per SM and
    loads in flight per thread."""
    import math

    import torch

    from paper_1509_02308_gb300 import api

    out = {}
    # latency regimes (medians of 2048 timed accesses, cycles, overhead removed)
    lat = {}
    for name, nbytes, sb, mode in (("l1_16KB_s128B", 16 << 10, 128, 0),
                                   ("l2_4MB_s128B", 4 << 20, 128, 1),
                                   ("hbm_512MB_s4KB", 512 << 20, 4096, 1)):
        n = nbytes // 4
        _, arr = api.pchase_build(n, sb // 4, 1, with_array=True)
        l, _, _, st = api.pchase_probe_latency(arr, n, iters=2048, warmup=n // (sb // 4) if
                                               nbytes <= (4 << 20) else 0, cache_mode=mode)
        torch.cuda.synchronize()
        lat[name] = float(np.median(l.cpu().numpy().view(np.uint32)))
        del arr
    out["latency_cycles"] = lat
    cyc, deg = api.pchase_probe_smem_bank(64, repeats=9)
    cyc, deg = cyc.cpu().numpy(), deg.cpu().numpy()
    out["smem_bank"] = {"cycles_by_degree": {int(d): float(np.median(cyc[deg == d]))
                                             for d in (1, 2, 4, 8, 16, 32)},
                        "degree_is_gcd_s_32": bool(all(deg[s - 1] == math.gcd(s, 32)
                                                       for s in range(1, 65)))}
    nbytes = 1 << 30
    a = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    b = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks, peak_kind = measured_peaks()
    thr = {}
    for kind, name in ((0, "read"), (1, "write"), (2, "copy")):
        best, cfg = 0.0, None
        for per_sm in (2, 4, 8):
            for ilp in (1, 2, 4, 8):
                g = api.pchase_probe_global_throughput(kind, 16, sms * per_sm, 256, ilp, a, b,
                                                       nbytes, reps=5)
                if g > best:
                    best, cfg = g, {"ctas_per_sm": per_sm, "threads": 256, "ilp": ilp,
                                    "vector_bytes": 16}
        thr[name] = {"gbs": best, "frac_of_measured": best / peaks["hbm_gbs"],
                     "frac_of_nominal_8TBs": best / 8000.0, "best_config": cfg}
    out["global_throughput_1GB"] = thr
    out["peak_kind"] = f"{peak_kind} HBM copy bandwidth {peaks['hbm_gbs']} GB/s"
    del a, b
    torch.cuda.empty_cache()
    out["smem_throughput"] = smem_throughput_sweep(dev)
    out["latency_spectrum"] = latency_spectrum(dev)
    out["pchase_sweep"] = pchase_sweep(dev)
    out["global_throughput_sweep"] = global_throughput_sweep(dev)
    return out


def pchase_sweep(dev, runs: int = 10, timed: int = 256, max_warm: int = 65536):
    """The fine-grained P-chase (Listing 3) over every array size N = 4 KB ..
    512 MB and stride s = 32 B .. 2 MB (powers of two, s <= N / 2) on this GPU,
    L1 on (ld.global.ca).  Each run starts after a 256 MB write has cleared
    L2, preheats with one pass over the chain's N / s elements (at most
    max_warm accesses: beyond that the timed accesses are first touches) and
    times the next `timed` accesses; a point reports the median over `runs`
    runs of each run's median latency, in cycles with the clock overhead
    removed."""
    import torch

    from paper_1509_02308_gb300 import api

    Ns = [1 << k for k in range(12, 30)]
    Ss = [1 << k for k in range(5, 22)]
    table = []
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    t0 = time.perf_counter()
    for nb in Ns:
        n = nb // 4
        row = []
        for sb in Ss:
            if sb > nb // 2:
                row.append(None)
                continue
            _, arr = api.pchase_build(n, sb // 4, 1, with_array=True)
            per = nb // sb
            meds = []
            for _ in range(runs):
                flush.fill_(1)
                lat, _, _, st = api.pchase_probe_latency(arr, n, iters=timed,
                                                         warmup=min(per, max_warm), cache_mode=0)
                torch.cuda.synchronize()
                if int(st.item()):
                    return {"error": f"probe status {int(st.item())} at N={nb} s={sb}"}
                meds.append(float(np.median(lat.cpu().numpy().view(np.uint32))))
            row.append(float(np.median(meds)))
            del arr
        table.append(row)
    del flush
    torch.cuda.empty_cache()
    return {"N_bytes": Ns, "s_bytes": Ss, "median_cycles": table, "runs_per_point": runs,
            "timed_accesses_per_run": timed, "preheat_accesses_max": max_warm,
            "cache_mode": "ld.global.ca (L1 and L2)", "wall_s": time.perf_counter() - t0}


def global_throughput_sweep(dev, reps: int = 10):
    """Sec. 5.1's throughput sweep on this GPU: read, write and copy (copy
    counts 2 x bytes, as the paper does) over buffers of 1 MB .. 4 GB (powers
    of two) with 4-byte (fp32) and 16-byte (int4) vectors; per point the best,
    over CTAs per SM {2, 4, 8} x loads in flight per thread {1, 2, 4, 8}, of
    the median of `reps` timed launches.  Buffers up to the 129 MB L2 are
    served from it, so only larger ones are against the HBM copy peak."""
    import torch

    from paper_1509_02308_gb300 import api

    peaks, peak_kind = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sizes = [1 << k for k in range(20, 33)]
    top = sizes[-1]
    a = torch.zeros(top, dtype=torch.uint8, device=dev)
    b = torch.empty(top, dtype=torch.uint8, device=dev)
    out = {"bytes": sizes, "peak_gbs": peaks["hbm_gbs"], "peak_kind": peak_kind,
           "l2_bytes": 129 * 10 ** 6}
    t0 = time.perf_counter()
    for kind, kname in ((0, "read"), (1, "write"), (2, "copy")):
        for vec, vname in ((4, "fp32"), (16, "int4")):
            gbs, cfgs = [], []
            for nb in sizes:
                best, cfg = 0.0, None
                for per_sm in (2, 4, 8):
                    for ilp in (1, 2, 4, 8):
                        if nb % (vec * ilp):
                            continue
                        g = api.pchase_probe_global_throughput(kind, vec, sms * per_sm, 256, ilp,
                                                               a, b, nb, reps=reps)
                        if g > best:
                            best, cfg = g, [per_sm, ilp]
                gbs.append(best)
                cfgs.append(cfg)
            out[f"{kname}_{vname}"] = {
                "gbs": gbs, "best_ctas_per_sm_ilp": cfgs,
                "frac_of_measured_above_l2": [g / peaks["hbm_gbs"] if nb > 129 * 10 ** 6 else None
                                              for g, nb in zip(gbs, sizes)]}
    out["wall_s"] = time.perf_counter() - t0
    del a, b
    torch.cuda.empty_cache()
    return out


def latency_spectrum(dev, reps: int = 5):
    """Sec. 5.2's non-uniform-stride P-chase on this GPU (Fig. 11's P1-P6):
    the chain of workloads.spectrum_chain() walked once, cold, with L1 on
    (ld.global.ca) and off (ld.global.cg); per segment the median latency in
    cycles over `reps` walks, each after writing 512 MB to clear the caches."""
    import torch

    from paper_1509_02308_gb300 import api, workloads as W

    path, labels, n = W.spectrum_chain()
    arr = torch.zeros(n, dtype=torch.int32, device=dev)
    arr[torch.tensor(path, dtype=torch.int64, device=dev)] = torch.tensor(
        path[1:] + path[:1], dtype=torch.int32, device=dev)
    lab = np.array(labels)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    out = {"segments": {"B_new_page": "1 MB stride, first access to a 2 MB page: cache miss, TLB miss (P5)",
                        "B_same_page": "1 MB stride, page of the previous access: cache miss, TLB hit (P4)",
                        "A_32MB": "32 MB stride over 2 GB: cache miss, TLB miss (P5/P6)",
                        "C_revisit": "B's lines again after A's sweep: cache hit, TLB miss (P2/P3)",
                        "D_same_line": "one 128-byte line: cache hit, TLB hit (P1)"}}
    for mode, name in ((0, "l1_on_ld_ca"), (1, "l1_off_ld_cg")):
        per = {k: [] for k in out["segments"]}
        for _ in range(reps):
            flush.fill_(1)
            lat, vis, _, st = api.pchase_probe_latency(arr, n, iters=len(path), warmup=0,
                                                       start=path[0], cache_mode=mode)
            torch.cuda.synchronize()
            if int(st.item()) or not np.array_equal(vis.cpu().numpy().view(np.uint32),
                                                    np.array(path, dtype=np.uint32)):
                return {"error": "the probe left the constructed chain"}
            l = lat.cpu().numpy().view(np.uint32)
            for k in per:
                per[k].append(float(np.median(l[lab == k])))
        out[name] = {k: float(np.median(v)) for k, v in per.items()}
    del arr, flush
    torch.cuda.empty_cache()
    return out


def smem_throughput_sweep(dev):
    """Sec. 6.1's grid on this GPU: CTA size {32 .. 1024} x CTAs per SM {1 .. 6}
    x ILP {1, 2, 4, 6, 8}, where the CTAs fit on an SM together (threads and
    shared memory).  Throughput per SM in bytes per SM cycle (read + write,
    as the paper counts), against 32 banks x 4 B = 128 B per cycle."""
    import torch

    from paper_1509_02308_gb300 import api

    prop = torch.cuda.get_device_properties(dev)
    max_thr = getattr(prop, "max_threads_per_multi_processor", 2048)
    smem_sm = getattr(prop, "shared_memory_per_multiprocessor", 228 * 1024)
    peaks, _ = measured_peaks()
    f_mhz = peaks.get("sm_max_mhz", 2070.0)
    best, best_cfg, by_warps = 0.0, None, {}
    for threads in (32, 64, 128, 256, 512, 1024):
        for per_sm in range(1, 7):
            for ilp in (1, 2, 4, 6, 8):
                cta_smem = 8 * ilp * threads
                if threads * per_sm > max_thr or (cta_smem + 1024) * per_sm > smem_sm:
                    continue
                r = api.pchase_probe_smem_throughput(per_sm, threads, ilp, iters=2048)
                if r["ctas_per_sm_seen"] != [per_sm, per_sm]:
                    continue
                bpc = r["bytes_per_cycle"]
                warps = threads // 32 * per_sm
                if bpc > by_warps.get(warps, (0.0,))[0]:
                    by_warps[warps] = (bpc, {"threads": threads, "ctas_per_sm": per_sm,
                                             "ilp": ilp})
                if bpc > best:
                    best, best_cfg = bpc, {"threads": threads, "ctas_per_sm": per_sm, "ilp": ilp,
                                           "active_warps": warps}
    return {"peak_bytes_per_sm_cycle": best, "theoretical_bytes_per_sm_cycle": 128.0,
            "efficiency": best / 128.0, "best_config": best_cfg,
            "peak_gbs_per_sm_at_max_clock": best * f_mhz * 1e6 / 1e9, "sm_max_mhz": f_mhz,
            "peak_by_active_warps": {str(w): round(v[0], 2) for w, v in sorted(by_warps.items())}}


def variants_bench(dev):
    """Set mappings from higher line bits and the weighted Fermi L1 policy on
    the paper's own sweeps.  The texture L1 caches of Sec. 4.3 (12 KB and
    24 KB, 32 B lines, 4 sets, address bits 7-8: mapping 2, LRU) over
    s = 4 B and 32 B with N from C to C + 512 B in 32 B steps, then to 60 KB in
    1 KB steps; the Fermi L1 data cache of Sec. 4.5 (16 KB, 128 B lines,
    4 ways, 32 sets, weighted policy) under 64 policy seeds over N = 15-24 KB
    in 128 B steps with s = 4 B and 128 B; 4 passes each, the first one
    warm-up.  Reports simulated accesses/s of the plan run, and whether the
    matcher, given the 12 KB texture cache's bitmaps, picks the bits-7-8
    mapping among mappings 0-3 x {LRU, FIFO, RANDOM}."""
    import torch

    from paper_1509_02308_gb300 import api, workloads as W

    def sweep(sizes, strides_b):
        out = []
        for nb in sizes:
            for sb in strides_b:
                n, s = nb // 4, sb // 4
                per = n // math.gcd(n, s)
                out.append(W.Run(n, s, 4 * per, per))
        return out

    tex_geoms = [W.Geom(12288, 32, 96, 4, W.LRU, mapping=2), W.Geom(24576, 32, 192, 4, W.LRU, mapping=2)]
    tex_runs = [sweep(list(range(C, C + 513, 32)) + list(range(C + 1024, 61441, 1024)), (4, 32))
                for C in (12288, 24576)]
    fermi_runs = sweep(list(range(15 * 1024, 24 * 1024 + 1, 128)), (4, 128))
    fermi_geoms = [W.Geom(16384, 128, 4, 32, W.WEIGHTED, 0xFE1 + 7919 * k) for k in range(64)]
    runs = tex_runs[0] + tex_runs[1] + fermi_runs
    geoms = tex_geoms + fermi_geoms
    pairs = [(0, t) for t in range(len(tex_runs[0]))]
    pairs += [(1, len(tex_runs[0]) + t) for t in range(len(tex_runs[1]))]
    f0 = len(tex_runs[0]) + len(tex_runs[1])
    pairs += [(2 + k, f0 + t) for k in range(len(fermi_geoms)) for t in range(len(fermi_runs))]
    flat, offs = api.pchase_build_batch(runs)
    traces = [(flat[int(offs[i]):int(offs[i + 1])], r.length, r.warmup, r.n_elems, r.stride)
              for i, r in enumerate(runs)]
    plan = api.SimPlan(geoms, traces, pairs=pairs)
    total = sum(runs[t].length for _, t in pairs)
    bitmaps, counts = plan.run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    a.record()
    for _ in range(reps):
        plan.run(bitmaps, counts)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    # recovery of the texture L1 mapping from its own bitmaps
    n0 = len(tex_runs[0])
    cands = [W.Geom(12288, 32, 96, 4, p, 0x7E57 + p, mapping=m) for m in range(4) for p in (0, 1, 2)]
    mplan = api.SimPlan(cands, traces[:n0])
    owo = torch.tensor(plan.word_offsets[:n0].astype(np.int64), device=dev)
    dist = mplan.match(bitmaps, owo).cpu().numpy()
    pick = api.pchase_canonical_pick(cands, torch.from_numpy(dist.astype(np.int64)).to(dev))
    picked = cands[int(pick[0])]
    return {"accesses_per_s": total / (ms * 1e-3), "ms_per_run": ms, "items": len(pairs),
            "accesses": total, "plan": plan.description,
            "texture_l1_mapping_recovered": picked.mapping == 2 and picked.policy in (0, 1),
            "texture_l1_min_distance_other_mappings":
                int(min(d for c, d in zip(cands, dist) if c.mapping != 2)),
            "note": "texture L1 (Sec. 4.3, bits 7-8) and 24 KB variant, LRU; Fermi L1 (Sec. 4.5) "
                    "weighted policy x 64 seeds; paper sweeps, 4 passes"}


def hierarchy_bench(dev, reps: int = 3):
    """Cache and TLB hierarchies (workloads.hierarchy_config: 1024 items, L1
    16-256 KB -> L2 0.5-3 MB, and a 16-entry L1 TLB -> 8-way L2 TLB over 4 KB
    or 64 KB pages, or the unequal-set L2 TLB of Sec. 4.4 over 2 MB pages,
    142 M trace accesses).  One step runs both cascades
    (4 levels: L1, L2 on L1's misses, L1 TLB, L2 TLB on its misses).  Reports
    trace accesses/s through both cascades, level accesses simulated per
    second, and where the accesses were served."""
    import torch

    from paper_1509_02308_gb300 import api, workloads as W

    l1, l2, t1, t2, runs = W.hierarchy_config()
    flat, offs = api.pchase_build_batch(runs)
    traces = [(flat[int(offs[i]):int(offs[i + 1])], r.length, r.warmup, r.n_elems, r.stride)
              for i, r in enumerate(runs)]
    pairs = [(i, i) for i in range(len(runs))]
    data = api.HierarchyPlan([l1, l2], traces, pairs=pairs)
    tlb = api.HierarchyPlan([t1, t2], traces, pairs=pairs)
    out = data.run() + tlb.run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        out = data.run() + tlb.run()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    # each level alone (the same launches, timed one plan at a time)
    level_ms = []
    for k, plan in enumerate(data.plans + tlb.plans):
        first = k in (0, len(data.plans))
        prev = None if first else out[k - 1][0]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            if first:
                plan.run()
            else:
                plan.run_filtered(prev, data._wo)
        e1.record()
        torch.cuda.synchronize()
        level_ms.append(e0.elapsed_time(e1) / reps)
    total = sum(r.length for r in runs)
    miss = [int(o[1].view(-1, 2)[:, 0].sum().item()) for o in out]  # L1, L2, TLB1, TLB2
    level_accesses = 2 * total + miss[0] + miss[2]
    return {"trace_accesses_per_s": total / (ms * 1e-3), "ms_per_step": ms,
            "level_accesses_per_s": level_accesses / (ms * 1e-3), "items": len(runs),
            "ms_by_level": dict(zip(("l1", "l2", "l1_tlb", "l2_tlb"), level_ms)),
            "trace_accesses": total, "served_from": {
                "l1": 1.0 - miss[0] / total, "l2": (miss[0] - miss[1]) / total,
                "memory": miss[1] / total},
            "translated_by": {"l1_tlb": 1.0 - miss[2] / total, "l2_tlb": (miss[2] - miss[3]) / total,
                              "page_walk": miss[3] / total},
            "plans": [p.description for p in data.plans + tlb.plans]}


def mixed_bench(dev, sample: int = 24):
    """The large mixed batch (workloads.mixed_config): 65,536 items, each an
    L1 (16-256 KB) -> L2 (1-128 MB) cache cascade and a 16-entry L1 TLB ->
    L2 TLB cascade (4 KB, 64 KB or 2 MB pages; over 2 MB pages the unequal
    L2 TLB of Sec. 4.4), over analytic P-chase streams of 4K-16M accesses
    (37 G in all).  One warm-up run, then one timed run of all four levels;
    the L2 caches that no shared-memory arena holds run as way scans over
    set state in the global-memory pool.  A seeded sample of items (the
    longest among them) is checked level by level against the oracle's
    cascade."""
    import torch

    import oracle
    from paper_1509_02308_gb300 import api, workloads as W

    l1, l2, t1, t2, runs = W.mixed_config()
    traces = [(None, r.length, r.warmup, r.n_elems, r.stride) for r in runs]
    pairs = [(i, i) for i in range(len(runs))]
    t0 = time.perf_counter()
    data = api.HierarchyPlan([l1, l2], traces, pairs=pairs)
    tlb = api.HierarchyPlan([t1, t2], traces, pairs=pairs)
    t_plan = time.perf_counter() - t0
    out = data.run() + tlb.run()
    torch.cuda.synchronize()
    del out
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    ev[0].record()
    o1 = data.plans[0].run()
    ev[1].record()
    o2 = data.plans[1].run_filtered(o1[0], data._wo)
    ev[2].record()
    o3 = tlb.plans[0].run()
    ev[3].record()
    o4 = tlb.plans[1].run_filtered(o3[0], tlb._wo)
    ev[4].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[4])
    level_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(4)]
    outs = [o1, o2, o3, o4]
    total = sum(r.length for r in runs)
    miss = [int(o[1].view(-1, 2)[:, 0].sum().item()) for o in outs]
    # parity: a seeded sample, half of it among the longest items
    rng = np.random.Generator(np.random.PCG64(0x5EED15))
    longest = sorted(range(len(runs)), key=lambda i: -runs[i].length)[:200]
    idx = sorted(set(rng.choice(len(runs), sample // 2, replace=False).tolist()) |
                 set(rng.choice(longest, sample // 2, replace=False).tolist()))
    words = [o[0] for o in outs]

    def want_of(i):
        r = runs[i]
        tr = oracle.pchase_trace(r.n_elems, r.stride, r.length)
        lv = [dict(C=g.C, b=g.b, ways=g.ways, T=g.sets, policy=g.policy, seed=g.seed,
                   extra=g.extra) for g in (l1[i], l2[i])]
        lt = [dict(C=g.C, b=g.b, ways=g.ways, T=g.sets, policy=g.policy, seed=g.seed,
                   extra=g.extra) for g in (t1[i], t2[i])]
        return oracle.hierarchy(lv, tr) + oracle.hierarchy(lt, tr)

    bad, acc = [], 0
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        for i, want in zip(idx, ex.map(want_of, idx)):
            r = runs[i]
            w0, nw = int(data.word_offsets[i]), (r.length + 31) // 32
            for k in range(4):
                got = api.unpack_bits(words[k][w0:w0 + nw].cpu().numpy().view(np.uint32),
                                      r.length)
                if not np.array_equal(got, want[k]):
                    bad.append((int(i), k))
            acc += r.length
    return {"items": len(runs), "trace_accesses": total, "ms_per_step": ms,
            "trace_accesses_per_s": total / (ms * 1e-3),
            "level_accesses_per_s": (2 * total + miss[0] + miss[2]) / (ms * 1e-3),
            "ms_by_level": dict(zip(("l1", "l2", "l1_tlb", "l2_tlb"), level_ms)),
            "plan_s": t_plan, "longest_trace": max(r.length for r in runs),
            "served_from": {"l1": 1.0 - miss[0] / total, "l2": (miss[0] - miss[1]) / total,
                            "memory": miss[1] / total},
            "translated_by": {"l1_tlb": 1.0 - miss[2] / total,
                              "l2_tlb": (miss[2] - miss[3]) / total,
                              "page_walk": miss[3] / total},
            "parity_ok": not bad, "parity_items_checked": len(idx),
            "parity_accesses_checked": acc, "parity_mismatches": bad[:8],
            "plans": [p.description for p in data.plans + tlb.plans]}


def learned_bench(args, dev):
    """Learned inverse: miss-rate table of every grid geometry under the
    512-point plan (simulator), training on synthetic traces, then held-out
    traces classified by the network with least-squares fallback, against
    the exhaustive least-squares matcher as judge."""
    import torch

    from paper_1509_02308_gb300 import inverse as INV

    cands = INV.candidate_table()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rates, _ = INV.rate_table(cands)
    torch.cuda.synchronize()
    t_rates = time.perf_counter() - t0
    rep_of, targets, l2c = INV.classes_from_rates(cands, rates)
    tt = torch.from_numpy(targets.astype(np.int32)).to(dev)
    l2c_t = torch.from_numpy(l2c.astype(np.int32)).to(dev)
    net = INV.LearnedInverse(max_batch=4096)
    net.init(seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = net.train(rates, tt, steps=args.inverse_steps, batch=4096, lr=2e-3,
                     log_every=max(1, args.inverse_steps // 4))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # inference in 65,536-trace chunks (fewer, fuller launches) over the trained
    # weights: a handle that shares the parameters and holds only the
    # inference buffers
    train_net = net
    net = INV.LearnedInverse(max_batch=65536, share_params=train_net, infer_only=True)
    n = args.inverse_eval
    x, _, truth = INV.LearnedInverse.synth(rates, tt, n, seed=0x5EED1004)
    truth = truth.cpu().numpy()
    # warm both paths once
    net.classify(x[:1024], l2c_t, rates, 0.9)
    INV.lsq_match(rates, x[:1024])
    out = {}
    for thr in (0.5, 0.6, 0.7, 0.8, 0.9, 0.97):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cand, nf = net.classify(x, l2c_t, rates, thr)
        torch.cuda.synchronize()
        out[thr] = (time.perf_counter() - t0, cand.cpu().numpy(), int(nf.item()))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    best, _ = INV.lsq_match(rates, x)
    torch.cuda.synchronize()
    t_lsq = time.perf_counter() - t0
    judge = rep_of[best.cpu().numpy()]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net.infer(x)
    torch.cuda.synchronize()
    t_net = time.perf_counter() - t0
    rep_exact, _, _ = INV.classes_from_rates(cands, rates, tol=0.0)
    rep_near, _, _ = INV.classes_from_rates(cands, rates, tol=0.01)
    # the exhaustive path on the same observation, simulation included: the
    # candidates x plan simulation that yields the rate table, then the
    # least-squares fit of every observation against every candidate
    t_exh = t_rates + t_lsq
    res = {"candidates": len(cands), "classes": int(len(set(rep_of.tolist()))),
           "class_tolerance": INV.CLASS_TOLERANCE,
           "classes_identical_rows": int(len(set(rep_exact.tolist()))),
           "classes_rows_within_0.01": int(len(set(rep_near.tolist()))),
           "plan_points": 512, "rate_table_s": t_rates,
           "train_samples": args.inverse_steps * 4096, "train_s": t_train,
           "train_ms_per_step": t_train / max(1, args.inverse_steps) * 1e3,
           "loss_history": hist, "eval_traces": n,
           "judge_traces_per_s": n / t_lsq,
           "exhaustive_with_simulation_traces_per_s": n / t_exh,
           "judge_accuracy_vs_truth": float((judge == rep_of[truth]).mean()),
           "judge_accuracy_identical_rows": float(
               (rep_exact[best.cpu().numpy()] == rep_exact[truth]).mean()),
           "network_only_traces_per_s": n / t_net,
           "exact_recovery": "identical_rows: the pick's miss-rate row equals the truth's at "
                             "all 512 points (the plan's identifiability classes)"}
    pick = None
    for thr, (dt, cand, nf) in out.items():
        acc = float((rep_of[cand] == rep_of[truth]).mean())
        acc_id = float((rep_exact[cand] == rep_exact[truth]).mean())
        res[f"thr{thr}"] = {"traces_per_s": n / dt, "fallback": nf,
                            "agreement_with_judge": float((rep_of[cand] == judge).mean()),
                            "accuracy_vs_truth": acc,
                            "accuracy_identical_rows": acc_id,
                            "speedup_vs_judge": (n / dt) / (n / t_lsq),
                            "speedup_vs_exhaustive_with_simulation": (n / dt) / (n / t_exh)}
        if acc_id >= 0.99 and (pick is None or n / dt > res[f"thr{pick}"]["traces_per_s"]):
            pick = thr
    res["at_99pct"] = ({"threshold": pick, "definition": "identical_rows", **res[f"thr{pick}"]}
                       if pick is not None else
                       {"threshold": None, "note": "no threshold reached 99 % on identical rows"})
    # a million held-out traces classified in one CUDA graph: the network in
    # 4096-trace chunks, then the least-squares fallback over every trace
    # below the confidence threshold, all captured once and replayed
    del x
    torch.cuda.empty_cache()
    n1 = 1 << 20
    thr1 = pick if pick is not None else 0.9
    x1, _, truth1 = INV.LearnedInverse.synth(rates, tt, n1, seed=0x5EED2004)
    net.classify(x1[:4096], l2c_t, rates, thr1)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        cand1, nf1 = net.classify(x1, l2c_t, rates, thr1)
    graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    g_ms = e0.elapsed_time(e1) / reps
    c1 = cand1.cpu().numpy()
    t1 = truth1.cpu().numpy()
    res["graph_1M"] = {"traces": n1, "threshold": thr1, "ms": g_ms,
                       "traces_per_s": n1 / (g_ms * 1e-3), "fallback": int(nf1.item()),
                       "accuracy_identical_rows": float((rep_exact[c1] == rep_exact[t1]).mean()),
                       "launch": "one CUDA graph replay (network chunks + fallback matcher)"}
    # the network alone over the same million traces (16 full 65,536-trace
    # chunks), CUDA events, after one untimed pass
    net.infer(x1)
    e0.record()
    for _ in range(reps):
        net.infer(x1)
    e1.record()
    torch.cuda.synchronize()
    n_ms = e0.elapsed_time(e1) / reps
    res["network_only_1M"] = {"traces": n1, "ms": n_ms, "traces_per_s": n1 / (n_ms * 1e-3),
                              "gflops": n1 * INVERSE_FLOP_PER_TRACE / (n_ms * 1e-3) / 1e9}
    del x1, graph
    torch.cuda.empty_cache()
    return res


# --------------------------------------------------------- reference arm
def reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_1509_02308_gb300 import workloads as W
    geoms, runs = W.config2(n_items=args.items, max_len=args.max_len)
    cores = os.cpu_count() or 1
    # the same seeded sample our arm's cpu_baseline times, every step
    idx = oracle_sample(geoms, runs, args.cpu_sample)
    per_step = len(idx)

    for _ in range(args.warmup):
        run_oracle(geoms, runs, idx[:4], cores)
    acc = 0
    dt = 0.0
    for _ in range(args.steps):
        a, t, _ = run_oracle(geoms, runs, idx, cores)
        acc += a
        dt += t
    value = acc / dt
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": WORKLOAD, "items_per_step": per_step},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"the same {per_step} seeded items of the batch every "
                                      f"step, at full length, one item per thread, per-access "
                                      f"miss flags out"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
