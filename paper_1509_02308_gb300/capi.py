"""Thin ctypes binding of include/pchase.h.

Argument marshalling only: every step runs in the CUDA library
(_build/libpchase.so).  There is no CPU fallback; if the library cannot be
loaded every call raises.  Device buffers are torch CUDA tensors; streams
default to torch's current stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpchase.so")

OK, EINVAL, ERANGE, ENOMEM, ETIMEOUT, ECUDA = range(6)
DEV_INDEX_RANGE, DEV_CHAIN_RANGE, DEV_TIMEOUT = 1, 2, 4
LRU, FIFO, RANDOM, WEIGHTED = 0, 1, 2, 3

_c_u32, _c_u64, _c_p = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p


class Geom(ctypes.Structure):
    _fields_ = [("C_bytes", _c_u32), ("line_bytes", _c_u32), ("ways", _c_u32),
                ("sets", _c_u32), ("policy", _c_u32), ("mapping", _c_u32), ("seed", _c_u64)]


class Trace(ctypes.Structure):
    _fields_ = [("idx", _c_p), ("len", _c_u64), ("warmup", _c_u64), ("n_elems", _c_u32),
                ("stride", _c_u32)]


class Pair(ctypes.Structure):
    _fields_ = [("geom", _c_u32), ("trace", _c_u32)]


class UnitInfo(ctypes.Structure):
    _fields_ = [("item", _c_u32), ("mode", _c_u32), ("parts", _c_u32), ("residue", _c_u32),
                ("first_step", _c_u32), ("end_step", _c_u32), ("flags", _c_u32),
                ("arena_bytes", _c_u32), ("state_offset", _c_u64), ("state_bytes", _c_u64),
                ("est_ns", ctypes.c_float), ("policy", _c_u32)]


UNIT_DIRECT, UNIT_TIME_PART, UNIT_GLOBAL_STATE, UNIT_UNEQUAL, UNIT_LEAD = 1, 2, 4, 8, 16


class Tune(ctypes.Structure):
    _fields_ = [("scan_max_ways", _c_u32), ("smem_budget_bytes", _c_u32),
                ("max_warps_per_cta", _c_u32), ("ctas_per_sm_cap", _c_u32),
                ("batch_max_sets", _c_u32), ("max_split", _c_u32), ("split_cost_ns", _c_u32),
                ("filtered", _c_u32), ("pool_warps", _c_u32), ("big_slots", _c_u32),
                ("kind_affinity", _c_u32), ("head_streams", _c_u32)]


assert ctypes.sizeof(Geom) == 32 and ctypes.sizeof(Trace) == 32 and ctypes.sizeof(UnitInfo) == 56

# every exported symbol of include/pchase.h with (restype, argtypes)
SIGNATURES = {
    "pchase_build": (ctypes.c_int, [_c_u32, _c_u32, _c_p, _c_u64, _c_p, _c_p, _c_p, _c_p]),
    "pchase_build_batch": (ctypes.c_int, [_c_p, _c_u32, _c_p, _c_p, _c_p]),
    "pchase_sim_plan_create": (ctypes.c_int, [_c_p, _c_u32, _c_p, _c_u32, _c_p, _c_u32, _c_p,
                                              ctypes.POINTER(_c_p)]),
    "pchase_sim_plan_destroy": (None, [_c_p]),
    "pchase_sim_plan_workspace_bytes": (ctypes.c_size_t, [_c_p]),
    "pchase_sim_plan_upload_bytes": (ctypes.c_size_t, [_c_p]),
    "pchase_sim_plan_items": (_c_u64, [_c_p]),
    "pchase_sim_plan_bitmap_words": (_c_u64, [_c_p]),
    "pchase_sim_plan_launches": (_c_u32, [_c_p]),
    "pchase_sim_plan_describe": (ctypes.c_size_t, [_c_p, ctypes.c_char_p, ctypes.c_size_t]),
    "pchase_sim_plan_units": (ctypes.c_size_t, [_c_p, _c_p, ctypes.c_size_t]),
    "pchase_sim_plan_upload": (ctypes.c_int, [_c_p, _c_p, ctypes.c_size_t, _c_p]),
    "pchase_sim_run": (ctypes.c_int, [_c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p]),
    "pchase_sim_run_profiled": (ctypes.c_int, [_c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p]),
    "cache_sim_batch": (ctypes.c_int, [_c_p, _c_u32, _c_p, _c_u32, _c_p, _c_u32, _c_p, _c_p, _c_p,
                                       _c_p, _c_p, ctypes.POINTER(ctypes.c_size_t), _c_p]),
    "pchase_classify_workspace_bytes": (ctypes.c_size_t, [_c_u32, _c_u64]),
    "pchase_classify": (ctypes.c_int, [_c_p, _c_p, _c_u32, _c_u64, _c_p, _c_p, _c_p, _c_p, _c_p]),
    "pchase_classify_noalloc": (ctypes.c_int, [_c_p, _c_p, _c_u32, _c_u64, _c_p, _c_p, _c_p, _c_p]),
    "pchase_classify_noalloc_limit_bytes": (ctypes.c_size_t, []),
    "pchase_match_run": (ctypes.c_int, [_c_p, _c_p, _c_p, _c_p, _c_u64, _c_p, _c_p, _c_p]),
    "pchase_canonical_pick": (ctypes.c_int, [_c_p, _c_p, _c_u32, _c_p, _c_p]),
    "pchase_infer_scratch_bytes": (ctypes.c_size_t, [_c_p]),
    "infer_geometry": (ctypes.c_int, [_c_p, _c_p, _c_p, _c_p, _c_u64, _c_p, _c_p, _c_p, _c_p]),
    "pchase_infer_batch_scratch_bytes": (ctypes.c_size_t, [_c_p, _c_u32]),
    "infer_geometry_batch": (ctypes.c_int, [_c_p, _c_p, _c_p, _c_u32, _c_p, _c_u64, _c_p, _c_p,
                                            _c_p, _c_p]),
    "pchase_probe_latency": (ctypes.c_int, [_c_p, _c_u32, _c_u32, _c_u32, _c_u32, ctypes.c_int,
                                            _c_p, _c_p, _c_p, _c_p, _c_p]),
    "pchase_probe_smem_bank": (ctypes.c_int, [_c_u32, _c_u32, _c_p, _c_p, _c_p]),
    "pchase_sim_run_filtered": (ctypes.c_int, [_c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p,
                                                _c_p]),
    "pchase_probe_smem_throughput": (ctypes.c_int, [_c_u32, _c_u32, _c_u32, _c_u32, _c_p, _c_p,
                                                     _c_p, _c_p]),
    "pchase_probe_global_throughput": (ctypes.c_int, [ctypes.c_int, _c_u32, _c_u32, _c_u32,
                                                      _c_u32, _c_p, _c_p, _c_u64, _c_u32,
                                                      ctypes.POINTER(ctypes.c_double), _c_p]),
    "pchase_inverse_create": (ctypes.c_int, [_c_u32, ctypes.POINTER(_c_p)]),
    "pchase_inverse_destroy": (None, [_c_p]),
    "pchase_inverse_param_count": (_c_u64, [_c_p]),
    "pchase_inverse_param_bytes": (ctypes.c_size_t, [_c_p]),
    "pchase_inverse_work_bytes": (ctypes.c_size_t, [_c_p]),
    "pchase_inverse_infer_work_bytes": (ctypes.c_size_t, [_c_p]),
    "pchase_inverse_status_offset": (ctypes.c_size_t, [_c_p]),
    "pchase_inverse_activation_offset": (ctypes.c_size_t, [_c_p, _c_u32]),
    "probe_pchase": (ctypes.c_int, [_c_p, _c_u32, _c_u32, _c_u32, _c_u32, ctypes.c_int, _c_p,
                                    _c_p, _c_p, _c_p, _c_p]),
    "probe_smem_bank": (ctypes.c_int, [_c_u32, _c_u32, _c_p, _c_p, _c_p]),
    "probe_global_throughput": (ctypes.c_int, [ctypes.c_int, _c_u32, _c_u32, _c_u32, _c_u32,
                                               _c_p, _c_p, _c_u64, _c_u32,
                                               ctypes.POINTER(ctypes.c_double), _c_p]),
    "inverse_load": (ctypes.c_int, [_c_p, ctypes.c_size_t, _c_p]),
    "inverse_free": (None, [_c_p]),
    "inverse_classify": (ctypes.c_int, [_c_p, _c_p, _c_u32, _c_p, _c_p, _c_u32, ctypes.c_float,
                                        _c_p, _c_p, _c_p, _c_p]),
    "pchase_miss_rates": (ctypes.c_int, [_c_p, _c_u32, _c_u32, _c_p, _c_p, _c_p]),
    "pchase_answer_classes_work_bytes": (ctypes.c_size_t, [_c_u32]),
    "pchase_answer_classes": (ctypes.c_int, [_c_p, _c_u32, _c_u32, ctypes.c_double, _c_p, _c_p,
                                             _c_p]),
    "pchase_inverse_param_offset": (ctypes.c_size_t, [_c_p, _c_u32]),
    "pchase_inverse_init": (ctypes.c_int, [_c_p, _c_p, _c_u64, _c_p]),
    "pchase_inverse_synth": (ctypes.c_int, [_c_p, _c_p, _c_u32, _c_u64, _c_u64, _c_u32, _c_p,
                                            _c_p, _c_p, _c_p, _c_p]),
    "pchase_inverse_train_step": (ctypes.c_int, [_c_p, _c_p, _c_p, _c_p, _c_p, _c_u32,
                                                 ctypes.c_float, _c_u32, _c_p, _c_p]),
    "pchase_inverse_infer": (ctypes.c_int, [_c_p, _c_p, _c_p, _c_p, _c_u32, _c_p, _c_p, _c_p, _c_p]),
    "pchase_lsq_work_bytes": (ctypes.c_size_t, [_c_u32]),
    "pchase_lsq_match": (ctypes.c_int, [_c_p, _c_u32, _c_p, _c_u32, _c_p, _c_p, _c_p, _c_p]),
    "pchase_inverse_classify": (ctypes.c_int, [_c_p, _c_p, _c_p, _c_p, _c_u32, _c_p, _c_p, _c_u32,
                                               ctypes.c_float, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p,
                                               _c_p, _c_p, _c_p]),
    "pchase_inverse_last_error": (ctypes.c_char_p, []),
    "pchase_last_error_string": (ctypes.c_char_p, []),
    "pchase_version": (ctypes.c_char_p, []),
    "pchase_device_sm_count": (ctypes.c_int, []),
}

_lock = threading.Lock()
_lib = None


class PchaseError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pchase status {code}: {msg}")
        self.code = code


def load(path: str | None = None) -> ctypes.CDLL:
    """Loads the CUDA library (building it first if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                from . import build as _b
                _b.build()
            L = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(rc: int):
    if rc != OK:
        raise PchaseError(rc, load().pchase_last_error_string().decode())


def ptr(t) -> int | None:
    if t is None:
        return None
    return int(t.data_ptr())


def stream_handle(stream=None) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream) or None


def geom_array(geoms) -> ctypes.Array:
    arr = (Geom * max(1, len(geoms)))()
    for i, g in enumerate(geoms):
        mapping = getattr(g, "mapping", 0) | (getattr(g, "extra", 0) << 8)
        arr[i] = Geom(g.C, g.b, g.ways, g.sets, g.policy, mapping, g.seed & 0xFFFFFFFFFFFFFFFF)
    return arr


def plan_units(h) -> list:
    """The plan's units (pchase_sim_plan_units) as a list of UnitInfo."""
    L = load()
    n = int(L.pchase_sim_plan_units(h, None, 0))
    arr = (UnitInfo * max(1, n))()
    L.pchase_sim_plan_units(h, ctypes.addressof(arr), n)
    return list(arr[:n])


def trace_array(descs) -> ctypes.Array:
    """descs: iterable of (idx_tensor_or_None, len, warmup, n_elems, stride)."""
    descs = list(descs)
    arr = (Trace * max(1, len(descs)))()
    for i, (t, L, w, n, s) in enumerate(descs):
        arr[i] = Trace(ptr(t), L, w, n, s)
    return arr


def pair_array(pairs) -> ctypes.Array:
    pairs = list(pairs)
    arr = (Pair * max(1, len(pairs)))()
    for i, (g, t) in enumerate(pairs):
        arr[i] = Pair(g, t)
    return arr


def u64_array(vals) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(vals, dtype=np.uint64))
