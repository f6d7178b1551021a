"""CPU oracle for the fine-grained P-chase method (Mei & Chu, Secs. 4-6).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and its ``--impl reference`` arm) may
import this package.  The product library under ``paper_1509_02308_gb300/``
never imports, links or runs it, and it imports nothing from there.

The arithmetic lives in ``pchase_oracle.c`` (plain, slow C compiled with gcc
-O2); this module only compiles it, loads it with ctypes and marshals numpy
arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pchase_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

LRU, FIFO, RANDOM, WEIGHTED, REPLAY = 0, 1, 2, 3, 4
OK, EINVAL, ERANGE, ENOMEM = 0, 1, 2, 3

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.or_pchase_array.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u32p]
            L.or_pchase_walk.argtypes = [_u32p, ctypes.c_uint32, ctypes.c_uint64, _u32p]
            L.or_splitmix64.argtypes = [ctypes.c_uint64]
            L.or_splitmix64.restype = ctypes.c_uint64
            L.or_random_victim.argtypes = [ctypes.c_uint64, ctypes.c_uint32,
                                           ctypes.c_uint64, ctypes.c_uint32]
            L.or_random_victim.restype = ctypes.c_uint32
            L.or_cache_sim.argtypes = [ctypes.c_uint32] * 4 + [
                ctypes.c_int, ctypes.c_uint64, _u32p, ctypes.c_uint64,
                ctypes.c_void_p, ctypes.c_uint64, _u8p, ctypes.c_void_p]
            L.or_cache_sim_ext.argtypes = [ctypes.c_uint32] * 4 + [
                ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, _u32p, ctypes.c_uint64,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, _u8p, ctypes.c_void_p,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                ctypes.POINTER(ctypes.c_uint64)]
            L.or_weighted_victim.argtypes = [ctypes.c_uint64, ctypes.c_uint32,
                                             ctypes.c_uint64, ctypes.c_uint32]
            L.or_weighted_victim.restype = ctypes.c_uint32
            L.or_cache_sim_uneq.argtypes = [ctypes.c_uint32] * 5 + [
                ctypes.c_int, _u32p, ctypes.c_uint64, ctypes.c_void_p, _u8p]
            L.or_cache_sim_counts.argtypes = [ctypes.c_uint32] * 4 + [
                ctypes.c_int, ctypes.c_uint64, _u32p, ctypes.c_uint64, ctypes.c_uint64,
                ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
            L.or_classify.argtypes = [_f32p, ctypes.c_uint64, _u8p,
                                      ctypes.POINTER(ctypes.c_float)]
            L.or_match.argtypes = [_u32p, _u64p, ctypes.c_uint32, _u32p, _u64p,
                                   ctypes.c_uint32, _u8p, _u64p]
            L.or_canonical_pick.argtypes = [_u32p, _u64p, ctypes.c_uint32,
                                            ctypes.POINTER(ctypes.c_uint32)]
            L.or_canonical_pick.restype = ctypes.c_uint32
            L.or_bank_degree.argtypes = [_u32p, ctypes.c_uint32, ctypes.c_uint32]
            L.or_bank_degree.restype = ctypes.c_uint32
            L.or_mean_latency.argtypes = [ctypes.c_double] * 3
            L.or_mean_latency.restype = ctypes.c_double
            _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != OK:
        raise OracleError(f"{what}: oracle status {rc}")


# --------------------------------------------------------------------- P-chase
def pchase_array(n_elems: int, stride_elems: int) -> np.ndarray:
    """Listing 1: A[i] = (i + stride) mod N."""
    A = np.empty(n_elems, dtype=np.uint32)
    _check(lib().or_pchase_array(n_elems, stride_elems, A), "pchase_array")
    return A


def pchase_walk(A: np.ndarray, length: int) -> np.ndarray:
    """Indices visited by j = A[j] from j = 0 (Listings 2-3)."""
    A = np.ascontiguousarray(A, dtype=np.uint32)
    out = np.empty(length, dtype=np.uint32)
    _check(lib().or_pchase_walk(A, A.size, length, out), "pchase_walk")
    return out


def pchase_trace(n_elems: int, stride_elems: int, length: int) -> np.ndarray:
    return pchase_walk(pchase_array(n_elems, stride_elems), length)


def splitmix64(x: int) -> int:
    return int(lib().or_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def random_victim(seed: int, set_: int, k: int, ways: int) -> int:
    return int(lib().or_random_victim(seed & 0xFFFFFFFFFFFFFFFF, set_, k, ways))


def weighted_victim(seed: int, set_: int, k: int, ways: int) -> int:
    return int(lib().or_weighted_victim(seed & 0xFFFFFFFFFFFFFFFF, set_, k, ways))


# ----------------------------------------------------------------------- cache
def cache_sim(C: int, b: int, ways: int, T: int, policy: int, trace: np.ndarray,
              seed: int = 0, victims=None, want_final: bool = False, mapping: int = 0,
              want_evictions: bool = False, filter=None):
    """Per-access miss flags (uint8, 1 = miss) of one replay; see or_cache_sim_ext.

    filter: per-access flags; the cache sees only the flagged accesses (a lower
    level of the hierarchy fed by the misses of the level above).
    want_final adds the line held by each way (T*ways, 0xFFFFFFFF when invalid);
    want_evictions adds (sets, ways) of every eviction in order."""
    trace = np.ascontiguousarray(trace, dtype=np.uint32)
    flt = None
    if filter is not None:
        flt = np.ascontiguousarray(filter, dtype=np.uint8)
        if flt.size != trace.size:
            raise ValueError("filter must flag every access")
    out = np.empty(trace.size, dtype=np.uint8)
    vic_p, nv = None, 0
    if victims is not None:
        vic = np.ascontiguousarray(victims, dtype=np.uint32)
        vic_p, nv = vic.ctypes.data, vic.size
    fin = np.empty(T * ways, dtype=np.uint32) if want_final else None
    cap = trace.size if want_evictions else 0
    es = np.empty(max(cap, 1), dtype=np.uint32)
    ew = np.empty(max(cap, 1), dtype=np.uint32)
    n_ev = ctypes.c_uint64()
    rc = lib().or_cache_sim_ext(C, b, ways, T, policy, seed & 0xFFFFFFFFFFFFFFFF, mapping,
                                trace, trace.size, flt.ctypes.data if flt is not None else None,
                                vic_p, nv, out,
                                fin.ctypes.data if fin is not None else None,
                                es.ctypes.data if cap else None,
                                ew.ctypes.data if cap else None, cap, ctypes.byref(n_ev))
    _check(rc, "cache_sim")
    res = [out]
    if want_final:
        res.append(fin)
    if want_evictions:
        n = int(n_ev.value)
        res += [es[:n].copy(), ew[:n].copy()]
    return tuple(res) if len(res) > 1 else out


def cache_sim_uneq(C: int, b: int, ways: int, T: int, extra: int, policy: int,
                   trace: np.ndarray, filter=None) -> np.ndarray:
    """Per-access miss flags of a cache whose set 0 has `extra` more ways
    (the unequal-set L2 TLB of Sec. 4.4); see or_cache_sim_uneq.  filter as
    in cache_sim."""
    trace = np.ascontiguousarray(trace, dtype=np.uint32)
    flt = None
    if filter is not None:
        flt = np.ascontiguousarray(filter, dtype=np.uint8)
        if flt.size != trace.size:
            raise ValueError("filter must flag every access")
    out = np.empty(trace.size, dtype=np.uint8)
    _check(lib().or_cache_sim_uneq(C, b, ways, T, extra, policy, trace, trace.size,
                                   flt.ctypes.data if flt is not None else None, out),
           "cache_sim_uneq")
    return out


def hierarchy(levels, trace):
    """Miss flags of each level of a cascade: levels[0] sees every access,
    levels[k] only the misses of levels[k-1] (Sec. 3's L1 -> L2 path; with
    page-sized lines, an L1 TLB -> L2 TLB path).  levels: dicts with C, b,
    ways, T, policy and optionally seed, mapping, extra (unequal sets, see
    cache_sim_uneq).  The level an access is served from is the sum of its
    flags."""
    out, flt = [], None
    for g in levels:
        if g.get("extra", 0):
            m = cache_sim_uneq(g["C"], g["b"], g["ways"], g["T"], g["extra"], g["policy"],
                               trace, filter=flt)
        else:
            m = cache_sim(g["C"], g["b"], g["ways"], g["T"], g["policy"], trace,
                          seed=g.get("seed", 0), mapping=g.get("mapping", 0), filter=flt)
        out.append(m)
        flt = m
    return out


def cache_sim_counts(C, b, ways, T, policy, trace, warmup, seed=0):
    trace = np.ascontiguousarray(trace, dtype=np.uint32)
    tot, aft = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().or_cache_sim_counts(C, b, ways, T, policy, seed & 0xFFFFFFFFFFFFFFFF,
                                     trace, trace.size, warmup,
                                     ctypes.byref(tot), ctypes.byref(aft)),
           "cache_sim_counts")
    return tot.value, aft.value


def classify(lat: np.ndarray):
    """Largest-gap two-level split; returns (miss flags uint8, threshold)."""
    lat = np.ascontiguousarray(lat, dtype=np.float32)
    out = np.empty(lat.size, dtype=np.uint8)
    thr = ctypes.c_float()
    _check(lib().or_classify(lat, lat.size, out, ctypes.byref(thr)), "classify")
    return out, thr.value


def match(cands: np.ndarray, seeds: np.ndarray, traces: list, observed: list) -> np.ndarray:
    """Hamming distance of every candidate over all plan traces (or_match).

    cands: (G, 5) uint32 rows {C, b, ways, T, policy}; traces / observed: lists
    of per-trace arrays (uint32 indices / uint8 miss flags)."""
    cands = np.ascontiguousarray(cands, dtype=np.uint32).reshape(-1, 5)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    lens = np.array([len(t) for t in traces], dtype=np.uint64)
    offsets = np.zeros(len(traces) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(lens)
    tr = np.ascontiguousarray(np.concatenate(traces) if traces else np.zeros(0), dtype=np.uint32)
    ob = np.ascontiguousarray(np.concatenate(observed) if observed else np.zeros(0), dtype=np.uint8)
    dist = np.zeros(cands.shape[0], dtype=np.uint64)
    _check(lib().or_match(cands, seeds, cands.shape[0], tr, offsets, len(traces), ob, dist),
           "match")
    return dist


def canonical_pick(cands: np.ndarray, dist: np.ndarray):
    """(index of the canonical pick, number of candidates at the best distance)."""
    cands = np.ascontiguousarray(cands, dtype=np.uint32).reshape(-1, 5)
    dist = np.ascontiguousarray(dist, dtype=np.uint64)
    nb = ctypes.c_uint32()
    i = lib().or_canonical_pick(cands, dist, cands.shape[0], ctypes.byref(nb))
    return int(i), int(nb.value)


def bank_degree(word_addr, n_banks: int = 32) -> int:
    w = np.ascontiguousarray(word_addr, dtype=np.uint32)
    return int(lib().or_bank_degree(w, w.size, n_banks))


def mean_latency(t0: float, tm: float, r: float) -> float:
    return float(lib().or_mean_latency(t0, tm, r))
