"""Seeded synthetic inputs: cache geometries and P-chase run descriptors.

This module only draws descriptors (which geometry, which array size, stride
and length); it holds none of the method's arithmetic: no trace is walked and
no cache is simulated here.  Both the CUDA path and the CPU oracle take their
inputs from it.  It imports numpy only.

Random draws use SplitMix64 streams (Steele, Lea & Flood, OOPSLA 2014): the
stream seeded with x yields mix(x + k*gamma) for k = 1, 2, ...
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

LRU, FIFO, RANDOM, WEIGHTED = 0, 1, 2, 3
POLICY_NAMES = ("LRU", "FIFO", "RANDOM")
_M64 = 0xFFFFFFFFFFFFFFFF
_GAMMA = 0x9E3779B97F4A7C15


class SplitMix64:
    """SplitMix64 stream (published definition), for drawing inputs only."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next(self) -> int:
        self.state = (self.state + _GAMMA) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Integer in [0, n) from the high 32 bits (multiply-shift)."""
        return ((self.next() >> 32) * n) >> 32

    def unit(self) -> float:
        """Float in [0, 1) from the high 53 bits."""
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)


@dataclass(frozen=True)
class Geom:
    """Cache geometry: capacity C and line size b in bytes, ways a, sets T."""
    C: int
    b: int
    ways: int
    sets: int
    policy: int = LRU
    seed: int = 0
    mapping: int = 0  # set = (line >> mapping) mod T
    # unequal sets (the L2 TLB of Sec. 4.4): set 0 has `extra` more ways and
    # C = (T * ways + extra) * b; line residues mod T*ways + extra below
    # T*ways go to set residue mod T, the others to set 0
    extra: int = 0

    def row(self):
        return (self.C, self.b, self.ways, self.sets, self.policy)


@dataclass(frozen=True)
class Run:
    """One P-chase run: array of n_elems 4-byte elements, stride in elements,
    `length` accesses of which the first `warmup` form the warm-up pass.
    `chain` (optional) is a caller-built next-index array that replaces the
    uniform stride (a non-uniform chain in the style of Fig. 10)."""
    n_elems: int
    stride: int
    length: int
    warmup: int
    chain: np.ndarray | None = None


# ----------------------------------------------------------------- geometries
CAPACITIES = sorted([1 << k for k in range(10, 19)] + [3 << k for k in range(9, 17)])
LINE_SIZES = (32, 64, 128, 256)
WAY_CHOICES = (1, 2, 4, 8, 16, 32, 0)  # 0 = fully associative (ways = C / b)


def geometry_grid(capacities=CAPACITIES, line_sizes=LINE_SIZES, way_choices=WAY_CHOICES):
    """Every (C, b, ways, T) with ways * b dividing C, without duplicates.

    Capacities {2^k, 3*2^k} in [1 KB, 256 KB], b in {32..256} B, ways in
    {1..32, full}."""
    out = []
    seen = set()
    for C in capacities:
        for b in line_sizes:
            if C % b:
                continue
            lines = C // b
            for w in way_choices:
                a = lines if w == 0 else w
                if a > lines or lines % a:
                    continue
                key = (C, b, a)
                if key in seen:
                    continue
                seen.add(key)
                out.append((C, b, a, lines // a))
    return out


# The cache geometries of Table 4 (Secs. 4.3-4.5) beyond the grid, as matcher
# candidates: the texture L1 caches (12 KB on Fermi/Kepler, 24 KB on Maxwell;
# 32 B lines, 4 sets, so 96 and 192 ways) under the standard mapping and under
# the bits 7-8 mapping Sec. 4.3 measured, and the Fermi L1 data cache (16 KB,
# 128 B, 32 sets, in the grid) under its measured non-LRU policy.
TABLE4_EXTRA = ((12288, 32, 96, 4), (24576, 32, 192, 4))


def table4_candidates(seed_base: int = 0x7AB1E4):
    out = []
    for C, b, a, T in TABLE4_EXTRA:
        for m in (0, 2):
            for p in (LRU, FIFO, RANDOM):
                out.append(Geom(C, b, a, T, p, seed_base + len(out), mapping=m))
    out.append(Geom(16384, 128, 4, 32, WEIGHTED, seed_base + len(out)))
    return out


def matcher_candidates(seed_base: int = 0x5EED):
    """The exhaustive matcher's candidates: every grid geometry under LRU,
    FIFO and RANDOM, then the Table 4 geometries outside the grid."""
    grid = [Geom(C, b, a, T, p, seed_base + i)
            for i, (C, b, a, T) in enumerate(geometry_grid()) for p in (LRU, FIFO, RANDOM)]
    return grid + table4_candidates()


def capacity_sweep(capacities=None):
    """Stage 1 of Fig. 6 (Sec. 4.2): s = 1 element over array sizes N equal to
    each candidate capacity, one warm-up pass and two more; the capacity is
    the largest N whose passes after the first all hit."""
    caps = sorted(set(capacities or (list(CAPACITIES) + [g[0] for g in TABLE4_EXTRA])))
    return caps, [Run(c // 4, 1, 3 * (c // 4), c // 4) for c in caps]


def two_stage_plan(C: int, with_retouch: bool = True):
    """Stage 2 of Fig. 6 (Sec. 4.2) for a cache whose capacity stage 1 found
    to be C bytes, as (Run, explicit trace or None) pairs:
      - s = 1 element, N = C + 4j bytes: the misses per pass jump once N
        passes C + b (the line size);
      - s = 32 B (the smallest line size), N = C + 32k bytes: each step makes
        one more set overflow (the number of sets, and the set mapping);
      - Fig. 10-style hot re-touch chains, streams of 32 B steps over C + 256 B,
        1.5C and 2C bytes: every set then receives more lines than it has
        ways, so a hot line touched every other access stays under LRU and
        is evicted in turn under FIFO (the policy, step 4).
    Each uniform run is one warm-up pass and two more."""
    pts = []
    for j in (1, 7, 8, 9, 15, 16, 17, 31, 32, 33, 63, 64, 65):
        n = (C + 4 * j) // 4
        pts.append((Run(n, 1, 3 * n, n), None))
    for k in (1, 2, 3, 4, 5, 6, 8, 12, 16, 24, 32, 48, 64, 128):
        n = (C + 32 * k) // 4
        per = n // math.gcd(n, 8)
        pts.append((Run(n, 8, 3 * per, per), None))
    if with_retouch:
        for nb in (C + 256, 3 * C // 2, 2 * C):
            tr = hot_retouch_trace(nb, stream_stride=32)
            pts.append((Run(int(tr.max()) + 1, 1, tr.size, tr.size // 2), tr))
    return pts


# ------------------------------------------------------------------- config 1
def config1():
    """One LRU cache (16 KB, 128 B lines, 4 ways, 32 sets); arrays of 12 KB to
    24 KB in 128 B steps, stride 128 B, one warm-up pass plus two passes."""
    g = Geom(16384, 128, 4, 32, LRU, 0)
    runs = []
    for nbytes in range(12288, 24576 + 1, 128):
        n = nbytes // 4
        s = 128 // 4
        per_pass = n // s
        runs.append(Run(n, s, 3 * per_pass, per_pass))
    return g, runs


# ------------------------------------------------------------------- config 2
def config2(n_items: int = 4096, seed_base: int = 0x5EED0002,
            min_len: int = 1024, max_len: int = 1 << 20):
    """Batched-simulation workload: item i is one geometry and one uniform run.

    Stream i (seed seed_base + i) draws, in order: a geometry uniformly from
    geometry_grid(); a policy from {LRU, FIFO, RANDOM}; a policy seed; a stride
    of 4 * 2^u bytes, u uniform on {0..10}; v uniform on [-1, 1) giving the
    array size round_down(C * 2^v, stride) (at least one stride); and a length
    L = floor(min_len * (max_len / min_len)^x), x uniform on [0, 1).  The
    warm-up is the first pass (array size / stride accesses, at most L)."""
    grid = geometry_grid()
    geoms, runs = [], []
    for i in range(n_items):
        r = SplitMix64(seed_base + i)
        C, b, a, T = grid[r.below(len(grid))]
        policy = r.below(3)
        pseed = r.next()
        sbytes = 4 << r.below(11)
        v = 2.0 * r.unit() - 1.0
        nbytes = int(C * (2.0 ** v)) // sbytes * sbytes
        nbytes = max(nbytes, sbytes)
        L = int(min_len * (max_len / min_len) ** r.unit())
        L = max(min_len, min(L, max_len))
        n, s = nbytes // 4, sbytes // 4
        per_pass = n // s
        geoms.append(Geom(C, b, a, T, policy, pseed))
        runs.append(Run(n, s, L, min(per_pass, L)))
    return geoms, runs


def random_small_geoms(n: int, seed: int, max_lines: int = 64,
                       line_sizes=(4, 8, 16, 32, 64), policies=(LRU, FIFO, RANDOM)):
    """Small geometries with arbitrary T (including T not a power of two)."""
    r = SplitMix64(seed)
    out = []
    while len(out) < n:
        b = line_sizes[r.below(len(line_sizes))]
        lines = 1 + r.below(max_lines)
        divs = [d for d in range(1, lines + 1) if lines % d == 0]
        a = divs[r.below(len(divs))]
        T = lines // a
        out.append(Geom(lines * b, b, a, T, policies[r.below(len(policies))], r.next()))
    return out


def random_index_trace(n: int, n_elems: int, seed: int, hot: int = 0) -> np.ndarray:
    """A general (non-chain) index trace: uniform indices below n_elems, with
    an optional fraction hot/16 of accesses drawn from the first 64 elements."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = rng.integers(0, n_elems, size=n, dtype=np.uint64).astype(np.uint32)
    if hot:
        m = rng.integers(0, 16, size=n) < hot
        t[m] = rng.integers(0, min(64, n_elems), size=int(m.sum()), dtype=np.uint64).astype(np.uint32)
    return t


def total_accesses(runs) -> int:
    return int(sum(r.length for r in runs))


def describe_config2(geoms, runs) -> dict:
    L = np.array([r.length for r in runs], dtype=np.float64)
    return {
        "items": len(runs),
        "accesses": int(L.sum()),
        "mean_len": float(L.mean()),
        "max_len": int(L.max()),
        "policies": [int(sum(g.policy == p for g in geoms)) for p in range(3)],
        "fully_assoc": int(sum(g.sets == 1 for g in geoms)),
    }


def log2i(x: int) -> int:
    return int(math.log2(x))


# ------------------------------------------------------- learned inverse (S7)
PLAN_POINTS = 512
WAY_LABELS = (1, 2, 4, 8, 16, 32)  # label 6: any other associativity (full)


def geometry_label(g) -> tuple:
    """(capacity index, line-size index, ways index, policy) of a grid geometry."""
    ci = CAPACITIES.index(g.C)
    bi = LINE_SIZES.index(g.b)
    wi = WAY_LABELS.index(g.ways) if g.ways in WAY_LABELS else 6
    return ci, bi, wi, g.policy


def _logspace_bytes(lo: int, hi: int, n: int, mult: int):
    out = []
    for k in range(n):
        v = lo * (hi / lo) ** (k / (n - 1))
        out.append(max(mult, int(round(v / mult)) * mult))
    return out


def hot_retouch_trace(n_bytes: int, stream_stride: int = 64, words: int = 8,
                      max_len: int = 1 << 15) -> np.ndarray:
    """Accesses alternate between a hot 32-byte line (its `words` words in
    turn, as a chain through distinct elements would) and a uniform stream
    over [stream_stride, n_bytes), in the style of the non-uniform chains of
    Fig. 10.  Returns element indices, two passes of the stream or max_len."""
    stream = np.arange(stream_stride, n_bytes, stream_stride, dtype=np.int64) // 4
    if stream.size == 0:
        stream = np.array([stream_stride // 4], dtype=np.int64)
    L = min(max_len, 4 * stream.size)
    k = np.arange(L)
    hot = (k // 2) % words
    st = stream[(k // 2) % stream.size]
    return np.where(k % 2 == 0, hot, st).astype(np.uint32)


def hot_stream_trace(span: int, step: int, stream_bytes: int = 1 << 20,
                     max_len: int = 1 << 15, warm_periods: int = 4):
    """A non-uniform chain in the style of Fig. 10 that tells LRU from FIFO:
    every period walks a hot region of span/2 bytes, then the next span/2
    bytes of a 1 MB stream region that follows it (both in `step`-byte steps,
    the stream wrapping around).  When the period's lines fit in a set's ways
    (span <= C at step <= b), LRU keeps the hot lines and misses only the
    stream, while FIFO evicts each hot line once its set has taken `ways`
    misses since it came in, so a quarter or so of the hot accesses miss.
    Returns (element indices, warm-up accesses): warm_periods periods of
    warm-up, then periods up to max_len measured accesses."""
    H = max(step, (span // 2) // step * step)
    hot = np.arange(0, H, step, dtype=np.int64) // 4
    per = len(hot)
    n_stream = stream_bytes // step
    periods = warm_periods + max(1, -(-max_len // (2 * per)))
    out = []
    for p in range(periods):
        k = (p * per + np.arange(per)) % n_stream
        out.append(hot)
        out.append((H + k * step) // 4)
    return np.concatenate(out).astype(np.uint32), warm_periods * 2 * per


def p512_plan():
    """The 512-point plan of the learned inverse: list of (Run, explicit
    trace or None).  Points: 176 with s = 4 B and 176 with s = 32 B over array
    sizes log-spaced from 512 B to 512 KB; 61 with s = 128 B over 1-512 KB;
    35 Saavedra stride sweeps (N = 512 KB and 1 MB, s = 4 B * 2^j); 64
    hot/stream chains (hot_stream_trace) over spans log-spaced from 1 KB to
    256 KB, 32 in 32-byte steps and 32 in 256-byte steps.  Each uniform point
    runs one warm-up pass (at most 2^17 accesses) and then at most 2^15
    measured accesses."""
    pts = []

    def uni(nb, sb):
        n, s = nb // 4, sb // 4
        per = n // math.gcd(n, s)
        warm = min(per, 1 << 17)
        meas = min(per, 1 << 15)
        pts.append((Run(n, s, warm + meas, warm), None))

    for nb in _logspace_bytes(512, 512 << 10, 176, 4):
        uni(nb, 4)
    for nb in _logspace_bytes(512, 512 << 10, 176, 32):
        uni(nb, 32)
    for nb in _logspace_bytes(1024, 512 << 10, 61, 128):
        uni(nb, 128)
    for nb, jmax in ((512 << 10, 17), (1 << 20, 18)):
        for j in range(jmax):
            uni(nb, 4 << j)
    for step in (32, 256):
        for span in _logspace_bytes(1024, 256 << 10, 32, step):
            tr, warm = hot_stream_trace(span, step)
            pts.append((Run(int(tr.max()) + 1, 1, tr.size, warm), tr))
    assert len(pts) == PLAN_POINTS, len(pts)
    return pts


def latency_noise_params():
    """Synthetic timing model of the learned-inverse traces (seeded on the
    device): per trace t0 ~ U[20, 400] cycles and t1 = t0 * rho with
    log(rho) ~ U[log 1.5, log 30] (within the span of Fig. 11's latency spectrum);
    per point latency t0 + (t1 - t0) * r, Gaussian relative jitter sigma
    2 %, spikes on 0.5 % of points scaled by U[2, 10]; then min-max
    normalisation to [0, 1]."""
    return {"t0_lo": 20.0, "t0_hi": 400.0, "rho_lo": 1.5, "rho_hi": 30.0, "sigma": 0.02,
            "spike_p": 0.005, "spike_lo": 2.0, "spike_hi": 10.0}


# ------------------------------------------------------------- hierarchies
def hierarchy_config(n_items: int = 1024, seed_base: int = 0x5EED0005):
    """Two-level cache and two-level TLB hierarchies over P-chase streams (a
    scaled-down mixed-hierarchy batch: L2 caches up to 3 MB, the most lines
    one simulated geometry holds).  Item i draws from stream seed_base + i:
      L1: C 16-256 KB (powers of two), b 32/64/128 B, 4/8/16 ways, a policy;
      L2: C 0.5/1/2/3 MB, b 64/128 B, 8/16/32 ways, a policy;
      TLBs (Sec. 4.4): a 16-entry fully associative L1 TLB and an 8-way L2 TLB
      of 8-64 sets, both LRU, over 4 KB or 64 KB pages; over 2 MB pages the
      L2 TLB the paper measures (Fig. 9): one set of 17 entries and six of 8;
      stream: s = 4 * 2^u B (u in 0..10), N = round_down(C_L2 * 2^v, s),
      v in [-1, 1), length 16K * 32^x (x in [0, 1)), warm-up one pass.
    Returns (l1, l2, tlb1, tlb2, runs), item i pairing entry i of each."""
    l1, l2, t1, t2, runs = [], [], [], [], []
    for i in range(n_items):
        r = SplitMix64(seed_base + i)
        a1 = 4 << r.below(3)
        b1 = 32 << r.below(3)
        C1 = (16 << 10) << r.below(5)
        l1.append(Geom(C1, b1, a1, C1 // (a1 * b1), r.below(3), r.next()))
        C2 = (512 << 10, 1 << 20, 2 << 20, 3 << 20)[r.below(4)]
        b2 = 64 << r.below(2)
        a2 = 8 << r.below(3)
        l2.append(Geom(C2, b2, a2, C2 // (a2 * b2), r.below(3), r.next()))
        page = (4096, 65536, 2 << 20)[r.below(3)]
        sets2 = 8 << r.below(4)
        t1.append(Geom(16 * page, page, 16, 1, LRU))
        if page == 2 << 20:
            t2.append(Geom(65 * page, page, 8, 7, LRU, extra=9))
        else:
            t2.append(Geom(sets2 * 8 * page, page, 8, sets2, LRU))
        s_elems = 1 << r.below(11)
        v = r.unit() * 2.0 - 1.0
        n = max(s_elems, int(C2 * 2.0 ** v) // 4 // s_elems * s_elems)
        L = int(16384 * 32.0 ** r.unit())
        per = n // math.gcd(n, s_elems)
        runs.append(Run(n, s_elems, L, min(per, L)))
    return l1, l2, t1, t2, runs


def mixed_config(n_items: int = 65536, seed_base: int = 0x5EED0015):
    """The large mixed batch: two-level cache and two-level TLB hierarchies
    over P-chase streams of uneven length.  Item i draws from stream
    seed_base + i:
      L1: C 16-256 KB (powers of two), b 32/64/128 B, 4/8/16 ways, a policy;
      L2: C 1-128 MB (powers of two), b 64/128 B, 8/16/32 ways, a policy;
      TLBs (Sec. 4.4): a 16-entry fully associative L1 TLB and an 8-way L2 TLB
      of 8-64 sets, both LRU, over 4 KB or 64 KB pages; over 2 MB pages the
      L2 TLB the paper measures (Fig. 9): one set of 17 entries and six of 8;
      stream: s = 4 * 2^u B (u in 0..10), N = round_down(C_L2 * 2^v, s),
      v in [-1, 1), warm-up one pass;
      length 4096 * 4096^(x^4) accesses (x in [0, 1)): 4K to 16M, most short,
      a long tail (about 0.57M on average).
    Returns (l1, l2, tlb1, tlb2, runs), item i pairing entry i of each."""
    l1, l2, t1, t2, runs = [], [], [], [], []
    for i in range(n_items):
        r = SplitMix64(seed_base + i)
        a1 = 4 << r.below(3)
        b1 = 32 << r.below(3)
        C1 = (16 << 10) << r.below(5)
        l1.append(Geom(C1, b1, a1, C1 // (a1 * b1), r.below(3), r.next()))
        C2 = (1 << 20) << r.below(8)
        b2 = 64 << r.below(2)
        a2 = 8 << r.below(3)
        l2.append(Geom(C2, b2, a2, C2 // (a2 * b2), r.below(3), r.next()))
        page = (4096, 65536, 2 << 20)[r.below(3)]
        sets2 = 8 << r.below(4)
        t1.append(Geom(16 * page, page, 16, 1, LRU))
        if page == 2 << 20:
            t2.append(Geom(65 * page, page, 8, 7, LRU, extra=9))
        else:
            t2.append(Geom(sets2 * 8 * page, page, 8, sets2, LRU))
        s_elems = 1 << r.below(11)
        v = r.unit() * 2.0 - 1.0
        n = max(s_elems, int(C2 * 2.0 ** v) // 4 // s_elems * s_elems)
        L = int(4096 * 4096.0 ** (r.unit() ** 4))
        per = n // math.gcd(n, s_elems)
        runs.append(Run(n, s_elems, L, min(per, L)))
    return l1, l2, t1, t2, runs


# --------------------------------------------------------- latency spectrum
def spectrum_chain():
    """The non-uniform-stride chain of Sec. 5.2 (Fig. 10(b)), as element
    indices visited in order, with a segment label per access, over an array
    of `n_elems` 4-byte elements (2.3 GB):

      B  65 accesses 1 MB apart (cold: data-cache misses; each new 2 MB page
         comes on an even access, the odd ones reuse the page of the previous);
      A  64 accesses 32 MB apart over 2 GB (cache misses on new pages);
      C  B's 65 lines again through their next element (a chase visits each
         element once), 32 lines apart in turn (data cached, pages last
         touched before A's sweep);
      D  32 accesses to the 32 elements of one 128-byte line (hits).

    No element repeats, so a chain A[path[i]] = path[i + 1] closing on itself
    walks exactly this path.  Returns (path, labels, n_elems)."""
    MB = (1 << 20) // 4
    base_b = 2048 * MB + 64 * MB
    b_lines = [base_b + k * MB for k in range(65)]
    a_lines = [k * 32 * MB + 16 for k in range(64)]
    c_order = [(k * 32) % 65 for k in range(65)]
    c_lines = [b_lines[k] + 1 for k in c_order]
    d_base = base_b + 70 * MB
    d_lines = [d_base + k for k in range(32)]
    path = b_lines + a_lines + c_lines + d_lines
    labels = (["B_new_page" if k % 2 == 0 else "B_same_page" for k in range(65)] +
              ["A_32MB"] * 64 + ["C_revisit"] * 65 + ["D_same_line"] * 32)
    n_elems = d_base + 64
    return path, labels, n_elems
