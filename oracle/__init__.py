"""Oracle: plain CPU definitions of what the kNN / FoF hot path computes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA path (``paper_2604_05885_gb300``) and never imports it.

Contents, each following the paper (jz-tree, Stuecker et al.):

* Results (the method is exact, so these are the plain definitions):
  - ``knn_brute`` / ``knn_cells``  -- k nearest neighbours, self included, ties by
    lower index; float64 distances (Sec. III).
  - ``fof_brute`` / ``fof_cells``  -- FoF groups at linking length b, labelled by
    the smallest index in each group (Sec. IV, R_link and linking rule).
* Tree (Sec. II, the plane-based hierarchy), bit-exact integer definitions:
  - ``morton_keys``   -- 3 x 21-bit interleaved keys (Sec. II-A: integer Morton key;
    x is the most significant coordinate, as in the z-order comparator).
  - ``zsort``         -- stable sort by key.
  - ``zorder_msb`` / ``zorder_less`` / ``zorder_sort`` / ``zorder_level`` -- the
    full-precision float comparator of Sec. II-A (Eq. msb, EMAX = 128 for float32;
    -0 read as +0) and the node level of Sec. II-C (Eq. lvl) on top of it;
    ``zorder_gap_levels`` / ``zorder_node_sizes_brute`` -- lvl_i and n_i of Sec. II-C
    on that order, which ``plane_splits_from_sizes`` turns into tree-planes.
  - ``gap_levels``    -- lvl_i between sorted neighbours i-1, i (Sec. II-C, eq. lvl_i),
    with the sentinel gaps at 0 and N.
  - ``node_sizes``    -- n_i, the size of the smallest node holding i-1 and i
    (Sec. II-C, l_b / r_b search).
  - ``plane_splits``  -- spl^(p): splits with n > N_max^(p) (Sec. II-C, tree-planes,
    N_max^(p) = N_max^(0) c^p, coarsening stops below N_target).
  - ``plane_nodes``   -- per-node point counts and bounding boxes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jzt_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP) into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        f32p = ctypes.POINTER(ctypes.c_float)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.oracle_knn_brute.argtypes = [f32p, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                         i64p, ctypes.c_int64, i32p, f64p, ctypes.c_int]
        lib.oracle_knn_cells.argtypes = lib.oracle_knn_brute.argtypes
        lib.oracle_knn_brute_sets.argtypes = [f32p, ctypes.c_int64, f32p, ctypes.c_int64, ctypes.c_int,
                                              ctypes.c_double, i32p, f64p, ctypes.c_int]
        lib.oracle_fof_brute.argtypes = [f32p, ctypes.c_int64, ctypes.c_double, ctypes.c_double, i32p]
        lib.oracle_fof_cells.argtypes = [f32p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, i32p, ctypes.c_int]
        lib.oracle_fof_cells2.argtypes = [f32p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, i32p, i32p, ctypes.c_int]
        lib.oracle_num_threads.argtypes = [ctypes.c_int]
        for f in (lib.oracle_knn_brute, lib.oracle_knn_cells, lib.oracle_fof_brute,
                  lib.oracle_fof_cells, lib.oracle_fof_cells2, lib.oracle_num_threads):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t)) if a is not None else None


def num_threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count the oracle uses."""
    return _load().oracle_num_threads(int(n))


# ------------------------------------------------------------------ kNN

def _knn(fn, xyz, k, periodic_L, queries, threads):
    x = np.ascontiguousarray(xyz, dtype=np.float32)
    n = x.shape[0]
    q = None if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    nq = n if q is None else q.shape[0]
    idx = np.empty((nq, k), dtype=np.int32)
    d2 = np.empty((nq, k), dtype=np.float64)
    rc = fn(_ptr(x, ctypes.c_float), n, int(k), float(periodic_L), _ptr(q, ctypes.c_int64), nq,
            _ptr(idx, ctypes.c_int32), _ptr(d2, ctypes.c_double), int(threads))
    if rc != 0:
        raise ValueError(f"oracle kNN failed (rc={rc})")
    return idx, d2


def knn_brute(xyz, k, periodic_L=0.0, queries=None, threads=0):
    """All-pairs exact kNN (Sec. III): rows ascending by (float64 d2, index), self included."""
    return _knn(_load().oracle_knn_brute, xyz, k, periodic_L, queries, threads)


def knn_brute_sets(src, qry, k, periodic_L=0.0, threads=0):
    """kNN of separate query points among source points (Sec. II-G): row r lists the
    k sources nearest to query r, ascending by (float64 d2, source index)."""
    s = np.ascontiguousarray(src, dtype=np.float32)
    q = np.ascontiguousarray(qry, dtype=np.float32)
    idx = np.empty((q.shape[0], k), dtype=np.int32)
    d2 = np.empty((q.shape[0], k), dtype=np.float64)
    rc = _load().oracle_knn_brute_sets(_ptr(s, ctypes.c_float), s.shape[0], _ptr(q, ctypes.c_float), q.shape[0],
                                       int(k), float(periodic_L), _ptr(idx, ctypes.c_int32),
                                       _ptr(d2, ctypes.c_double), int(threads))
    if rc != 0:
        raise ValueError(f"oracle kNN failed (rc={rc})")
    return idx, d2


def knn_cells(xyz, k, periodic_L=0.0, queries=None, threads=0):
    """Same result as ``knn_brute`` via an exact cell-list search (large N)."""
    return _knn(_load().oracle_knn_cells, xyz, k, periodic_L, queries, threads)


# ------------------------------------------------------------------ FoF

def link_b2(b: float, rel: float = 0.0) -> float:
    """float64 squared linking length from the float32 argument b, scaled by (1+rel)."""
    b64 = float(np.float32(b))
    return b64 * b64 * (1.0 + rel)


def fof_brute(xyz, b, periodic_L=0.0, rel=0.0):
    """All-pairs FoF (Sec. IV): link when d2 <= b^2; label = smallest index in the group."""
    x = np.ascontiguousarray(xyz, dtype=np.float32)
    lab = np.empty(x.shape[0], dtype=np.int32)
    rc = _load().oracle_fof_brute(_ptr(x, ctypes.c_float), x.shape[0], link_b2(b, rel),
                                  float(periodic_L), _ptr(lab, ctypes.c_int32))
    if rc != 0:
        raise ValueError(f"oracle FoF failed (rc={rc})")
    return lab


def fof_cells(xyz, b, periodic_L=0.0, rel=0.0, threads=0):
    """Same result as ``fof_brute`` via clique cells of side < b/sqrt(3) (large N)."""
    x = np.ascontiguousarray(xyz, dtype=np.float32)
    lab = np.empty(x.shape[0], dtype=np.int32)
    b2 = link_b2(b, rel)
    rc = _load().oracle_fof_cells(_ptr(x, ctypes.c_float), x.shape[0], float(np.sqrt(b2)), b2,
                                  float(periodic_L), _ptr(lab, ctypes.c_int32), int(threads))
    if rc != 0:
        raise ValueError(f"oracle FoF (cells) failed (rc={rc})")
    return lab


def fof_bracket(xyz, b, periodic_L=0.0, rel=1e-6, cells=None, threads=0):
    """(labels at b^2(1-rel), labels at b^2(1+rel)): the strict and loose link graphs."""
    if cells is None:
        cells = np.asarray(xyz).shape[0] > 20000
    if not cells:
        return fof_brute(xyz, b, periodic_L, -rel), fof_brute(xyz, b, periodic_L, rel)
    x = np.ascontiguousarray(xyz, dtype=np.float32)
    la = np.empty(x.shape[0], dtype=np.int32)
    lb = np.empty(x.shape[0], dtype=np.int32)
    rc = _load().oracle_fof_cells2(_ptr(x, ctypes.c_float), x.shape[0], link_b2(b, -rel), link_b2(b, rel),
                                   float(periodic_L), _ptr(la, ctypes.c_int32), _ptr(lb, ctypes.c_int32),
                                   int(threads))
    if rc != 0:
        raise ValueError(f"oracle FoF (cells) failed (rc={rc})")
    return la, lb


# ------------------------------------------------------------------ tree (Sec. II)

KEY_BITS = 21
SENTINEL_LEVEL = 64
INDEX_LEVEL_OFFSET = 32


def key_box(xyz, periodic_L=0.0):
    """Quantisation box (lo[3], ext) in float32: [0,L)^3 if periodic, else the
    bounding box with the largest side as a common extent (1 if degenerate)."""
    x = np.asarray(xyz, dtype=np.float32)
    if periodic_L > 0:
        return np.zeros(3, np.float32), np.float32(periodic_L)
    lo = x.min(axis=0).astype(np.float32)
    hi = x.max(axis=0).astype(np.float32)
    ext = np.float32(np.max(hi - lo))
    if not ext > 0:
        ext = np.float32(1.0)
    return lo, ext


def quantise(xyz, periodic_L=0.0):
    """q_d = min(floor(fl32(fl32(x_d - lo_d) * fl32(2^21 / ext))), 2^21 - 1), all in float32."""
    x = np.asarray(xyz, dtype=np.float32)
    lo, ext = key_box(x, periodic_L)
    scale = np.float32(np.float32(1 << KEY_BITS) / ext)
    t = (x - lo[None, :]).astype(np.float32)
    u = (t * scale).astype(np.float32)
    q = np.floor(u).astype(np.int64)
    return np.clip(q, 0, (1 << KEY_BITS) - 1).astype(np.uint64)


def interleave_bits(q) -> np.ndarray:
    """Morton key: bit j of q_x -> key bit 3j+2, of q_y -> 3j+1, of q_z -> 3j
    (one bit at a time; the plain form of the definition)."""
    q = np.asarray(q, dtype=np.uint64)
    key = np.zeros(q.shape[0], dtype=np.uint64)
    for j in range(KEY_BITS):
        for d in range(3):
            bit = (q[:, d] >> np.uint64(j)) & np.uint64(1)
            key |= bit << np.uint64(3 * j + (2 - d))
    return key


def _spread_byte_table() -> np.ndarray:
    """spread[v] for v < 256: bit j of v moved to bit 3j (the definition, per byte)."""
    t = np.zeros(256, dtype=np.uint64)
    for v in range(256):
        w = 0
        for j in range(8):
            w |= ((v >> j) & 1) << (3 * j)
        t[v] = w
    return t


_SPREAD = _spread_byte_table()


def interleave(q) -> np.ndarray:
    """The same key as ``interleave_bits``, one byte of each coordinate at a time:
    byte b of q_d (bits 8b..8b+7) lands on key bits 3(8b+j) + (2-d)."""
    q = np.asarray(q, dtype=np.uint64)
    key = np.zeros(q.shape[0], dtype=np.uint64)
    for d in range(3):
        for b in range(3):  # 21 bits = bytes 0, 1, 2 (the top byte holds 5 bits)
            byte = ((q[:, d] >> np.uint64(8 * b)) & np.uint64(0xFF)).astype(np.intp)
            key |= _SPREAD[byte] << np.uint64(24 * b + (2 - d))
    return key


def morton_keys(xyz, periodic_L=0.0):
    """63-bit z-order keys of float32 points (Sec. II-A, integer Morton key)."""
    return interleave(quantise(xyz, periodic_L))


def zsort(keys):
    """Stable ascending sort by key: (sorted keys, perm) with perm[i] = original index."""
    perm = np.argsort(keys, kind="stable").astype(np.int64)
    return np.asarray(keys)[perm], perm


# ---- full-precision z-order of float32 points (Sec. II-A, Eq. msb and the
# comparator after it; the float alternative to the 21-bit integer keys) ----

ZORDER_EMAX32 = 128  # one above the largest float32 exponent


def _exact32(v) -> int:
    """The float32 value v as the exact integer v * 2^149 (every float32, normal or
    subnormal, is an integer multiple of 2^-149); -0 and +0 both give 0."""
    bits = int(np.asarray(v, dtype=np.float32).view(np.uint32))
    e, f = (bits >> 23) & 0xFF, bits & 0x7FFFFF
    m = f if e == 0 else (f | 0x800000) << (e - 1)  # (2^23 + f) 2^(e-150) = (2^23 + f) 2^(e-1) 2^-149
    return -m if bits >> 31 else m


def zorder_msb(a, b) -> int:
    """msb(a, b) of Eq. msb for float32 a, b: EMAX when the signs differ, otherwise
    the power of two of the highest bit at which |a| and |b| differ when both are
    written as fixed-point numbers (this is max(ex(a), ex(b)) when the exponents
    differ and ex + msb_fixed of the mantissas when they agree).  Equal values give
    -150, below every bit a float32 has.  Zero counts as positive."""
    x, y = _exact32(a), _exact32(b)
    if (x < 0) != (y < 0):
        return ZORDER_EMAX32
    return (abs(x) ^ abs(y)).bit_length() - 150


def zorder_less(p, q) -> bool:
    """p strictly before q in the z-order of Sec. II-A: k is the first dimension of
    the largest msb(p_i, q_i), and p precedes q when p_k < q_k (equal vectors
    precede neither way)."""
    ms = [zorder_msb(p[i], q[i]) for i in range(len(p))]
    k = ms.index(max(ms))
    return _exact32(p[k]) < _exact32(q[k])


def zorder_level(p, q) -> int:
    """lvl(p, q) = (msb(p_k, q_k) + 1) d - k of Sec. II-C (Eq. lvl) at full float32
    precision, k the dimension the comparator compares (d = len(p)).  Equal
    vectors give (-150 + 1) d, below every real level."""
    ms = [zorder_msb(p[i], q[i]) for i in range(len(p))]
    k = ms.index(max(ms))
    return (ms[k] + 1) * len(p) - k


ZORDER_INDEX_LEVEL = -479   # equal vectors: level bit_length((i-1) XOR i) - 479, in [-478, -447]
ZORDER_SENTINEL_LEVEL = 388  # the gaps before the first and after the last point: above (128+1)*3


def zorder_gap_levels(sxyz) -> np.ndarray:
    """lvl_i for gaps i = 0..N between z-sorted float32 points i-1 and i (Sec. II-C)
    at full precision (``zorder_level``).  As for the integer keys, equal points are
    made distinct by their sorted position, whose levels lie below every level of
    distinct points, and the two outer gaps carry a sentinel above every level."""
    x = np.asarray(sxyz, dtype=np.float32)
    n = len(x)
    lvl = np.full(n + 1, ZORDER_SENTINEL_LEVEL, dtype=np.int64)
    for i in range(1, n):
        if np.all(x[i - 1] == x[i]):
            lvl[i] = ((i - 1) ^ i).bit_length() + ZORDER_INDEX_LEVEL
        else:
            lvl[i] = zorder_level(x[i - 1], x[i])
    return lvl


def zorder_node_sizes_brute(sxyz, lvl=None) -> np.ndarray:
    """n_i (Sec. II-C) on the float z-order by direct counting: the points that agree
    with point i above level lvl_i (zorder_level at most lvl_i), or, for a gap
    between equal points, the equal points in the same aligned block of sorted
    positions.  O(N^2): tiny N only."""
    x = np.asarray(sxyz, dtype=np.float32)
    n = len(x)
    if lvl is None:
        lvl = zorder_gap_levels(x)
    out = np.full(n + 1, n, dtype=np.int64)
    for i in range(1, n):
        g = int(lvl[i])
        cnt = 0
        for j in range(n):
            if g > ZORDER_INDEX_LEVEL + 32:
                cnt += zorder_level(x[j], x[i]) <= g
            else:
                bits = g - ZORDER_INDEX_LEVEL
                cnt += bool(np.all(x[j] == x[i])) and (j >> bits) == (i >> bits)
        out[i] = cnt
    return out


def zorder_node_sizes(sxyz, lvl=None) -> np.ndarray:
    """n_i on the float z-order, counted outward from the gap: a node is a
    contiguous range of the sorted points (it holds every point whose prefix
    above its level agrees), so the count walks left from i-1 and right from i
    while the points stay in the node.  Same values as ``zorder_node_sizes_brute``
    (pinned against it), in O(sum of n_i)."""
    x = np.asarray(sxyz, dtype=np.float32)
    n = len(x)
    if lvl is None:
        lvl = zorder_gap_levels(x)
    out = np.full(n + 1, n, dtype=np.int64)
    for i in range(1, n):
        g = int(lvl[i])
        if g > ZORDER_INDEX_LEVEL + 32:
            def inside(j):
                return zorder_level(x[j], x[i]) <= g
        else:
            bits = g - ZORDER_INDEX_LEVEL

            def inside(j):
                return bool(np.all(x[j] == x[i])) and (j >> bits) == (i >> bits)
        lo = i - 1
        while lo - 1 >= 0 and inside(lo - 1):
            lo -= 1
        hi = i + 1
        while hi < n and inside(hi):
            hi += 1
        out[i] = hi - lo
    return out


def zorder_sort(xyz) -> np.ndarray:
    """Stable sort of float32 points by the comparator of Sec. II-A at full
    precision: perm with perm[i] = original index of the i-th point in z order."""
    import functools
    pts = np.asarray(xyz, dtype=np.float32)

    def cmp(i, j):
        return -1 if zorder_less(pts[i], pts[j]) else (1 if zorder_less(pts[j], pts[i]) else 0)
    return np.array(sorted(range(len(pts)), key=functools.cmp_to_key(cmp)), dtype=np.int64)


def _bit_length(v: np.ndarray) -> np.ndarray:
    """Bit length of unsigned 64-bit values (0 for 0).  Each 32-bit half is exact
    in float64, whose frexp exponent is the half's bit length."""
    v = np.asarray(v, dtype=np.uint64)
    hi = (v >> np.uint64(32)).astype(np.float64)
    lo = (v & np.uint64(0xFFFFFFFF)).astype(np.float64)
    return np.where(hi > 0, 32 + np.frexp(hi)[1], np.frexp(lo)[1]).astype(np.int64)


def gap_levels(skeys):
    """lvl_i for gaps i = 0..N between sorted points i-1 and i (Sec. II-C).

    With integer keys lvl(a, b) is the bit length of a XOR b.  Equal keys are
    made distinct by appending the sorted position as 32 lower bits, which gives
    the level bit_length((i-1) XOR i) - 32 (negative).  The gaps before the first
    and after the last point carry the sentinel level 64 (the paper's -inf/+inf
    points)."""
    k = np.asarray(skeys, dtype=np.uint64)
    n = k.shape[0]
    lvl = np.full(n + 1, SENTINEL_LEVEL, dtype=np.int64)
    if n > 1:
        x = k[:-1] ^ k[1:]
        i = np.arange(1, n, dtype=np.uint64)
        idx_lvl = _bit_length((i - np.uint64(1)) ^ i) - INDEX_LEVEL_OFFSET
        lvl[1:n] = np.where(x != 0, _bit_length(x), idx_lvl)
    return lvl


def node_sizes(skeys, lvl=None):
    """n_i: number of points in the smallest node holding sorted points i-1 and i.

    A node at level g holds the points whose (extended) key agrees with point i
    in every bit at or above g; its range [l_b, r_b) is found with searchsorted on
    the sorted keys (Sec. II-C: binary searches to the left and right)."""
    k = np.asarray(skeys, dtype=np.uint64)
    n = k.shape[0]
    if lvl is None:
        lvl = gap_levels(k)
    out = np.full(n + 1, n, dtype=np.int64)
    if n < 2:
        return out
    g = np.asarray(lvl[1:n], dtype=np.int64)
    i = np.arange(1, n, dtype=np.int64)
    ki = k[1:n]
    # distinct-key gaps: the node is the key range sharing every bit >= g
    sh = np.where(g > 0, g, 0).astype(np.uint64)
    lo_key = (ki >> sh) << sh
    hi_key = lo_key | ((np.uint64(1) << sh) - np.uint64(1))
    lb = np.searchsorted(k, lo_key, side="left")
    rb = np.searchsorted(k, hi_key, side="right")
    # equal-key gaps: the aligned block of sorted positions inside the run of equal keys
    bits = np.where(g > 0, 0, g + INDEX_LEVEL_OFFSET)
    run_lo = np.searchsorted(k, ki, side="left")
    run_hi = np.searchsorted(k, ki, side="right")
    blk = (i >> bits) << bits
    lb_eq = np.maximum(run_lo, blk)
    rb_eq = np.minimum(run_hi, blk + (np.int64(1) << bits))
    out[1:n] = np.where(g > 0, rb - lb, rb_eq - lb_eq)
    return out


def node_sizes_brute(skeys, lvl=None):
    """n_i by direct counting of the points that share the prefix (O(N^2), tiny N)."""
    k = [int(v) for v in np.asarray(skeys, dtype=np.uint64)]
    n = len(k)
    if lvl is None:
        lvl = gap_levels(np.asarray(skeys, dtype=np.uint64))
    out = np.full(n + 1, n, dtype=np.int64)
    for i in range(1, n):
        g = int(lvl[i])
        cnt = 0
        for j in range(n):
            if g > 0:
                same = (k[j] >> g) == (k[i] >> g)
            else:
                bits = g + INDEX_LEVEL_OFFSET
                same = k[j] == k[i] and (j >> bits) == (i >> bits)
            cnt += same
        out[i] = cnt
    return out


def num_planes(n: int, nmax0: int = 48, c: int = 8, n_target: int = 1000) -> int:
    """Number of tree-planes: plane 0 always; plane p >= 1 while the estimated node
    count N / (N_max^(p) / 2) stays >= N_target (Sec. II-C, eq. N_nodes)."""
    p = 1
    while 2 * n >= n_target * nmax0 * c ** p:
        p += 1
    return p


VOLUME_BINS = 97  # node-volume classes: 0 = single point, 1 + (level + 32) = volume 2^level


def node_level_bins(lvl, gaps):
    """Volume class of every node [gaps[j], gaps[j+1]) of a plane: 0 for a single
    point (no extent), else 1 + 32 + the largest gap level inside the node."""
    out = np.zeros(len(gaps) - 1, dtype=np.int64)
    for j in range(len(gaps) - 1):
        a, b = int(gaps[j]), int(gaps[j + 1])
        if b - a >= 2:
            out[j] = 1 + 32 + int(np.max(lvl[a + 1:b]))
    return out


def regularization_level(counts, bins, n, f_max):
    """lvl_max of Sec. II-D: 2^lvl_max <= f_max V_90%, V_90% = point-weighted mean
    node volume over the smallest nodes that together hold 90 % of the points.
    Reading: nodes are taken by volume class, smallest first; within the class
    that reaches 90 % only the points still needed are counted.  Evaluated in
    float64 in exactly this order (volume 2^level, single points volume 0);
    returns None (no regularisation) when V_90% is 0."""
    hist = np.zeros(VOLUME_BINS, dtype=np.int64)
    np.add.at(hist, bins, counts)
    target = 0.9 * float(n)
    acc = 0.0
    cum = 0
    for b in range(VOLUME_BINS):
        if hist[b] == 0:
            continue
        vol = 0.0 if b == 0 else float(np.ldexp(1.0, b - 33))
        if float(cum + hist[b]) >= target:
            acc = acc + (target - float(cum)) * vol
            break
        acc = acc + float(hist[b]) * vol
        cum += int(hist[b])
    v90 = acc / target
    x = float(np.float32(f_max)) * v90
    if not x > 0.0:
        return None
    return int(np.frexp(x)[1]) - 1  # floor(log2(x))


def plane_splits(skeys, nmax0: int = 48, c: int = 8, n_target: int = 1000, n_planes=None, f_max: float = 0.0):
    """Tree-plane splits (Sec. II-C, Fig. tree_construction).

    Returns (spl, gaps): spl[p] holds the splits of plane p -- point indices for
    p = 0 and indices into plane p-1's node array for p >= 1 -- and gaps[p] the
    point-space gap index of every split.  A gap is a split of plane p when its
    n exceeds N_max^(p) = N_max^(0) c^p; the first and last gap always are.
    f_max > 0 adds the regularisation of Sec. II-D: after the count splits of a
    plane, every candidate gap whose level exceeds lvl_max^(p) is kept as well."""
    k = np.asarray(skeys, dtype=np.uint64)
    return plane_splits_from_sizes(node_sizes(k), gap_levels(k), nmax0, c, n_target, n_planes, f_max)


def plane_splits_from_sizes(nsz, lvl, nmax0: int = 48, c: int = 8, n_target: int = 1000, n_planes=None,
                            f_max: float = 0.0):
    """``plane_splits`` from the node sizes n_i and gap levels lvl_i of any z order
    (the integer keys, or the float order of ``zorder_gap_levels``; the
    regularisation's volume classes are defined on the integer levels only)."""
    nsz = np.asarray(nsz, dtype=np.int64)
    lvl = np.asarray(lvl, dtype=np.int64)
    n = nsz.shape[0] - 1
    if n_planes is None:
        n_planes = num_planes(n, nmax0, c, n_target)
    gaps = []
    spl = []
    cand = np.arange(n + 1)
    for p in range(n_planes):
        nmax = nmax0 * c ** p
        keep = nsz[cand] > nmax
        keep[0] = True
        keep[-1] = True
        if f_max > 0 and n > 1:
            g0 = cand[np.nonzero(keep)[0]]
            lmax = regularization_level(np.diff(g0), node_level_bins(lvl, g0), n, f_max)
            if lmax is not None:
                keep |= lvl[cand] > lmax
        pos = np.nonzero(keep)[0]
        spl.append(pos.astype(np.int64))
        cand = cand[pos]
        gaps.append(cand.astype(np.int64))
    return spl, gaps


def plane_nodes(sxyz, gaps):
    """Per plane: (count[n_nodes], lo[n_nodes,3], hi[n_nodes,3]) of the sorted points:
    node j holds sorted points gaps[j] .. gaps[j+1]-1 (never empty), its box is their
    coordinate-wise min and max (numpy's segmented reduction over those ranges)."""
    x = np.asarray(sxyz, dtype=np.float32)
    out = []
    for g in gaps:
        g = np.asarray(g, dtype=np.int64)
        cnt = np.diff(g)
        if len(cnt):
            assert (cnt > 0).all(), "empty node"
            lo = np.minimum.reduceat(x, g[:-1], axis=0)
            hi = np.maximum.reduceat(x, g[:-1], axis=0)
        else:
            lo = hi = np.zeros((0, 3), np.float32)
        out.append((cnt.astype(np.int64), lo.astype(np.float32), hi.astype(np.float32)))
    return out


def plane_nodes_loop(sxyz, gaps):
    """``plane_nodes`` with one slice per node (the plain form, for small sets)."""
    x = np.asarray(sxyz, dtype=np.float32)
    out = []
    for g in gaps:
        cnt = np.diff(g)
        lo = np.stack([x[a:b].min(axis=0) for a, b in zip(g[:-1], g[1:])]) if len(cnt) else np.zeros((0, 3), np.float32)
        hi = np.stack([x[a:b].max(axis=0) for a, b in zip(g[:-1], g[1:])]) if len(cnt) else np.zeros((0, 3), np.float32)
        out.append((cnt.astype(np.int64), lo.astype(np.float32), hi.astype(np.float32)))
    return out


def canonical_labels(labels) -> np.ndarray:
    """Relabel a partition so that each group carries its smallest member index."""
    lab = np.asarray(labels)
    n = lab.shape[0]
    first = {}
    out = np.empty(n, dtype=np.int32)
    for i in range(n):
        v = int(lab[i])
        if v not in first:
            first[v] = i
        out[i] = first[v]
    return out


# ------------------------------------------------------------------ FoF catalogue

def fof_catalogue(xyz, labels, periodic_L=0.0, vel=None, min_count=20, particle_mass=1.0):
    """Catalogue reduction after FoF (Sec. IV-B), written from its definition.

    Group order: a stable sort of the points in z order by the z position of their
    group's root (the member with the lowest z position), so roots keep their z
    order and every group is a contiguous block in z order.  Per group of at least
    ``min_count`` points (in group order): mass = count * particle_mass; centre of
    mass of the positions taken relative to the root by the minimum image (periodic)
    and wrapped back into [0, L); inertia radius = sqrt of the mean squared distance
    to the centre of mass; centre-of-mass velocity (zero without velocities).
    Returns (order: original indices in group order, groups: list of dicts with
    label, count, offset, mass, x_cm, v_cm, r_inertia), all float64.
    """
    x = np.asarray(xyz, dtype=np.float32)
    lab = np.asarray(labels, dtype=np.int64)
    n = x.shape[0]
    _, zperm = zsort(morton_keys(x, periodic_L))  # z position -> original index
    zpos = np.empty(n, dtype=np.int64)
    zpos[zperm] = np.arange(n)
    root = np.full(n, n, dtype=np.int64)  # per label: lowest z position of its members
    np.minimum.at(root, lab, zpos)
    zroot = root[lab[zperm]]  # root z position of the point at each z position
    order = zperm[np.argsort(zroot, kind="stable")]
    x64 = x.astype(np.float64)
    v64 = None if vel is None else np.asarray(vel, dtype=np.float32).astype(np.float64)
    groups = []
    starts = np.flatnonzero(np.r_[True, lab[order[1:]] != lab[order[:-1]]])
    ends = np.r_[starts[1:], n]
    for s, e in zip(starts, ends):
        cnt = int(e - s)
        if cnt < min_count:
            continue
        mem = order[s:e]
        ref = x64[mem[0]]
        d = x64[mem] - ref
        if periodic_L > 0:
            d -= periodic_L * np.round(d / periodic_L)
        dm = d.mean(axis=0)
        xcm = ref + dm
        if periodic_L > 0:
            xcm = np.mod(xcm, periodic_L)
        r2 = ((d - dm) ** 2).sum(axis=1).mean()
        groups.append(dict(label=int(lab[mem[0]]), count=cnt, offset=int(s), mass=cnt * float(particle_mass),
                           x_cm=xcm, v_cm=np.zeros(3) if v64 is None else v64[mem].mean(axis=0),
                           r_inertia=float(np.sqrt(r2))))
    return order, groups
