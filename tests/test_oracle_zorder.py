"""Pins of the oracle's full-precision float z-order (Sec. II-A, Eq. msb and the
comparator after it), each from something other than the oracle itself: the
paper's msb_fixed example, the cases of Eq. msb, the integer Morton order it must
reproduce on the 2^-21 grid, numeric order along one axis, the axioms of a strict
weak order (brute force), invariance under exact power-of-two scaling, and the
order of full-precision (278 bits per coordinate) interleaved integer keys."""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "msb_example.txt")


def _binary(s: str) -> float:
    whole, frac = s.split(".")
    return int(whole, 2) + sum(int(c) * 2.0 ** -(i + 1) for i, c in enumerate(frac))


def test_paper_msb_example():
    rows = dict(line.split() for line in open(GOLDEN) if line.strip() and not line.startswith("#"))
    a, b = _binary(rows["a"]), _binary(rows["b"])
    assert (a, b) == (169.3125, 165.6875)
    assert oracle.zorder_msb(a, b) == int(rows["msb"]) == oracle.zorder_msb(b, a)


def test_msb_cases():
    assert oracle.zorder_msb(-1.0, 1.0) == oracle.ZORDER_EMAX32 == 128      # signs differ
    assert oracle.zorder_msb(-2.0 ** -149, 3.0e38) == 128
    assert oracle.zorder_msb(1.0, 2.0) == 1                                 # exponents differ: the larger
    assert oracle.zorder_msb(0.75, 3.0) == 1
    assert oracle.zorder_msb(-0.75, -3.0) == 1
    assert oracle.zorder_msb(2.0 ** 127 * 1.5, 1.0) == 127
    assert oracle.zorder_msb(1.5, 1.25) == -1                               # same exponent: ex + msb_fixed
    assert oracle.zorder_msb(12.0, 13.0) == 0
    assert oracle.zorder_msb(2.0 ** -149, 2.0 ** -148) == -148              # subnormals
    assert oracle.zorder_msb(0.0, 2.0 ** -149) == -149
    assert oracle.zorder_msb(2.0 ** -126, 2.0 ** -126 - 2.0 ** -149) == -126  # normal vs subnormal
    assert oracle.zorder_msb(5.0, 5.0) == -150 == oracle.zorder_msb(-0.0, 0.0)


def test_grid_points_follow_the_integer_morton_order():
    """On the 2^-21 grid of [0,1)^3 the comparator and the interleaved 21-bit key
    (x the most significant coordinate) give the same order."""
    rng = np.random.default_rng(11)
    q = rng.integers(0, 1 << 21, (3000, 3))
    q[100:140] = q[100]                                     # exact duplicates: stable order
    q[200:260, 1:] = q[200, 1:]                             # points sharing two coordinates
    x = (q.astype(np.float64) / (1 << 21)).astype(np.float32)
    _, perm = oracle.zsort(oracle.interleave(q.astype(np.int64)))
    assert np.array_equal(oracle.zorder_sort(x), perm)


def test_one_axis_is_numeric_order():
    rng = np.random.default_rng(12)
    v = np.concatenate([rng.standard_normal(200) * 10.0 ** rng.uniform(-40, 38, 200),
                        [0.0, -0.0, 2.0 ** -149, -2.0 ** -149, 3.0e38, -3.0e38, 1.0, 1.0]]).astype(np.float32)
    x = np.zeros((len(v), 3), np.float32)
    x[:, 0] = v
    want = np.argsort(v.astype(np.float64) + 0.0, kind="stable")  # -0 == +0
    assert np.array_equal(oracle.zorder_sort(x), want)
    y = np.zeros((len(v), 3), np.float32)                       # along z alone, the same
    y[:, 2] = v
    assert np.array_equal(oracle.zorder_sort(y), want)


def test_strict_weak_order_brute_force():
    rng = np.random.default_rng(13)
    pool = np.array([0.0, -0.0, 1.0, -1.0, 0.5, 3.0, -2.5, 2.0 ** -140, 7.0e20, -1.0e-30], np.float32)
    x = rng.choice(pool, (36, 3)).astype(np.float32)
    x[::5] = rng.standard_normal((8, 3)).astype(np.float32)
    n = len(x)
    less = np.array([[oracle.zorder_less(x[i], x[j]) for j in range(n)] for i in range(n)])
    same = np.array([[bool(np.all(x[i] == x[j])) for j in range(n)] for i in range(n)])
    assert not less.diagonal().any()                            # irreflexive
    assert not (less & less.T).any()                            # asymmetric
    assert np.array_equal(~(less | less.T), same)               # only equal vectors are unordered
    two = (less.astype(np.int64) @ less.astype(np.int64)) > 0   # i < j < k for some j
    assert not (two & ~less).any()                              # transitive


def test_power_of_two_scaling_keeps_the_order():
    rng = np.random.default_rng(14)
    x = (rng.standard_normal((800, 3)) * 10.0 ** rng.uniform(-3, 3, (800, 3))).astype(np.float32)
    base = oracle.zorder_sort(x)
    for s in (-40, -3, 5, 60):
        assert np.array_equal(oracle.zorder_sort((x * np.float32(2.0 ** s)).astype(np.float32)), base)


def _wide_key(p) -> int:
    """Morton key of a float32 point at full precision: each coordinate becomes the
    278-bit unsigned U = 2^277 + m (v >= 0) or 2^277 - 1 - m (v < 0), where
    m = |v| 2^149 is exact, and the three U are interleaved bit by bit, x most
    significant.  Same-sign values keep the XOR of their magnitudes and the sign
    becomes the top bit, so this integer order is the comparator's order."""
    import struct
    key = 0
    us = []
    for v in p:
        bits = struct.unpack("<I", struct.pack("<f", float(v)))[0]
        e, f = (bits >> 23) & 0xFF, bits & 0x7FFFFF
        m = f if e == 0 else (f + (1 << 23)) << (e - 1)
        neg = bool(bits >> 31) and m != 0
        us.append((1 << 277) - 1 - m if neg else (1 << 277) + m)
    for b in range(278):
        for d in range(3):
            key |= ((us[d] >> b) & 1) << (3 * b + 2 - d)
    return key


def test_comparator_equals_wide_integer_morton_order():
    rng = np.random.default_rng(15)
    x = (rng.standard_normal((500, 3)) * 10.0 ** rng.uniform(-44, 37, (500, 3))).astype(np.float32)
    x[::9, 0] = 0.0
    x[::13, 1] = -0.0
    x[::17] = x[4]
    keys = [_wide_key(p) for p in x]
    want = sorted(range(len(x)), key=lambda i: (keys[i], i))
    assert oracle.zorder_sort(x).tolist() == want


def _u278(v) -> int:
    import struct
    bits = struct.unpack("<I", struct.pack("<f", float(v)))[0]
    e, f = (bits >> 23) & 0xFF, bits & 0x7FFFFF
    m = f if e == 0 else (f + (1 << 23)) << (e - 1)
    return (1 << 277) - 1 - m if (bits >> 31) and m else (1 << 277) + m


def test_windowed_radix_plan_equals_comparator():
    """The GPU plan for the float z-order: T = the highest bit at which any
    coordinate of the set varies (bits above it are common to all points), then
    63-bit keys from aligned 21-bit windows [T-20, T], [T-41, T-21], ... of the
    three coordinates, and a stable sort by the windows from the lowest to the
    highest (LSD) -- the same order as the comparator."""
    rng = np.random.default_rng(16)
    for scale_lo, scale_hi in ((-2, 2), (-44, 37), (-1, 0)):
        x = (rng.standard_normal((400, 3)) * 10.0 ** rng.uniform(scale_lo, scale_hi, (400, 3))).astype(np.float32)
        if scale_hi == 0:
            x = np.abs(x) % 1.0                                   # box-bounded, non-negative
        x[::23] = x[7]
        u = [[_u278(v) for v in p] for p in x]
        top = max((min(c) ^ max(c)).bit_length() for c in zip(*u)) - 1
        perm = list(range(len(x)))
        lows = list(range(top - 20, -21, -21))[::-1]              # window bottoms, lowest first
        for lo in lows:
            def key(i, lo=lo):
                k = 0
                for b in range(20, -1, -1):
                    for d in range(3):
                        bit = (u[i][d] >> (lo + b)) & 1 if lo + b >= 0 else 0
                        k = (k << 1) | bit
                return k
            perm = sorted(perm, key=key)                          # stable: LSD over the windows
        assert perm == oracle.zorder_sort(x).tolist()


def test_float_level_matches_integer_gap_level_on_the_grid():
    """Eq. lvl at full precision against the integer form bit_length(key XOR key):
    on the 2^-21 grid of [0,1)^3 bit j of a coordinate weighs 2^(j-21), so the two
    differ by the constant 3 * 21 = 63."""
    rng = np.random.default_rng(17)
    q = rng.integers(0, 1 << 21, (2000, 3))
    q[50:60] = q[50]
    q[300:400, :2] = q[300, :2]
    x = (q.astype(np.float64) / (1 << 21)).astype(np.float32)
    skeys, perm = oracle.zsort(oracle.interleave(q.astype(np.int64)))
    lvl = oracle.gap_levels(skeys)
    for i in range(1, len(x)):
        a, b = x[perm[i - 1]], x[perm[i]]
        if skeys[i - 1] != skeys[i]:
            assert oracle.zorder_level(a, b) == lvl[i] - 63
        else:
            assert oracle.zorder_level(a, b) == -447
    assert oracle.zorder_level((1.0, 0.0, 0.0), (1.0, 0.5, 0.0)) == (-1 + 1) * 3 - 1
    assert oracle.zorder_level((-1.0, 0.0, 0.0), (1.0, 0.0, 0.0)) == (128 + 1) * 3


def test_float_tree_levels_and_sizes_match_the_integer_tree_on_the_grid():
    rng = np.random.default_rng(18)
    q = rng.integers(0, 1 << 21, (400, 3))
    q[10:30] = q[10]                                            # a run of equal points
    q[100:160, 0] = q[100, 0]
    x = (q.astype(np.float64) / (1 << 21)).astype(np.float32)
    skeys, perm = oracle.zsort(oracle.interleave(q.astype(np.int64)))
    lvl_i, n_i = oracle.gap_levels(skeys), oracle.node_sizes(skeys)
    sx = x[oracle.zorder_sort(x)]
    lvl_f = oracle.zorder_gap_levels(sx)
    inner = slice(1, len(x))
    dup = np.concatenate([[False], skeys[1:] == skeys[:-1]])[inner]
    d = lvl_f[inner] - lvl_i[inner]
    assert np.all(d[~dup] == -63) and np.all(d[dup] == -447)
    assert np.array_equal(oracle.zorder_node_sizes_brute(sx, lvl_f), n_i)


def test_float_node_sizes_are_contiguous_segments():
    """The points of a node form one segment of the z order, bounded by the first
    gaps on either side whose level exceeds the node's (extreme ranges, duplicates)."""
    rng = np.random.default_rng(19)
    x = (rng.standard_normal((70, 3)) * 10.0 ** rng.uniform(-30, 30, (70, 3))).astype(np.float32)
    x[5:12] = x[5]
    x[40:44, 1:] = x[40, 1:]
    sx = x[oracle.zorder_sort(x)]
    lvl = oracle.zorder_gap_levels(sx)
    sizes = oracle.zorder_node_sizes_brute(sx, lvl)
    n = len(sx)
    for i in range(1, n):
        l = i - 1
        while l > 0 and lvl[l] <= lvl[i]:
            l -= 1
        r = i
        while r < n - 1 and lvl[r + 1] <= lvl[i]:
            r += 1
        assert sizes[i] == r - l + 1


def test_float_tree_planes_match_the_integer_tree_on_the_grid():
    rng = np.random.default_rng(20)
    q = rng.integers(0, 1 << 21, (600, 3))
    q[200:260] = q[200]
    x = (q.astype(np.float64) / (1 << 21)).astype(np.float32)
    skeys, _ = oracle.zsort(oracle.interleave(q.astype(np.int64)))
    sx = x[oracle.zorder_sort(x)]
    lvl = oracle.zorder_gap_levels(sx)
    sizes = oracle.zorder_node_sizes_brute(sx, lvl)
    for nmax0, c, nt in ((4, 2, 20), (8, 4, 10), (48, 8, 1000)):
        spl_i, gaps_i = oracle.plane_splits(skeys, nmax0, c, nt)
        spl_f, gaps_f = oracle.plane_splits_from_sizes(sizes, lvl, nmax0, c, nt)
        assert len(spl_i) == len(spl_f)
        assert all(np.array_equal(a, b) for a, b in zip(gaps_i, gaps_f))
        assert all(np.array_equal(a, b) for a, b in zip(spl_i, spl_f))


def test_node_sizes_walk_equals_brute_count():
    """The outward count of n_i (used at the sizes of the GPU tests) equals the
    direct count over all points, on mixed-scale data with duplicates and zeros."""
    rng = np.random.default_rng(31)
    x = (rng.standard_normal((160, 3)) * 10.0 ** rng.uniform(-30, 30, (160, 3))).astype(np.float32)
    x[::11] = x[5]
    x[::13, 2] = -0.0
    sx = x[oracle.zorder_sort(x)]
    lvl = oracle.zorder_gap_levels(sx)
    assert np.array_equal(oracle.zorder_node_sizes(sx, lvl), oracle.zorder_node_sizes_brute(sx, lvl))
