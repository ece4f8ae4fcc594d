"""Pins for the oracle: each test checks it against something other than itself
(the paper's worked example, closed forms, an independent enumeration, a
library routine, or an invariance of the definition)."""
import os

import numpy as np
import pytest

import oracle
import workloads
from tests import parity

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or ":" not in line:
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = v.split()
    return out


# ------------------------------------------------------------------ tree: worked example

def test_worked_example_1d():
    """Fig. tree_construction (Sec. II-C): levels, n, spl^(0), spl^(1)."""
    g = _golden("worked_example.txt")
    x = np.array([float(v) for v in g["x"]])
    keys = np.floor(x * 8).astype(np.uint64)
    assert keys.tolist() == [int(v) for v in g["fixed_keys"]]
    lvl = oracle.gap_levels(keys)
    assert lvl.tolist() == [int(v) for v in g["key_levels"]]
    paper = [int(v) for v in g["paper_levels_inner"]]
    assert (lvl[1:-1] - 3).tolist() == paper
    n = oracle.node_sizes(keys)
    assert n.tolist() == [int(v) for v in g["n"]]
    assert oracle.node_sizes_brute(keys).tolist() == n.tolist()
    spl, _ = oracle.plane_splits(keys, nmax0=int(g["nmax0"][0]), c=int(g["c"][0]), n_planes=2)
    assert spl[0].tolist() == [int(v) for v in g["spl0"]]
    assert spl[1].tolist() == [int(v) for v in g["spl1"]]


def test_worked_example_3d_on_x_axis():
    """Same example through the 3-D quantiser: points on the x axis of a periodic box
    of side 2^18 quantise to q_x = floor(8x); levels scale by 3, n and splits match."""
    g = _golden("worked_example.txt")
    x = np.array([float(v) for v in g["x"]], dtype=np.float32)
    pts = np.zeros((8, 3), np.float32)
    pts[:, 0] = x
    rng = np.random.default_rng(0)
    perm = rng.permutation(8)
    keys = oracle.morton_keys(pts[perm], periodic_L=float(1 << 18))
    sk, order = oracle.zsort(keys)
    assert np.array_equal(perm[order], np.arange(8))
    lvl = oracle.gap_levels(sk)
    assert (lvl[1:-1] // 3).tolist() == [int(v) for v in g["key_levels"]][1:-1]
    assert oracle.node_sizes(sk).tolist() == [int(v) for v in g["n"]]
    spl, _ = oracle.plane_splits(sk, nmax0=2, c=2, n_planes=2)
    assert spl[0].tolist() == [int(v) for v in g["spl0"]]
    assert spl[1].tolist() == [int(v) for v in g["spl1"]]


# ------------------------------------------------------------------ tree: keys and order

def test_interleave_bits():
    q = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [2, 0, 0], [(1 << 21) - 1] * 3, [5, 3, 6]], np.uint64)
    k = oracle.interleave(q)
    assert k[0] == 4 and k[1] == 2 and k[2] == 1 and k[3] == 32
    assert k[4] == (1 << 63) - 1
    # 5 = 101, 3 = 011, 6 = 110 -> triples (x,y,z) per bit j: j0 (1,1,0) j1 (0,1,1) j2 (1,0,1)
    assert int(k[5]) == (0b110) | (0b011 << 3) | (0b101 << 6)


def test_interleave_forms_agree():
    """The byte-table interleave equals the bit-by-bit definition (and the hand
    values above hold for both)."""
    rng = np.random.default_rng(5)
    q = rng.integers(0, 1 << 21, (20000, 3)).astype(np.uint64)
    q[:3] = [[0, 0, 0], [(1 << 21) - 1] * 3, [1 << 20, 1, 1 << 7]]
    assert np.array_equal(oracle.interleave(q), oracle.interleave_bits(q))


def test_bit_length_matches_python():
    rng = np.random.default_rng(6)
    v = np.concatenate([rng.integers(0, 2**63, 5000, dtype=np.uint64) >> rng.integers(0, 64, 5000).astype(np.uint64),
                        np.array([0, 1, 2, 3, 2**32 - 1, 2**32, 2**53 + 1, 2**63, 2**64 - 1], dtype=np.uint64)])
    assert oracle._bit_length(v).tolist() == [int(x).bit_length() for x in v]


def test_plane_nodes_forms_agree():
    """Segmented min/max boxes equal one slice per node."""
    x = workloads.clustered(5000, 21, n_blobs=5)
    sk, perm = oracle.zsort(oracle.morton_keys(x, 1.0))
    _, gaps = oracle.plane_splits(sk, nmax0=8, c=4, n_target=10)
    a = oracle.plane_nodes(x[perm], gaps)
    b = oracle.plane_nodes_loop(x[perm], gaps)
    assert len(a) == len(b) >= 3
    for (ca, la, ha), (cb, lb, hb) in zip(a, b):
        assert np.array_equal(ca, cb) and np.array_equal(la, lb) and np.array_equal(ha, hb)


def _msb_int(a, b):
    x = a ^ b
    return x.bit_length() - 1 if x else -1


def test_key_order_matches_paper_comparator():
    """Sorting by the interleaved key equals sorting with the paper's comparator
    (Sec. II-A): compare along the dimension with the highest differing bit, the
    first such dimension winning ties (x most significant)."""
    import functools
    rng = np.random.default_rng(3)
    q = rng.integers(0, 1 << 21, size=(300, 3)).astype(np.uint64)
    q[::7] = q[3]  # duplicates
    q[::11, 1] = q[5, 1]

    def cmp(a, b):
        m = [_msb_int(int(a[d]), int(b[d])) for d in range(3)]
        kd = int(np.argmax(m))
        if m[kd] < 0:
            return 0
        return -1 if int(a[kd]) < int(b[kd]) else 1

    order_cmp = sorted(range(len(q)), key=functools.cmp_to_key(lambda i, j: cmp(q[i], q[j]) or (i - j)))
    keys = oracle.interleave(q)
    _, order_key = oracle.zsort(keys)
    assert order_key.tolist() == order_cmp


def test_quantise_periodic_unit_box_exact():
    x = workloads.uniform(1000, 7)
    q = oracle.quantise(x, 1.0)
    assert np.array_equal(q, np.floor(x.astype(np.float64) * (1 << 21)).astype(np.uint64))


def test_quantise_open_box_covers_range():
    x = workloads.uniform(1000, 8) * np.float32(0.5) + np.float32(0.25)
    q = oracle.quantise(x, 0.0)
    assert q.min() == 0 and q.max() == (1 << 21) - 1


def test_node_sizes_with_duplicate_keys():
    rng = np.random.default_rng(11)
    keys = np.sort(rng.integers(0, 40, 300).astype(np.uint64))  # long equal runs
    lvl = oracle.gap_levels(keys)
    assert lvl[0] == 64 and lvl[-1] == 64
    assert ((lvl[1:-1] >= -31) & (lvl[1:-1] <= 63) & (lvl[1:-1] != 0)).all()
    assert np.array_equal(oracle.node_sizes(keys, lvl), oracle.node_sizes_brute(keys, lvl))


@pytest.mark.parametrize("nmax0,c", [(48, 8), (32, 8), (4, 2)])
def test_plane_invariants(nmax0, c):
    """Sec. II-C: every plane partitions the points, nodes hold <= N_max^(p) points,
    coarser splits are a subset of finer ones, and every split has n > N_max^(p)."""
    x = workloads.clustered(20000, 5, n_blobs=20)
    x[100:400] = x[100]  # a run of 300 identical points
    keys = oracle.morton_keys(x, 1.0)
    sk, _ = oracle.zsort(keys)
    n = oracle.node_sizes(sk)
    spl, gaps = oracle.plane_splits(sk, nmax0=nmax0, c=c, n_target=10)
    assert len(spl) == oracle.num_planes(20000, nmax0, c, 10)
    for p, (s, g) in enumerate(zip(spl, gaps)):
        nmax = nmax0 * c ** p
        assert g[0] == 0 and g[-1] == len(x)
        assert (np.diff(g) > 0).all()
        assert (np.diff(g) <= nmax).all()
        assert (n[g[1:-1]] > nmax).all()
        if p > 0:
            assert np.isin(g, gaps[p - 1]).all()
            assert np.array_equal(gaps[p - 1][s], g)


def test_num_planes_large():
    assert oracle.num_planes(1 << 27, 48, 8, 1000) == 5
    assert oracle.num_planes(32768, 48, 8, 1000) == 1


# ------------------------------------------------------------------ kNN

def _knn_full_sort(x, k, L):
    """Independent enumeration: the complete distance matrix sorted by (d2, j)."""
    xd = x.astype(np.float64)
    d = xd[None, :, :] - xd[:, None, :]
    if L > 0:
        d = d - L * np.round(d / L)
    d2 = (d * d).sum(-1)
    n = len(x)
    idx = np.empty((n, k), np.int64)
    for i in range(n):
        o = np.lexsort((np.arange(n), d2[i]))
        idx[i] = o[:k]
    return idx, np.take_along_axis(d2, idx, 1)


@pytest.mark.parametrize("L", [0.0, 1.0])
@pytest.mark.parametrize("seed", [0, 1])
def test_knn_brute_vs_full_sort(L, seed):
    x = workloads.uniform(64, 100 + seed)
    x[5] = x[9]  # an exact duplicate
    for k in (1, 5, 16, 64):
        ii, dd = oracle.knn_brute(x, k, L)
        ri, rd = _knn_full_sort(x, k, L)
        assert np.array_equal(ii, ri)
        assert np.array_equal(dd, rd)


def test_knn_brute_vs_scipy():
    from scipy.spatial import cKDTree
    x = workloads.uniform(2000, 5)
    for L in (0.0, 1.0):
        ii, dd = oracle.knn_brute(x, 12, L)
        t = cKDTree(x.astype(np.float64), boxsize=1.0 if L > 0 else None)
        sd, si = t.query(x.astype(np.float64), k=12)
        assert np.allclose(dd, sd ** 2, rtol=1e-12, atol=0)
        # continuous random data: no ties, so the index sets agree too
        assert np.array_equal(np.sort(ii, 1), np.sort(si, 1))


def test_knn_lattice_closed_form():
    """Interior point of a cubic lattice: self, then 6 at h^2, 12 at 2h^2, 8 at 3h^2;
    k = 16 takes 9 of the 12 second neighbours, chosen by lowest index."""
    m = 7
    x = workloads.lattice(m, spacing_bits=9)
    h2 = (1.0 / 512) ** 2
    c = (3 * m + 3) * m + 3
    ii, dd = oracle.knn_brute(x, 27, 0.0, queries=[c])
    assert ii[0, 0] == c and dd[0, 0] == 0
    assert np.allclose(dd[0, 1:7], h2) and np.allclose(dd[0, 7:19], 2 * h2) and np.allclose(dd[0, 19:27], 3 * h2)
    # the expected 12 second neighbours, in index order
    second = sorted(((3 + a) * m + 3 + b) * m + 3 + e for a in (-1, 0, 1) for b in (-1, 0, 1) for e in (-1, 0, 1)
                    if abs(a) + abs(b) + abs(e) == 2)
    assert ii[0, 7:19].tolist() == second
    i16, _ = oracle.knn_brute(x, 16, 0.0, queries=[c])
    assert i16[0, 7:16].tolist() == second[:9]


def test_knn_periodic_lattice_wraps():
    """On a periodic lattice every point sees 6 neighbours at h^2, including across the box edge."""
    x = workloads.lattice(8, spacing_bits=3)  # spacing 1/8 fills the unit box
    ii, dd = oracle.knn_brute(x, 7, 1.0)
    assert np.allclose(dd[:, 1:], (1.0 / 8) ** 2)
    ii_open, dd_open = oracle.knn_brute(x, 7, 0.0)
    assert dd_open[0, 6] > (1.0 / 8) ** 2  # a corner has only 3 nearest neighbours when open


def test_knn_permutation_and_translation_invariance():
    x = workloads.clustered(3000, 9, n_blobs=10)
    k = 10
    ii, dd = oracle.knn_brute(x, k, 1.0)
    perm = np.random.default_rng(1).permutation(len(x))
    ip, dp = oracle.knn_brute(x[perm], k, 1.0)
    assert np.array_equal(dd[perm], dp)
    shift = np.array([12345, 999, 777777], np.float64) / (1 << 24)
    xs = workloads.snap_unit(x.astype(np.float64) + shift)
    it, dt = oracle.knn_brute(xs, k, 1.0)
    assert np.array_equal(dt, dd)
    assert (np.diff(dd, axis=1) >= 0).all()


@pytest.mark.parametrize("L", [0.0, 1.0])
@pytest.mark.parametrize("gen", ["uniform", "clustered"])
def test_knn_cells_equals_brute(L, gen):
    x = workloads.uniform(6000, 21) if gen == "uniform" else workloads.clustered(6000, 22, n_blobs=8)
    x[10:20] = x[10]
    for k in (1, 16, 32):
        a = oracle.knn_brute(x, k, L)
        b = oracle.knn_cells(x, k, L)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ------------------------------------------------------------------ FoF

def _fof_warshall(x, b2, L):
    """Independent enumeration: boolean transitive closure of the link matrix."""
    xd = x.astype(np.float64)
    d = xd[None, :, :] - xd[:, None, :]
    if L > 0:
        d = d - L * np.round(d / L)
    adj = (d * d).sum(-1) <= b2
    n = len(x)
    r = adj.copy()
    for m in range(n):
        r |= r[:, m:m + 1] & r[m:m + 1, :]
    return np.array([int(np.argmax(r[i])) for i in range(n)], np.int32)


@pytest.mark.parametrize("L", [0.0, 1.0])
def test_fof_brute_vs_warshall(L):
    for seed in range(3):
        x = workloads.uniform(60, 200 + seed)
        for b in (0.05, 0.12, 0.2):
            lab = oracle.fof_brute(x, b, L)
            assert np.array_equal(lab, _fof_warshall(x, oracle.link_b2(b), L))


def test_fof_brute_vs_scipy():
    from scipy.sparse.csgraph import connected_components
    from scipy.spatial import cKDTree
    x = workloads.clustered(5000, 3, n_blobs=30)
    b = 0.01
    for L in (0.0, 1.0):
        lab = oracle.fof_brute(x, b, L)
        t = cKDTree(x.astype(np.float64), boxsize=1.0 if L > 0 else None)
        pairs = t.query_pairs(float(np.float32(b)), output_type="ndarray")
        import scipy.sparse as sp
        g = sp.coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(len(x),) * 2)
        _, cc = connected_components(g, directed=False)
        assert np.array_equal(oracle.canonical_labels(cc), lab)


def test_fof_lattice_closed_form():
    """Cubic lattice of spacing h: b < h gives singletons, b = h (<= is the linking
    rule, Sec. IV-A) and h < b < sqrt(2) h give one group; periodic too; removing one
    plane of the open lattice splits it in two."""
    m = 6
    h = 1.0 / 512
    x = workloads.lattice(m, spacing_bits=9)
    n = len(x)
    assert np.array_equal(oracle.fof_brute(x, 0.999 * h), np.arange(n))
    for b in (h, 1.001 * h, 1.4 * h):
        assert (oracle.fof_brute(x, b) == 0).all()
    xp = workloads.lattice(8, spacing_bits=3)
    assert (oracle.fof_brute(xp, 1.0 / 8, 1.0) == 0).all()
    assert np.array_equal(oracle.fof_brute(xp, 0.99 / 8, 1.0), np.arange(len(xp)))
    ii = np.indices((m, m, m)).reshape(3, -1).T
    keep = ii[:, 0] != 2
    lab = oracle.fof_brute(x[keep], h)
    assert len(np.unique(lab)) == 2
    # the periodic lattice minus one plane stays connected through the wrap
    iip = np.indices((8, 8, 8)).reshape(3, -1).T
    labp = oracle.fof_brute(xp[iip[:, 0] != 2], 1.0 / 8, 1.0)
    assert len(np.unique(labp)) == 1


def test_fof_symmetry_and_permutation_invariance():
    x = workloads.clustered(2000, 13, n_blobs=12)
    b = 0.02
    lab = oracle.fof_brute(x, b, 1.0)
    parity.check_canonical(lab)
    perm = np.random.default_rng(4).permutation(len(x))
    labp = oracle.fof_brute(x[perm], b, 1.0)
    # same partition: relabel through the permutation
    assert np.array_equal(oracle.canonical_labels(lab[perm]), labp)
    # linking is symmetric: reversing every pair's order gives the same partition
    xr = x[::-1].copy()
    assert np.array_equal(oracle.canonical_labels(lab[::-1]), oracle.fof_brute(xr, b, 1.0))


@pytest.mark.parametrize("L", [0.0, 1.0])
@pytest.mark.parametrize("gen", ["uniform", "clustered"])
def test_fof_cells_equals_brute(L, gen):
    n = 8000
    x = workloads.uniform(n, 31) if gen == "uniform" else workloads.clustered(n, 32, n_blobs=8)
    x[50:90] = x[50]
    for fac in (0.2, 0.5, 1.0):
        b = fac * workloads.mean_spacing(n)
        assert np.array_equal(oracle.fof_cells(x, b, L), oracle.fof_brute(x, b, L))
    # a large linking length relative to the box (many cells per neighbourhood)
    assert np.array_equal(oracle.fof_cells(x[:500], 0.3, L), oracle.fof_brute(x[:500], 0.3, L))
    # the strict/loose bracket computed in one pass equals two all-pairs runs
    b = 0.5 * workloads.mean_spacing(n)
    s_c, l_c = oracle.fof_bracket(x, b, L, rel=0.05, cells=True)
    s_b, l_b = oracle.fof_bracket(x, b, L, rel=0.05, cells=False)
    assert np.array_equal(s_c, s_b) and np.array_equal(l_c, l_b)
    assert not np.array_equal(s_b, l_b)  # the two thresholds differ on this set


# ------------------------------------------------------------------ comparison rules

def test_knn_rule_rejects_wrong_and_accepts_ties():
    x = workloads.lattice(5, spacing_bits=9)
    q = np.array([62])
    ri, rd = oracle.knn_brute(x, 8, 0.0, queries=q)
    gd = rd.astype(np.float32)
    parity.check_knn(x, q, ri, gd, ri, rd)
    # swapping two tied neighbours (both at h^2) is accepted
    gi = ri.copy()
    gi[0, 1], gi[0, 2] = gi[0, 2], gi[0, 1]
    parity.check_knn(x, q, gi, gd, ri, rd)
    # replacing a neighbour by a farther point is rejected
    gi = ri.copy()
    gi[0, 7] = 0
    with pytest.raises(AssertionError):
        parity.check_knn(x, q, gi, gd, ri, rd)
    # a d2 off by more than 2 ulp is rejected
    bad = gd.copy()
    bad[0, 3] = np.nextafter(np.nextafter(np.nextafter(bad[0, 3], 1), 1), 1)
    with pytest.raises(AssertionError):
        parity.check_knn(x, q, ri, bad, ri, rd)


def test_fof_rule():
    x = workloads.uniform(500, 3)
    b = 0.08
    s, lo = oracle.fof_bracket(x, b)
    lab = oracle.fof_brute(x, b)
    parity.check_fof(lab, s, lo)
    wrong = lab.copy()
    wrong[wrong == wrong[7]] = 7 if wrong[7] != 7 else wrong[7]
    wrong[123] = 0 if lab[123] != 0 else 1
    with pytest.raises(AssertionError):
        parity.check_fof(wrong, s, lo)


def test_knn_sets_pins():
    """Query-vs-source oracle: against a full lexsort of the cross distance matrix,
    against scipy's cKDTree on separate sets, equal to the self query when the
    query set is the source set, and a query placed on a source point finds it first."""
    rng = np.random.default_rng(41)
    src = workloads.snap_unit(rng.random((700, 3)))
    qry = workloads.snap_unit(rng.random((300, 3)))
    for L in (0.0, 1.0):
        ri, rd = oracle.knn_brute_sets(src, qry, 9, L)
        d = qry[:, None, :].astype(np.float64) - src[None, :, :].astype(np.float64)
        if L > 0:
            d -= L * np.round(d / L)
        d2 = (d * d).sum(-1)
        order = np.lexsort((np.broadcast_to(np.arange(len(src)), d2.shape), d2), axis=1)[:, :9]
        assert np.array_equal(ri, order)
        assert np.allclose(rd, np.take_along_axis(d2, order, 1), rtol=0, atol=0)
    from scipy.spatial import cKDTree
    dd, ii = cKDTree(src.astype(np.float64)).query(qry.astype(np.float64), 5)
    ri, rd = oracle.knn_brute_sets(src, qry, 5, 0.0)
    assert np.allclose(np.sqrt(rd), dd) and np.array_equal(ri, ii)
    si, sd = oracle.knn_brute(src, 7, 1.0)
    qi, qd = oracle.knn_brute_sets(src, src, 7, 1.0)
    assert np.array_equal(si, qi) and np.array_equal(sd, qd)
    qi, qd = oracle.knn_brute_sets(src, src[[5, 17]], 1, 0.0)
    assert list(qi[:, 0]) == [5, 17] and np.all(qd == 0.0)


def test_fof_catalogue_pins():
    """Catalogue: group order keeps roots in z order and members contiguous in z
    order; counts and offsets partition the points; a two-point group across the
    periodic boundary has its centre of mass on the boundary side and inertia radius
    = half the separation; velocities average; groups below min_count drop."""
    L = 1.0
    x = np.array([[0.999, 0.5, 0.5], [0.001, 0.5, 0.5],   # pair across x = 0
                  [0.25, 0.25, 0.25], [0.25, 0.25, 0.2578125], [0.25, 0.2578125, 0.25],  # triple
                  [0.7, 0.1, 0.9]], dtype=np.float32)
    x = workloads.snap_unit(x)
    lab = oracle.fof_brute(x, 0.01, L)
    v = np.arange(18, dtype=np.float32).reshape(6, 3)
    order, groups = oracle.fof_catalogue(x, lab, L, vel=v, min_count=2)
    assert sorted(order.tolist()) == list(range(6))
    by = {g["label"]: g for g in groups}
    assert set(by) == {0, 2} and by[0]["count"] == 2 and by[2]["count"] == 3
    pair = by[0]
    sep = (1.0 - float(x[0, 0])) + float(x[1, 0])
    assert abs(pair["r_inertia"] - sep / 2) < 1e-12
    assert min(pair["x_cm"][0], 1.0 - pair["x_cm"][0]) < 1e-3
    assert np.allclose(pair["v_cm"], (v[0] + v[1]) / 2)
    # contiguity and offsets: members of each group sit at [offset, offset + count)
    for g in groups:
        assert set(lab[order[g["offset"]:g["offset"] + g["count"]]]) == {g["label"]}
    # group order: roots in z order, members in z order
    _, zp = oracle.zsort(oracle.morton_keys(x, L))
    zpos = np.empty(6, int)
    zpos[zp] = np.arange(6)
    zo = zpos[order]
    rootz = np.array([min(zpos[lab == lab[i]]) for i in order])
    assert np.all(np.diff(rootz) >= 0)
    same = rootz[1:] == rootz[:-1]
    assert np.all(np.diff(zo)[same] > 0)
    # min_count drops small groups; singletons everywhere gives the z order itself
    _, g20 = oracle.fof_catalogue(x, lab, L, min_count=20)
    assert g20 == []
    o1, _ = oracle.fof_catalogue(x, np.arange(6), L, min_count=1)
    assert np.array_equal(o1, zp)


def test_fof_catalogue_matches_direct_sums_on_clusters():
    """Random clustered set: every catalogue entry equals a direct computation from
    the members of its label (open box: plain mean and spread)."""
    x = workloads.clustered(3000, 19, n_blobs=5)
    lab = oracle.fof_brute(x, 0.004, 0.0)
    order, groups = oracle.fof_catalogue(x, lab, 0.0, min_count=5, particle_mass=2.5)
    assert groups
    for g in groups:
        mem = np.flatnonzero(lab == g["label"])
        assert g["count"] == len(mem) and g["mass"] == 2.5 * len(mem)
        p = x[mem].astype(np.float64)
        assert np.allclose(g["x_cm"], p.mean(0), rtol=0, atol=1e-12)
        assert abs(g["r_inertia"] - np.sqrt(((p - p.mean(0)) ** 2).sum(1).mean())) < 1e-12


def test_regularisation_pins():
    """Sec. II-D in the oracle: f_max = 0 or huge leaves the planes unchanged; with
    regularisation no node of a plane has level above lvl_max^(p) unless it is one
    point; the lvl_max value equals an independent computation (points expanded by
    node volume, sorted, the first 90 % averaged)."""
    rng = np.random.default_rng(12)
    x = workloads.clip_unit(np.concatenate([rng.normal(0.5, 0.01, (3000, 3)), rng.random((30, 3))]))
    sk, _ = oracle.zsort(oracle.morton_keys(x, 0.0))
    plain = oracle.plane_splits(sk, 32, 8, 20)[1]
    for f in (0.0, 1e30):
        got = oracle.plane_splits(sk, 32, 8, 20, f_max=f)[1]
        assert all(np.array_equal(a, b) for a, b in zip(got, plain))
    lvl = oracle.gap_levels(sk)
    reg = oracle.plane_splits(sk, 32, 8, 20, f_max=50.0)[1]
    assert len(reg[0]) > len(plain[0])
    # lvl_max of plane 0 from its count splits, independently
    g0 = plain[0]
    cnt = np.diff(g0)
    bins = oracle.node_level_bins(lvl, g0)
    vols = np.where(bins == 0, 0.0, np.ldexp(1.0, bins - 33))
    per_point = np.sort(np.repeat(vols, cnt))
    m = 0.9 * len(sk)
    whole = int(np.floor(m))
    v90 = (per_point[:whole].sum() + (m - whole) * per_point[whole]) / m
    lmax = int(np.floor(np.log2(50.0 * v90)))
    assert oracle.regularization_level(cnt, bins, len(sk), 50.0) == lmax
    # every regularised leaf with two or more points lies inside a cell of level <= lmax
    for a, b in zip(reg[0][:-1], reg[0][1:]):
        if b - a >= 2:
            assert lvl[a + 1:b].max() <= lmax
