"""The full-precision float z-order on the GPU (Sec. II-A, Eq. msb and the
comparator after it; Sec. II-C, Eq. lvl at float32 precision), selected with
jzt_params.float_order = 1.

* Extreme-range points (1e-30 .. 1e30, mixed signs, -0 and +0, subnormals,
  duplicates): the sorted order equals the oracle's comparator sort, and every
  plane's splits, counts and boxes equal the oracle's tree-planes built from the
  float gap levels and node sizes.
* On points of the 2^-21 grid the float order builds the integer-key tree.
* Multi-scale clusters (scales 2^-50 .. 2^40, exact small-mantissa coordinates):
  kNN rows and FoF labels equal the all-pairs oracle, and equal the rows and
  labels of the integer-key tree.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests import parity
from tests.gpu_util import knn_parity, to_dev

pytestmark = pytest.mark.gpu

FLOAT = dict(float_order=1)


def _extreme(n, seed):
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal((n, 3)) * 10.0 ** rng.uniform(-30, 30, (n, 3))).astype(np.float32)
    x[::17] = x[min(3, n - 1)]                        # duplicates
    x[::19, 0] = 0.0
    x[::23, 1] = -0.0
    sub = rng.integers(1, 1 << 20, (len(x[::29]), 3)).astype(np.float64) * 2.0 ** -149
    x[::29] = sub.astype(np.float32)                 # subnormals
    return np.ascontiguousarray(x)


def _clusters(n_per, seed, exps=(-50, -40, -30, -20, -10, 0, 10, 20, 30, 40), centre_seed=0):
    """One cluster per scale 2^e: its centre lies 2^(e+9) .. 2^(e+10) from the origin
    in every dimension (random signs, from centre_seed), its points in a cube of
    side 2^e around it.  Every coordinate is 2^(e-8) times an integer below 2^19,
    so differences inside a cluster are exact in float32, and any other cluster
    is much farther than a point's own (a point's neighbours lie in its cluster)."""
    crng = np.random.default_rng(centre_seed)
    rng = np.random.default_rng(seed)
    out = []
    for e in exps:
        c = crng.integers(1 << 9, 1 << 10, 3).astype(np.float64) * crng.choice([-1.0, 1.0], 3) * 256
        q = rng.integers(0, 256, (n_per, 3)).astype(np.float64)
        out.append((c + q) * 2.0 ** e / 256)
    x = np.concatenate(out).astype(np.float32)
    return np.ascontiguousarray(x[rng.permutation(len(x))])


def _tree_check(x, params):
    import paper_2604_05885_gb300 as jzt
    p = dict(params)
    nmax0, c, nt = p.get("nmax0", 32), p.get("plane_factor", 8), p.get("n_target", 1000)
    tree = jzt.build(to_dev(x), periodic_L=0.0, params=p)
    assert tree.status()["code"] == 0
    keys, pts, n_planes = tree.arrays()
    assert keys is None
    pts = pts.cpu().numpy()
    perm = oracle.zorder_sort(x)
    assert np.array_equal(pts[:, 3].view(np.int32), perm.astype(np.int32)), "float z-order"
    sx = x[perm]
    assert np.array_equal(pts[:, :3], sx)
    lvl = oracle.zorder_gap_levels(sx)
    spl_ref, gaps_ref = oracle.plane_splits_from_sizes(oracle.zorder_node_sizes(sx, lvl), lvl, nmax0, c, nt)
    assert n_planes == len(spl_ref)
    nodes_ref = oracle.plane_nodes(sx, gaps_ref)
    for pl in range(n_planes):
        spl, cnt, box = tree.plane(pl)
        assert np.array_equal(spl, spl_ref[pl].astype(np.int32)), f"plane {pl} splits"
        rc, rlo, rhi = nodes_ref[pl]
        assert np.array_equal(cnt, rc.astype(np.int32)), f"plane {pl} counts"
        assert np.array_equal(box[:, :3], rlo) and np.array_equal(box[:, 3:], rhi), f"plane {pl} boxes"
    return n_planes


@pytest.mark.parametrize("n,params", [(3000, dict(nmax0=8, n_target=20)), (2049, dict(nmax0=4, plane_factor=2, n_target=30)),
                                      (5000, dict(nmax0=32, n_target=5)), (1, {}), (2, {}), (33, dict(nmax0=3))])
def test_float_order_tree_matches_oracle(n, params):
    """Points spread over 60 decades give lopsided planes (most upper nodes hold a
    handful of points), more nodes than Eq. alloc_nodes estimates for balanced
    data: the node allocation factor is raised accordingly."""
    x = _extreme(n, 100 + n)
    planes = _tree_check(x, dict(params, alloc_fac_nodes=16.0, **FLOAT))
    if n >= 2049:
        assert planes >= 2


def test_float_order_equals_integer_tree_on_the_grid():
    """On the 2^-21 grid of [0, 1)^3 the float comparator is the integer Morton
    order and the float levels are the integer levels (shifted): same tree."""
    import paper_2604_05885_gb300 as jzt
    rng = np.random.default_rng(7)
    x = (rng.integers(0, 1 << 21, (20000, 3)).astype(np.float64) / (1 << 21)).astype(np.float32)
    x[100:180] = x[5]
    xt = to_dev(x)
    a = jzt.build(xt, periodic_L=1.0, params=dict(n_target=4))
    b = jzt.build(xt, periodic_L=1.0, params=dict(n_target=4, **FLOAT))
    _, pa, na = a.arrays()
    _, pb, nb = b.arrays()
    assert na == nb >= 3
    assert np.array_equal(pa.cpu().numpy(), pb.cpu().numpy())
    for pl in range(na):
        for u, v in zip(a.plane(pl), b.plane(pl)):
            assert np.array_equal(u, v)


@pytest.mark.parametrize("k", [1, 8, 16, 32])
def test_float_order_knn_on_multiscale_clusters(k):
    import paper_2604_05885_gb300 as jzt
    x = _clusters(300, 40 + k)
    tree = jzt.build(to_dev(x), periodic_L=0.0, params=FLOAT)
    idx, d2 = knn_parity(tree, x, k, 0.0)
    ref = jzt.build(to_dev(x), periodic_L=0.0)
    ri, rd = ref.knn(k)
    assert np.array_equal(idx, ri.cpu().numpy()) and np.array_equal(d2, rd.cpu().numpy())


def test_float_order_fof_on_multiscale_clusters():
    import paper_2604_05885_gb300 as jzt
    x = _clusters(300, 51)
    for b in (2.0 ** -50 * 3, 2.0 ** -20 * 1.5, 2.0 ** 10 * 2):
        tree = jzt.build(to_dev(x), periodic_L=0.0, params=FLOAT)
        lab = tree.fof(b).cpu().numpy()
        assert tree.status()["code"] == 0
        s, lo = oracle.fof_bracket(x, b, 0.0)
        parity.check_fof(lab, s, lo)
        ref = jzt.build(to_dev(x), periodic_L=0.0).fof(b).cpu().numpy()
        assert np.array_equal(lab, ref)


def test_float_order_query_sets():
    import paper_2604_05885_gb300 as jzt
    src = _clusters(200, 61, centre_seed=6)
    qry = _clusters(50, 62, centre_seed=6)  # queries inside the source clusters
    tree = jzt.build_query(to_dev(src), to_dev(qry), params=FLOAT, k_max=12)
    idx, d2 = tree.knn(12)
    assert tree.status()["code"] == 0
    ri, rd = oracle.knn_brute_sets(src, qry, 12, 0.0)
    parity.check_knn(src, np.arange(len(qry)), idx.cpu().numpy(), d2.cpu().numpy(), ri, rd, 0.0, query_xyz=qry)


def test_float_order_reports_node_capacity():
    """The default node allocation is an estimate for balanced data (Eq. alloc_nodes):
    the lopsided extreme-range tree overflows it and says so (JZT_ERR_CAPACITY)."""
    import paper_2604_05885_gb300 as jzt
    tree = jzt.build(to_dev(_extreme(3000, 3100)), params=dict(nmax0=8, n_target=20, **FLOAT))
    assert tree.status()["code"] == jzt.JZT_ERR_CAPACITY


def test_float_order_with_regularisation_is_refused():
    import paper_2604_05885_gb300 as jzt
    with pytest.raises(jzt.JztError) as e:
        jzt.build(to_dev(workloads.uniform(100, 1)), params=dict(reg_fmax=2.0, **FLOAT))
    assert e.value.code == jzt.JZT_ERR_UNSUPPORTED
