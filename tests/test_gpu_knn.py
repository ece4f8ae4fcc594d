"""kNN parity (Sec. III) against the oracle: neighbour indices and float32 squared
distances under the rule in tests/parity.py."""
import numpy as np
import pytest

import oracle
import workloads
from tests import parity
from tests.gpu_util import knn_parity, to_dev

pytestmark = pytest.mark.gpu


def test_small_uniform_open_k16():
    """N = 32768 uniform in the unit cube, open boundaries, k = 16 (full parity)."""
    import paper_2604_05885_gb300 as jzt
    w, x = workloads.config_small_uniform()
    tree = jzt.build(to_dev(x), periodic_L=w.periodic_L)
    knn_parity(tree, x, w.k, w.periodic_L)


@pytest.mark.parametrize("k", [1, 2, 5, 8, 13, 16, 24, 32])
def test_k_values_periodic(k):
    import paper_2604_05885_gb300 as jzt
    x = workloads.uniform(9001, 10 + k)
    tree = jzt.build(to_dev(x), periodic_L=1.0)
    knn_parity(tree, x, k, 1.0)


@pytest.mark.parametrize("params", [dict(nmax0=1), dict(nmax0=3, plane_factor=2, n_target=20),
                                    dict(nmax0=16, n_target=10), dict(heap_size=2), dict(heap_size=16),
                                    dict(ngr=1), dict(ngr=7, n_target=50)])
def test_tree_parameters_do_not_change_results(params):
    import paper_2604_05885_gb300 as jzt
    x = workloads.clustered(6000, 11, n_blobs=12)
    tree = jzt.build(to_dev(x), periodic_L=1.0, params=params)
    knn_parity(tree, x, 16, 1.0)


def test_clustered_periodic_k32_multiplane():
    import paper_2604_05885_gb300 as jzt
    x = workloads.clustered(60000, 2, n_blobs=15)
    tree = jzt.build(to_dev(x), periodic_L=1.0, params=dict(n_target=20))
    assert tree.arrays()[2] >= 2
    q = np.random.default_rng(0).choice(len(x), 4000, replace=False)
    knn_parity(tree, x, 32, 1.0, queries=q)


def test_lattice_ties_by_index():
    """Exact ties: every interior point of a lattice has 12 neighbours at sqrt(2) h,
    of which k = 16 keeps the 9 with the lowest indices."""
    import paper_2604_05885_gb300 as jzt
    for L, xs in ((0.0, workloads.lattice(10, spacing_bits=9)), (1.0, workloads.lattice(16, spacing_bits=4))):
        tree = jzt.build(to_dev(xs), periodic_L=L)
        idx, _ = knn_parity(tree, xs, 16, L)
        ri, _ = oracle.knn_brute(xs, 16, L)
        assert np.array_equal(idx, ri)  # ties are exact in float32: indices must agree


@pytest.mark.parametrize("k", [2, 5, 10, 20, 30])
def test_lattice_ties_by_index_small_k(k):
    """Rows ending inside a shell of equal distances (6 at h, 12 at sqrt(2) h, 8 at
    sqrt(3) h around the point itself) under every candidate-list size (4, 8, 16,
    32): the tied entries kept are those with the lowest indices."""
    import paper_2604_05885_gb300 as jzt
    for L, xs in ((0.0, workloads.lattice(9, spacing_bits=9)), (1.0, workloads.lattice(12, spacing_bits=4))):
        tree = jzt.build(to_dev(xs), periodic_L=L)
        idx, _ = knn_parity(tree, xs, k, L)
        ri, _ = oracle.knn_brute(xs, k, L)
        assert np.array_equal(idx, ri)


def test_duplicates_and_degenerate_geometry():
    import paper_2604_05885_gb300 as jzt
    x = workloads.uniform(2000, 12)
    x[50:450] = x[50]            # 400 copies of one point
    x[600:700, 2] = x[600, 2]     # a flat patch
    dup = np.arange(50, 450)
    for L in (0.0, 1.0):
        tree = jzt.build(to_dev(x), periodic_L=L, params=dict(nmax0=8, n_target=8))
        idx, d2 = knn_parity(tree, x, 16, L)
        # duplicates tie exactly at d2 = 0: each copy lists the 16 lowest indices of
        # the run, in index order (the parity rule alone would accept any order)
        ri, _ = oracle.knn_brute(x, 16, L, queries=dup)
        assert np.array_equal(idx[dup], ri)
        assert np.array_equal(idx[dup], np.broadcast_to(np.arange(50, 66), (len(dup), 16)))
        assert np.all(d2[dup] == 0.0)
    line = np.zeros((500, 3), np.float32)
    line[:, 1] = workloads.uniform(500, 13)[:, 1]
    tree = jzt.build(to_dev(line), periodic_L=0.0)
    knn_parity(tree, line, 8, 0.0)


@pytest.mark.parametrize("n,k", [(1, 1), (2, 2), (3, 1), (32, 32), (33, 32), (52, 1), (100, 7)])
@pytest.mark.parametrize("gen", ["uniform", "clustered"])
def test_tiny_sets(n, k, gen):
    import paper_2604_05885_gb300 as jzt
    x = workloads.uniform(n, 100 + n) if gen == "uniform" else workloads.clustered(n, 7000 + n, n_blobs=2)
    for L in (0.0, 1.0):
        tree = jzt.build(to_dev(x), periodic_L=L)
        knn_parity(tree, x, k, L)


def test_z_order_rows():
    import paper_2604_05885_gb300 as jzt
    x = workloads.uniform(7000, 14)
    tree = jzt.build(to_dev(x), periodic_L=1.0)
    knn_parity(tree, x, 12, 1.0, order=1)


def test_one_call_form_and_repeat_queries():
    import paper_2604_05885_gb300 as jzt
    x = workloads.uniform(5000, 15)
    xt = to_dev(x)
    idx, d2 = jzt.knn(xt, 10, 1.0)
    ri, rd = oracle.knn_brute(x, 10, 1.0)
    from tests import parity
    parity.check_knn(x, np.arange(5000), idx.cpu().numpy(), d2.cpu().numpy(), ri, rd, 1.0)
    tree = jzt.build(xt, periodic_L=1.0)
    a = tree.knn(10)
    b = tree.knn(10)
    assert np.array_equal(a[0].cpu().numpy(), b[0].cpu().numpy())
    assert np.array_equal(a[1].cpu().numpy(), b[1].cpu().numpy())


def test_capacity_error_then_retry():
    """Too small an interaction-list allocation factor reports JZT_ERR_CAPACITY with a
    larger required size (Eq. alloc_ilist); the default factor then succeeds."""
    import paper_2604_05885_gb300 as jzt
    x = workloads.uniform(20000, 16)
    xt = to_dev(x)
    p = dict(alloc_fac_ilist=0.5)
    tree = jzt.build(xt, periodic_L=1.0, params=p)
    tree.knn(16)
    st = tree.status()
    assert st["code"] == jzt.JZT_ERR_CAPACITY
    assert st["required_bytes"] > tree.workspace.numel()
    tree = jzt.build(xt, periodic_L=1.0)
    knn_parity(tree, x, 16, 1.0)


@pytest.mark.parametrize("k,L,gen", [(33, 1.0, "clustered"), (64, 0.0, "clustered"), (100, 1.0, "uniform"),
                                     (256, 1.0, "clustered"), (97, 0.0, "uniform")])
def test_k_above_32_passes(k, L, gen):
    """k > 32 runs ceil(k/32) LeafToLeaf passes; rows equal the all-pairs oracle."""
    import paper_2604_05885_gb300 as jzt
    n = 5000
    x = workloads.clustered(n, 70 + k, n_blobs=6) if gen == "clustered" else workloads.uniform(n, 70 + k)
    tree = jzt.build(to_dev(x), periodic_L=L, workspace=jzt.alloc_workspace(n, k))
    knn_parity(tree, x, k, L)


def test_k_above_32_ties_across_pass_boundary():
    """Lattice shells: the 32nd neighbour lies inside the 6-point shell at 2h, so the
    tie at the pass boundary must continue in index order in the second pass."""
    import paper_2604_05885_gb300 as jzt
    xs = workloads.lattice(12, spacing_bits=4)
    for k in (40, 64):
        tree = jzt.build(to_dev(xs), periodic_L=1.0, workspace=jzt.alloc_workspace(len(xs), k))
        idx, _ = knn_parity(tree, xs, k, 1.0)
        ri, _ = oracle.knn_brute(xs, k, 1.0)
        assert np.array_equal(idx, ri)


def test_k_above_32_one_call_and_z_order():
    import paper_2604_05885_gb300 as jzt
    x = workloads.clustered(3000, 77, n_blobs=3)
    idx, d2 = jzt.knn(to_dev(x), 70, 1.0)
    ri, rd = oracle.knn_brute(x, 70, 1.0)
    parity.check_knn(x, np.arange(len(x)), idx.cpu().numpy(), d2.cpu().numpy(), ri, rd, 1.0)
    tree = jzt.build(to_dev(x), periodic_L=1.0, workspace=jzt.alloc_workspace(len(x), 70))
    knn_parity(tree, x, 70, 1.0, order=1)
