"""FoF parity (Sec. IV) against the oracle under the strict/loose rule in tests/parity.py."""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import fof_parity, to_dev

pytestmark = pytest.mark.gpu


def test_small_uniform_open():
    """N = 32768 uniform, open, b = 0.2 N^(-1/3)."""
    import paper_2604_05885_gb300 as jzt
    w, x = workloads.config_small_uniform()
    tree = jzt.build(to_dev(x), periodic_L=w.periodic_L)
    fof_parity(tree, x, w.b, w.periodic_L)


@pytest.mark.parametrize("fac", [0.2, 0.5, 0.9, 1.5])
@pytest.mark.parametrize("L", [0.0, 1.0])
def test_linking_lengths(fac, L):
    import paper_2604_05885_gb300 as jzt
    n = 20000
    x = workloads.uniform(n, 21)
    tree = jzt.build(to_dev(x), periodic_L=L, params=dict(n_target=10))
    fof_parity(tree, x, fac * workloads.mean_spacing(n), L)


def test_clustered_whole_node_links():
    """Dense blobs: node-node links (d_up <= b) carry most of the grouping."""
    import paper_2604_05885_gb300 as jzt
    n = 50000
    x = workloads.clustered(n, 22, n_blobs=20, sigma_lo=1e-4, sigma_hi=3e-3)
    for L in (1.0,):
        tree = jzt.build(to_dev(x), periodic_L=L, params=dict(n_target=20))
        fof_parity(tree, x, 0.2 * workloads.mean_spacing(n), L)


def test_lattice_closed_forms():
    import paper_2604_05885_gb300 as jzt
    h = 1.0 / 512
    x = workloads.lattice(12, spacing_bits=9)
    tree = jzt.build(to_dev(x), periodic_L=0.0)
    lab = tree.fof(0.999 * h).cpu().numpy()
    assert np.array_equal(lab, np.arange(len(x)))
    for b in (h, 1.001 * h, 1.4 * h):
        assert (tree.fof(b).cpu().numpy() == 0).all()
    xp = workloads.lattice(16, spacing_bits=4)
    tree = jzt.build(to_dev(xp), periodic_L=1.0)
    assert (tree.fof(1.0 / 16).cpu().numpy() == 0).all()
    ii = np.indices((16, 16, 16)).reshape(3, -1).T
    cut = xp[ii[:, 0] != 5]
    tree = jzt.build(to_dev(cut), periodic_L=0.0)
    assert len(np.unique(tree.fof(1.0 / 16).cpu().numpy())) == 2
    tree = jzt.build(to_dev(cut), periodic_L=1.0)
    assert len(np.unique(tree.fof(1.0 / 16).cpu().numpy())) == 1


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 1000])
def test_tiny_sets(n):
    import paper_2604_05885_gb300 as jzt
    x = workloads.uniform(n, 200 + n)
    for L in (0.0, 1.0):
        tree = jzt.build(to_dev(x), periodic_L=L)
        fof_parity(tree, x, 0.3, L) if L == 0.0 else fof_parity(tree, x, 0.3, L)


def test_duplicates():
    import paper_2604_05885_gb300 as jzt
    x = workloads.uniform(3000, 23)
    x[10:500] = x[10]
    tree = jzt.build(to_dev(x), periodic_L=1.0, params=dict(nmax0=8))
    fof_parity(tree, x, 0.2 * workloads.mean_spacing(3000), 1.0)


def test_permutation_invariance():
    import paper_2604_05885_gb300 as jzt
    x = workloads.clustered(8000, 24, n_blobs=10)
    b = 0.3 * workloads.mean_spacing(8000)
    a = jzt.build(to_dev(x), periodic_L=1.0).fof(b).cpu().numpy()
    perm = np.random.default_rng(2).permutation(len(x))
    c = jzt.build(to_dev(x[perm]), periodic_L=1.0).fof(b).cpu().numpy()
    assert np.array_equal(oracle.canonical_labels(a[perm]), c)


def test_repeated_runs_near_percolation():
    """Many concurrent unions (b near the percolation threshold): every repeat of
    the walk must give the oracle's labels, so no union or contraction is lost
    to a race."""
    import paper_2604_05885_gb300 as jzt
    n = 20000
    x = workloads.uniform(n, 21)
    b = 0.9 * workloads.mean_spacing(n)
    s, lo = oracle.fof_bracket(x, b, 0.0, cells=True)
    for nt in (10, 1000):
        tree = jzt.build(to_dev(x), periodic_L=0.0, params=dict(n_target=nt))
        for _ in range(6):
            lab = tree.fof(b).cpu().numpy()
            assert tree.status()["code"] == 0
            from tests import parity
            parity.check_fof(lab, s, lo)
