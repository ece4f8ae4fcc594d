"""Tree construction parity (Sec. II) at the full benchmark sizes, bit-exact
against the oracle, in the launch configuration bench.py times (default tree
parameters): Morton keys, the stable sort order, the gathered points and, for
every tree-plane, the splits, node counts and node boxes.

At these sizes the radix sort runs tens of thousands of tiles per pass through
the decoupled look-back, and the split compaction runs its chained scan over
more than a hundred thousand tiles: the paths small sets never reach.

* 2^24 clustered points (4096 Gaussian blobs), periodic unit box.
* 2^27 = 512^3 Zel'dovich points, periodic unit box.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import to_dev, zeldovich_cached

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NMAX0, PLANE_FACTOR, N_TARGET = 32, 8, 1000  # the library defaults


def _gpu_tree(x, L):
    """Build on the GPU; host copies of keys, points and every plane."""
    import torch
    import paper_2604_05885_gb300 as jzt
    n = x.shape[0]
    xt = to_dev(x)
    tree = jzt.build(xt, periodic_L=L, workspace=jzt.alloc_workspace(n, 0, None, xt.device))
    st = tree.status()
    assert st["code"] == 0, st
    keys, pts, n_planes = tree.arrays()
    keys = keys.cpu().numpy().view(np.uint64)
    pts = pts.cpu().numpy()
    planes = [tree.plane(p) for p in range(n_planes)]
    del tree, xt
    torch.cuda.empty_cache()
    return keys, pts, planes


def _check(x, L):
    n = x.shape[0]
    keys, pts, planes = _gpu_tree(x, L)
    sk, perm = oracle.zsort(oracle.morton_keys(x, L))
    assert np.array_equal(keys, sk), f"sorted keys differ at {int(np.argmax(keys != sk))}"
    assert np.array_equal(pts[:, 3].view(np.int32), perm.astype(np.int32)), "sort order (permutation)"
    xs = x[perm]
    assert np.array_equal(pts[:, :3], xs), "gathered points"
    del keys, pts
    assert len(planes) == oracle.num_planes(n, NMAX0, PLANE_FACTOR, N_TARGET)
    spl_ref, gaps_ref = oracle.plane_splits(sk, nmax0=NMAX0, c=PLANE_FACTOR, n_target=N_TARGET)
    nodes_ref = oracle.plane_nodes(xs, gaps_ref)
    for p, ((spl, cnt, box), (rc, rlo, rhi)) in enumerate(zip(planes, nodes_ref)):
        assert np.array_equal(spl, spl_ref[p].astype(np.int32)), f"plane {p} splits"
        assert np.array_equal(cnt, rc.astype(np.int32)), f"plane {p} counts"
        assert np.array_equal(box[:, :3], rlo) and np.array_equal(box[:, 3:], rhi), f"plane {p} boxes"
    return [len(s) - 1 for s in spl_ref]


def test_tree_clustered_2_24():
    _, x = workloads.config_clustered_16m()
    nodes = _check(x, 1.0)
    assert nodes[0] > 100_000 and len(nodes) >= 4


def test_tree_zeldovich_512_cubed():
    x = zeldovich_cached(512)
    nodes = _check(x, 1.0)
    assert nodes[0] > 1_000_000 and len(nodes) >= 5
