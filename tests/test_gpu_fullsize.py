"""Parity at the full benchmark sizes, in the launch configuration bench.py times
(default parameters, workspace sized by jzt_workspace_bytes(N, k)).

* 512^3 = 2^27 Zel'dovich points, periodic unit box, k = 16, b = 0.2/512: kNN rows
  of 20000 sampled points against the cell-list oracle; every FoF label against
  the cell-list oracle run on all 2^27 points.
* 2^24 clustered points (4096 blobs), periodic, k = 32, b = 0.2/256: kNN rows of
  20000 sampled points; FoF labels of all points.

The oracle side runs on the host cores (float64), the GPU side through the C ABI.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests import parity
from tests.gpu_util import to_dev, zeldovich_cached

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _zeldovich512():
    return zeldovich_cached(512)


def _run(x, k, b, L):
    import torch
    import paper_2604_05885_gb300 as jzt
    n = x.shape[0]
    xt = to_dev(x)
    ws = jzt.alloc_workspace(n, k, None, xt.device)
    tree = jzt.build(xt, periodic_L=L, workspace=ws)
    idx, d2 = tree.knn(k)
    lab = tree.fof(b)
    st = tree.status()
    assert st["code"] == 0, st
    out = (idx.cpu().numpy(), d2.cpu().numpy(), lab.cpu().numpy())
    del tree, ws, idx, d2, lab, xt
    torch.cuda.empty_cache()
    return out


def _check(x, k, b, L, idx, d2, lab, n_sample, seed):
    q = np.sort(np.random.default_rng(seed).choice(x.shape[0], n_sample, replace=False))
    ri, rd = oracle.knn_cells(x, k, L, queries=q)
    parity.check_knn(x, q, idx[q], d2[q], ri, rd, L)
    s, lo = oracle.fof_bracket(x, b, L, cells=True)
    parity.check_fof(lab, s, lo)


def test_zeldovich_512_cubed():
    x = _zeldovich512()
    k, b, L = 16, 0.2 / 512, 1.0
    idx, d2, lab = _run(x, k, b, L)
    _check(x, k, b, L, idx, d2, lab, 20000, 7)


def test_clustered_2_24():
    w, x = workloads.config_clustered_16m()
    idx, d2, lab = _run(x, w.k, w.b, w.periodic_L)
    _check(x, w.k, w.b, w.periodic_L, idx, d2, lab, 20000, 8)


def test_cell_oracle_matches_brute_force_at_full_size():
    """The cell-list kNN oracle used above, checked against all-pairs brute force on
    1000 seeded sampled queries of the 2^27-point set (exact rows, including ties)."""
    x = _zeldovich512()
    q = np.sort(np.random.default_rng(9).choice(x.shape[0], 1000, replace=False))
    ci, cd = oracle.knn_cells(x, 16, 1.0, queries=q)
    bi, bd = oracle.knn_brute(x, 16, 1.0, queries=q)
    assert np.array_equal(ci, bi)
    assert np.array_equal(cd, bd)
