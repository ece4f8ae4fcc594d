"""Separate query and source points (Sec. II-G): every query row equals the
all-pairs query-vs-source oracle under the kNN rule of tests/parity.py."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests import parity
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _check(src, qry, k, L, idx, d2):
    ri, rd = oracle.knn_brute_sets(src, qry, k, L)
    parity.check_knn(src, np.arange(len(qry)), idx.cpu().numpy(), d2.cpu().numpy(), ri, rd, L, query_xyz=qry)


@pytest.mark.parametrize("ns,nq,k,L,gen", [
    (5000, 3000, 16, 1.0, "clustered"), (3000, 7000, 8, 0.0, "clustered"), (6000, 6000, 32, 1.0, "uniform"),
    (4000, 2500, 50, 1.0, "clustered"), (2000, 100, 1, 0.0, "uniform"), (40, 3, 40, 1.0, "uniform"),
    (1, 77, 1, 0.0, "uniform"), (20000, 17, 16, 1.0, "clustered")])
def test_query_sets_match_oracle(ns, nq, k, L, gen):
    import paper_2604_05885_gb300 as jzt
    if gen == "clustered":
        src = workloads.clustered(ns, 900 + ns, n_blobs=max(1, ns // 700))
        qry = workloads.clustered(nq, 901 + nq, n_blobs=max(1, nq // 700))
    else:
        src, qry = workloads.uniform(ns, 902 + ns), workloads.uniform(nq, 903 + nq)
    tree = jzt.build_query(to_dev(src), to_dev(qry), periodic_L=L, k_max=k)
    idx, d2 = tree.knn(k)
    assert tree.status()["code"] == 0
    assert idx.shape == (nq, k)
    _check(src, qry, k, L, idx, d2)


def test_query_on_source_points_and_duplicates():
    """Queries placed on sources find them at d2 = 0 (ties among duplicate sources
    by index); all queries identical."""
    import paper_2604_05885_gb300 as jzt
    src = workloads.uniform(3000, 5)
    src = np.concatenate([src, src[:500]])  # duplicate sources
    qry = np.concatenate([src[::7], np.repeat(src[3:4], 64, axis=0)])
    idx, d2 = jzt.knn_query(to_dev(src), to_dev(qry), 12, 1.0)
    _check(src, qry, 12, 1.0, idx, d2)
    d2 = d2.cpu().numpy()
    idx = idx.cpu().numpy()
    assert np.all(d2[:, 0] == 0.0)
    # a query on a duplicated source ties exactly at d2 = 0 with both copies: the
    # lower index comes first; every row's exact zero-distance ties are in index order
    ri, _ = oracle.knn_brute_sets(src, qry, 12, 1.0)
    zero = d2 == 0.0
    assert np.array_equal(np.where(zero, idx, -1), np.where(zero, ri, -1))
    on_dup = np.nonzero((np.arange(len(qry)) * 7 < 500) & (np.arange(len(qry)) < len(src[::7])))[0]
    assert len(on_dup) > 50
    assert np.array_equal(idx[on_dup, :2], np.stack([on_dup * 7, on_dup * 7 + 3000], axis=1))
    assert np.array_equal(idx[-64:], np.broadcast_to(ri[-1], (64, 12)))


def test_query_far_from_sources_open_box():
    import paper_2604_05885_gb300 as jzt
    src = workloads.clip_unit(workloads.clustered(4000, 8, n_blobs=3) * 0.25)  # back on the 2^-24 grid
    qry = workloads.uniform(900, 9)
    idx, d2 = jzt.knn_query(to_dev(src), to_dev(qry), 10, 0.0)
    _check(src, qry, 10, 0.0, idx, d2)


def test_query_tree_rejects_fof_and_large_k():
    import paper_2604_05885_gb300 as jzt
    src, qry = to_dev(workloads.uniform(100, 1)), to_dev(workloads.uniform(50, 2))
    tree = jzt.build_query(src, qry)
    with pytest.raises(jzt.JztError) as e:
        tree.fof(0.01)
    assert e.value.code == jzt.JZT_ERR_UNSUPPORTED
    with pytest.raises(jzt.JztError) as e:
        tree.knn(101)
    assert e.value.code == jzt.JZT_ERR_INVALID
    torch.cuda.synchronize()


def test_query_sets_on_the_bucket_sort():
    """A combined set of 2^16 points and more sorts its keys by fine bins (sources
    and queries under one index): rows as the all-pairs oracle's."""
    import paper_2604_05885_gb300 as jzt
    src, qry = workloads.uniform(60000, 931), workloads.uniform(10000, 932)
    tree = jzt.build_query(to_dev(src), to_dev(qry), periodic_L=1.0, k_max=16)
    idx, d2 = tree.knn(16)
    st = tree.status()
    assert st["code"] == 0 and st["sort_path"] == 1
    _check(src, qry, 16, 1.0, idx, d2)
