"""Helpers for the GPU parity tests."""
import numpy as np
import torch

import oracle
from tests import parity


def dev():
    return torch.device("cuda:0")


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev())


def knn_parity(tree, x, k, L, queries=None, ref=None, order=0):
    import paper_2604_05885_gb300 as jzt  # noqa: F401
    idx, d2 = tree.knn(k, order=order)
    st = tree.status()
    assert st["code"] == 0, st
    idx = idx.cpu().numpy()
    d2 = d2.cpu().numpy()
    n = x.shape[0]
    if order == 1:
        _, pts, _ = tree.arrays()
        orig = pts[:, 3].contiguous().view(torch.int32).cpu().numpy()
        gi = np.empty_like(idx)
        gd = np.empty_like(d2)
        gi[orig] = idx
        gd[orig] = d2
        idx, d2 = gi, gd
    if queries is None:
        queries = np.arange(n)
    if ref is None:
        ref = oracle.knn_brute(x, k, L, queries=queries) if n <= 40000 else oracle.knn_cells(x, k, L, queries=queries)
    parity.check_knn(x, queries, idx[queries], d2[queries], ref[0], ref[1], L)
    return idx, d2


def fof_parity(tree, x, b, L):
    lab = tree.fof(b)
    st = tree.status()
    assert st["code"] == 0, st
    lab = lab.cpu().numpy()
    s, lo = oracle.fof_bracket(x, b, L, cells=x.shape[0] > 6000)
    parity.check_fof(lab, s, lo)
    return lab
