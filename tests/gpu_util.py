"""Helpers for the GPU parity tests."""
import os

import numpy as np
import torch

import workloads

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


CACHE = os.path.join(os.environ.get("TMPDIR", "/tmp"), "jzt_bench_cache")


def zeldovich_cached(n_side=512):
    """The n_side^3 Zel'dovich set (seed 3), cached as .npy between runs on one machine."""
    path = os.path.join(CACHE, f"zeldovich_{n_side}_seed3.npy")
    if os.path.exists(path):
        return np.load(path)
    x = workloads.zeldovich(n_side, 3)
    os.makedirs(CACHE, exist_ok=True)
    np.save(path + ".tmp.npy", x)
    os.replace(path + ".tmp.npy", path)
    return x
