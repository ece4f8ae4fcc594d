"""Comparison rules shared by the parity tests (GPU result vs oracle result).

kNN: the GPU row must equal the oracle row index by index, except where the two
indices sit at float64 squared distances within 1e-6 relative of each other (a
tie, or a near-tie that float32 cannot order); every returned float32 d2 must be
within 2 ulp of the float64 recomputation of its own pair; a row holds no index
twice.

FoF: the oracle labels the strict graph (d2 <= b^2 (1 - 1e-6)) and the loose graph
(d2 <= b^2 (1 + 1e-6)).  When they agree the GPU labels must be identical;
otherwise every GPU group must be a union of strict groups and lie inside one
loose group.  GPU labels must also be canonical: each group carries its smallest
member index.
"""
from __future__ import annotations

import numpy as np

KNN_REL = 1e-6
D2_ULPS = 2


def check_knn(xyz, queries, gpu_idx, gpu_d2, ref_idx, ref_d2, periodic_L=0.0, rel=KNN_REL, query_xyz=None):
    """Raise AssertionError with a short report if the rows disagree beyond the rule.
    xyz holds the points the rows index; the query of row r is xyz[queries[r]], or
    query_xyz[r] when the queries are a separate point set."""
    gpu_idx = np.asarray(gpu_idx).astype(np.int64)
    gpu_d2 = np.asarray(gpu_d2, dtype=np.float32)
    ref_idx = np.asarray(ref_idx).astype(np.int64)
    ref_d2 = np.asarray(ref_d2, dtype=np.float64)
    q = np.asarray(queries, dtype=np.int64)
    assert gpu_idx.shape == ref_idx.shape, (gpu_idx.shape, ref_idx.shape)
    n = np.asarray(xyz).shape[0]
    assert gpu_idx.min() >= 0 and gpu_idx.max() < n, "index out of range"
    x = np.asarray(xyz, dtype=np.float64)
    xq = x[q] if query_xyz is None else np.asarray(query_xyz, dtype=np.float64)
    d = x[gpu_idx] - xq[:, None, :]
    if periodic_L > 0:
        d = d - periodic_L * np.round(d / periodic_L)
    g64 = np.sum(d * d, axis=-1)
    # 1) indices equal, or the two candidates are (near-)tied
    differ = gpu_idx != ref_idx
    tol = rel * np.maximum(ref_d2, np.finfo(np.float64).tiny)
    bad = differ & (np.abs(g64 - ref_d2) > tol)
    if bad.any():
        r, c = np.argwhere(bad)[0]
        raise AssertionError(
            f"kNN mismatch: {int(bad.sum())} entries; first row {r} (query {q[r]}) pos {c}: "
            f"gpu idx {gpu_idx[r, c]} d2 {g64[r, c]!r} vs oracle idx {ref_idx[r, c]} d2 {ref_d2[r, c]!r}")
    # 2) float32 distances within 2 ulp of the float64 value of the same pair
    ulp = np.spacing(np.abs(g64).astype(np.float32)).astype(np.float64)
    err = np.abs(gpu_d2.astype(np.float64) - g64)
    badd = err > D2_ULPS * ulp
    if badd.any():
        r, c = np.argwhere(badd)[0]
        raise AssertionError(f"kNN d2 off by {err[r, c] / ulp[r, c]:.2f} ulp at row {r} pos {c}: "
                             f"{gpu_d2[r, c]!r} vs {g64[r, c]!r}")
    # 3) no duplicates within a row
    s = np.sort(gpu_idx, axis=1)
    dup = (s[:, 1:] == s[:, :-1]).any(axis=1)
    assert not dup.any(), f"duplicate neighbour in row {int(np.argmax(dup))}"


def check_canonical(labels):
    lab = np.asarray(labels).astype(np.int64)
    n = lab.shape[0]
    assert lab.min() >= 0 and lab.max() < n, "label out of range"
    i = np.arange(n)
    assert (lab <= i).all(), "a label is larger than its point index"
    assert (lab[lab] == lab).all(), "a label is not its own group's label"


def check_fof(gpu_labels, strict, loose):
    g = np.asarray(gpu_labels).astype(np.int64)
    s = np.asarray(strict).astype(np.int64)
    lo = np.asarray(loose).astype(np.int64)
    check_canonical(g)
    if np.array_equal(s, lo):
        if not np.array_equal(g, s):
            bad = np.nonzero(g != s)[0]
            raise AssertionError(f"FoF labels differ at {bad.size} points; first {bad[0]}: "
                                 f"gpu {g[bad[0]]} oracle {s[bad[0]]}")
        return
    # every strict group maps to one GPU group
    assert np.array_equal(g[s], g), "a strict (d2 <= b^2(1-1e-6)) group is split by the GPU labels"
    # every GPU group lies inside one loose group
    assert np.array_equal(lo[g], lo), "a GPU group spans two loose (d2 <= b^2(1+1e-6)) groups"
