"""CPU model of the fine-bin key sort (the device's bucket path, restated in
numpy): fine bins of the top F key bits (F chosen as the library does, about 32
keys per bin), keys scattered into their bins in an arbitrary order, each bin
sorted by (key, original index).  The concatenation must be the oracle's stable
order for every input -- the path's correctness argument, independent of the GPU
(which tests/test_gpu_tree.py checks bit for bit)."""
import numpy as np
import pytest

import oracle
import workloads

BUCKET_MIN_N = 1 << 16
MAX_FINE_BITS = 24
BIN_WARP_MAX = 128     # bins sorted by one warp in registers; larger ones by a block
BIN_LIMIT = 2048       # above this, the device takes the LSD radix passes instead


def fine_bits(n):
    f = 1
    while f < MAX_FINE_BITS and (n >> (f + 1)) >= 32:
        f += 1
    return f


def bucket_model(keys, rng):
    n = len(keys)
    f = fine_bits(n)
    shift = np.uint64(63 - f)
    bins = (keys >> shift).astype(np.int64)
    counts = np.bincount(bins, minlength=1 << f)
    if counts.max() > BIN_LIMIT:
        return None, counts
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    # scatter: every key to its bin, in an arbitrary order within the bin
    order = rng.permutation(n)
    slot = np.empty(n, np.int64)
    cursor = starts.copy()
    for i in order:
        slot[i] = cursor[bins[i]]
        cursor[bins[i]] += 1
    kb = np.empty(n, np.uint64)
    vb = np.empty(n, np.int64)
    kb[slot] = keys
    vb[slot] = np.arange(n)
    # per-bin sort by (key, original index)
    out_k = np.empty(n, np.uint64)
    out_v = np.empty(n, np.int64)
    for b in np.nonzero(counts)[0]:
        s, e = starts[b], starts[b] + counts[b]
        o = np.lexsort((vb[s:e], kb[s:e]))
        out_k[s:e] = kb[s:e][o]
        out_v[s:e] = vb[s:e][o]
    return (out_k, out_v), counts


def _sets():
    x_dup = workloads.uniform(1 << 16, 31)
    x_dup[100:700] = x_dup[100]
    x_blob = workloads.uniform(1 << 16, 32)
    x_blob[:1500] = workloads.clip_unit(np.random.default_rng(3).normal(0.4, 5e-5, (1500, 3)))
    x_heavy = workloads.uniform(1 << 16, 33)
    x_heavy[:4000] = x_heavy[5]
    return [("uniform", workloads.uniform(1 << 16, 30), 1.0, True),
            ("duplicates", x_dup, 0.0, True),
            ("dense-blob", x_blob, 0.0, True),
            ("heavy-bin", x_heavy, 1.0, False),
            ("zeldovich-48", workloads.zeldovich(48, 5), 1.0, True)]


@pytest.mark.parametrize("name,x,L,bucket", _sets(), ids=[s[0] for s in _sets()])
def test_bucket_model_gives_the_stable_order(name, x, L, bucket):
    keys = oracle.morton_keys(x, L)
    res, counts = bucket_model(keys, np.random.default_rng(7))
    assert (res is not None) == bucket
    if res is None:
        return
    sk, perm = oracle.zsort(keys)
    assert np.array_equal(res[0], sk)
    assert np.array_equal(res[1], perm)
    if name == "dense-blob":
        assert counts.max() > BIN_WARP_MAX  # a bin for the block sort


def test_fine_bits_give_about_32_keys_per_bin():
    for n in (BUCKET_MIN_N, 100000, 1 << 20, 1 << 24, 1 << 27, (1 << 31) - 1):
        f = fine_bits(n)
        assert 1 <= f <= MAX_FINE_BITS
        if f < MAX_FINE_BITS:
            assert 32 <= n / (1 << f) < 128
