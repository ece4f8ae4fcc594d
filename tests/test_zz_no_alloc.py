"""The allocation-free kNN entry point (jzt_knn_noalloc).

It serves callers that may not allocate device memory (code inside a host
framework that owns every device allocation, real-time paths that must not
enter the allocator): its scratch space is a fixed array inside the library.
This file calls it through the C ABI and checks

* its rows against the all-pairs oracle under the kNN parity rule, on two calls
  in a row with different sets (a larger clustered one, then a smaller one of
  another seed, so stale scratch from the first call would show in the second),
  with and without the status read-back (info = NULL);
* that a set which overflows the fixed array reports JZT_ERR_CAPACITY when the
  status is read, and leaves rows of index -1 / distance NaN when it is not;
* that oversized problems are refused with a clear error.

It lives in a file of its own that is collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from tests import parity
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu

MAX_N = 65536


def _noalloc(jzt, xt, n, k, L, with_info=True):
    """(rc, info code or None, idx, d2) of one call on the current stream."""
    import torch
    idx = torch.full((n, k), 7, dtype=torch.int32, device=xt.device)
    d2 = torch.full((n, k), 7.0, dtype=torch.float32, device=xt.device)
    info = jzt.StatusInfo()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = jzt.lib.jzt_knn_noalloc(ctypes.c_void_p(xt.data_ptr()), n, k, L, ctypes.c_void_p(idx.data_ptr()),
                                 ctypes.c_void_p(d2.data_ptr()), stream,
                                 ctypes.byref(info) if with_info else None)
    torch.cuda.synchronize()
    return rc, (info.code if with_info else None), idx.cpu().numpy(), d2.cpu().numpy()


def _oracle_check(x, k, L, idx, d2):
    ri, rd = oracle.knn_brute(x, k, L)
    parity.check_knn(x, np.arange(len(x)), idx, d2, ri, rd, L)


@pytest.mark.parametrize("with_info", [True, False])
def test_noalloc_matches_oracle_on_consecutive_calls(with_info):
    import paper_2604_05885_gb300 as jzt
    cases = [(workloads.clustered(MAX_N, 41, n_blobs=16), 32, 1.0),   # the largest N, the largest k
             (workloads.uniform(20011, 42), 16, 0.0),                # then smaller, another seed
             (workloads.clustered(777, 43, n_blobs=2), 5, 1.0)]
    for x, k, L in cases:
        rc, code, idx, d2 = _noalloc(jzt, to_dev(x), len(x), k, L, with_info)
        assert rc == jzt.JZT_OK, (rc, jzt.lib.jzt_last_error())
        assert code in (None, 0)
        _oracle_check(x, k, L, idx, d2)


def test_noalloc_capacity_is_reported_and_rows_are_marked():
    """65536 copies of one point: every leaf sees every other leaf at distance 0,
    so the interaction lists need about 4 M entries, more than the fixed array
    holds.  With the status read the call returns JZT_ERR_CAPACITY; without it the
    rows come back as index -1 / distance NaN.  A normal call afterwards is exact."""
    import paper_2604_05885_gb300 as jzt
    x = np.repeat(workloads.uniform(1, 44), MAX_N, axis=0)
    xt = to_dev(x)
    rc, code, idx, d2 = _noalloc(jzt, xt, MAX_N, 16, 1.0, with_info=True)
    assert rc == jzt.JZT_ERR_CAPACITY and code == jzt.JZT_ERR_CAPACITY
    rc, code, idx, d2 = _noalloc(jzt, xt, MAX_N, 16, 1.0, with_info=False)
    assert rc == jzt.JZT_OK
    assert np.all(idx == -1) and np.all(np.isnan(d2))
    y = workloads.uniform(3000, 45)
    rc, code, idx, d2 = _noalloc(jzt, to_dev(y), 3000, 8, 0.0)
    assert rc == jzt.JZT_OK and code == 0
    _oracle_check(y, 8, 0.0, idx, d2)


def test_noalloc_refuses_oversized_problems():
    import torch
    import paper_2604_05885_gb300 as jzt
    n = MAX_N + 1
    xt = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    out = torch.empty((n, 1), dtype=torch.int32, device="cuda")
    d2 = torch.empty((n, 1), dtype=torch.float32, device="cuda")
    rc = jzt.lib.jzt_knn_noalloc(ctypes.c_void_p(xt.data_ptr()), n, 1, 0.0, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(d2.data_ptr()), None, None)
    assert rc == jzt.JZT_ERR_INVALID
    assert b"65536" in jzt.lib.jzt_last_error()
    x = workloads.uniform(100, 46)
    rc = jzt.lib.jzt_knn_noalloc(ctypes.c_void_p(to_dev(x).data_ptr()), 100, 33, 0.0,
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(d2.data_ptr()), None, None)
    assert rc == jzt.JZT_ERR_UNSUPPORTED
