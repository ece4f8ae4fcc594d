"""The allocation-free kNN entry point (jzt_knn_noalloc).

It exists for callers that may not allocate device memory (a host framework
that owns all device allocations, code running during stream capture): its
scratch space is a fixed array inside the library.  This test calls it through
the C ABI twice in a row and checks each result against the ordinary entry
point jzt_knn (which uses a caller workspace) under the kNN parity rule, and
checks that oversized problems are refused with a clear error.  It lives in a
file of its own that is collected last.
"""
import ctypes

import numpy as np
import pytest

import workloads
from tests import parity
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu

MAX_N = 65536


def _noalloc(jzt, xt, n, k, L):
    import torch
    idx = torch.empty((n, k), dtype=torch.int32, device=xt.device)
    d2 = torch.empty((n, k), dtype=torch.float32, device=xt.device)
    info = jzt.StatusInfo()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = jzt.lib.jzt_knn_noalloc(ctypes.c_void_p(xt.data_ptr()), n, k, L, ctypes.c_void_p(idx.data_ptr()),
                                 ctypes.c_void_p(d2.data_ptr()), stream, ctypes.byref(info))
    assert rc == jzt.JZT_OK, (rc, jzt.lib.jzt_last_error())
    assert info.code == 0
    return idx.cpu().numpy(), d2.cpu().numpy()


@pytest.mark.parametrize("n,k,L,seed", [(20000, 16, 1.0, 41), (MAX_N, 32, 0.0, 42), (777, 5, 1.0, 43)])
def test_noalloc_matches_workspace_entry_point(n, k, L, seed):
    import paper_2604_05885_gb300 as jzt
    x = workloads.clustered(n, seed, n_blobs=8) if n > 1000 else workloads.uniform(n, seed)
    xt = to_dev(x)
    ref_idx, ref_d2 = jzt.knn(xt, k, L)  # jzt_knn with its own workspace
    ref_idx = ref_idx.cpu().numpy()
    ref_d2 = ref_d2.cpu().numpy().astype(np.float64)
    q = np.arange(n)
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        idx, d2 = _noalloc(jzt, xt, n, k, L)
        parity.check_knn(x, q, idx, d2, ref_idx, ref_d2, L)


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
