"""Failure detection on the GPU without a fault: the library's bounded waits are
made to run out (an mbarrier phase nobody completes, a published word nobody
sets); each ends with JZT_ERR_TIMEOUT in the status word, within a bounded time,
and the context stays usable for the next call."""
import time

import numpy as np
import pytest
import torch

import oracle
import workloads
from tests import parity
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which,limit", [(0, 1024), (1, 1 << 16)])
def test_bounded_wait_reports_timeout(which, limit):
    import paper_2604_05885_gb300 as jzt
    ws = jzt.alloc_workspace(1000)
    s = torch.cuda.current_stream()
    t0 = time.time()
    rc = jzt.lib.jzt_selftest_wait(which, limit, ws.data_ptr(), ws.numel(), s.cuda_stream, None)
    assert rc == jzt.JZT_ERR_TIMEOUT
    assert time.time() - t0 < 30.0
    # the context is still usable: a normal call on the same workspace succeeds and is exact
    x = workloads.uniform(1000, 3)
    idx, d2 = jzt.knn(to_dev(x), 8, 1.0, workspace=ws)
    ri, rd = oracle.knn_brute(x, 8, 1.0)
    parity.check_knn(x, np.arange(1000), idx.cpu().numpy(), d2.cpu().numpy(), ri, rd, 1.0)


def test_selftest_rejects_bad_arguments():
    import paper_2604_05885_gb300 as jzt
    ws = jzt.alloc_workspace(1000)
    assert jzt.lib.jzt_selftest_wait(2, 10, ws.data_ptr(), ws.numel(), None, None) == jzt.JZT_ERR_INVALID
    assert jzt.lib.jzt_selftest_wait(0, 0, ws.data_ptr(), ws.numel(), None, None) == jzt.JZT_ERR_INVALID
