"""HostPipeline (transfers overlapped with compute across steps): every step's
host outputs equal one jzt_knn / jzt_fof call on that step's points."""
import numpy as np
import pytest
import torch

import workloads
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("depth", [1, 2])
def test_pipeline_steps_equal_one_call(depth):
    import paper_2604_05885_gb300 as jzt
    from paper_2604_05885_gb300.pipeline import HostPipeline
    n, k, L = 30000, 12, 1.0
    b = 0.3 * workloads.mean_spacing(n)
    sets = [workloads.clustered(n, 300 + i, n_blobs=9) for i in range(5)]
    pipe = HostPipeline(n, k, b, L, depth=depth)
    outs = []
    for x in sets:
        xh = torch.from_numpy(x).pin_memory()
        oh = (torch.empty((n, k), dtype=torch.int32).pin_memory(), torch.empty((n, k), dtype=torch.float32).pin_memory(),
              torch.empty(n, dtype=torch.int32).pin_memory())
        pipe.submit(xh, *oh)
        outs.append((xh, oh))
    pipe.synchronize()
    assert pipe.status()["code"] == 0
    for x, (xh, (ih, dh, lh)) in zip(sets, outs):
        ri, rd = jzt.knn(to_dev(x), k, L)
        rl = jzt.fof(to_dev(x), b, L)
        assert np.array_equal(ih.numpy(), ri.cpu().numpy())
        assert np.array_equal(dh.numpy(), rd.cpu().numpy())
        assert np.array_equal(lh.numpy(), rl.cpu().numpy())
