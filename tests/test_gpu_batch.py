"""Batched jobs (jzt_batch_run, and jzt_batch_run_queue with the kNN LeafToLeaf
of all jobs in persistent launches over a device work queue): every job's result
equals the one-call result of the same set (jzt_knn / jzt_fof), eagerly and
replayed from a CUDA graph, and small jobs also match the oracle."""
import numpy as np
import pytest

import oracle
import workloads
from tests import parity
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _sets(n_sets=24, seed=5):
    rng = np.random.default_rng(seed)
    sets = []
    for j in range(n_sets):
        n = int(np.exp(rng.uniform(np.log(50), np.log(60000))))
        L = 1.0 if j % 3 else 0.0
        x = workloads.clustered(n, 1000 + j, n_blobs=max(1, n // 4096 + 1))
        if j % 2 == 0:
            sets.append(dict(points=to_dev(x), host=x, op="knn", k=int(min(n, rng.choice([1, 8, 16, 32]))),
                             periodic_L=L))
        else:
            sets.append(dict(points=to_dev(x), host=x, op="fof",
                             b=float(rng.choice([0.15, 0.2, 0.5])) * workloads.mean_spacing(n), periodic_L=L))
    return sets


@pytest.mark.parametrize("queue", [False, True])
@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("n_lanes", [1, 5])
def test_batch_matches_one_call(graph, n_lanes, queue):
    import paper_2604_05885_gb300 as jzt
    sets = _sets()
    if queue:  # every k class and both boundaries in the queue; one k > 32 job on its lane
        x = workloads.clustered(4000, 77, n_blobs=2)
        sets += [dict(points=to_dev(x), host=x, op="knn", k=k, periodic_L=L)
                 for k, L in ((3, 0.0), (5, 1.0), (12, 0.0), (40, 1.0))]
    b = jzt.Batch(sets, n_lanes=n_lanes, graph=graph, queue=queue)
    for _ in range(2):
        b.run()
        assert b.statuses() == [0] * len(sets)
        for st, out in zip(sets, b.outputs):
            if st["op"] == "knn":
                ri, rd = jzt.knn(st["points"], st["k"], st["periodic_L"])
                assert np.array_equal(out[0].cpu().numpy(), ri.cpu().numpy())
                assert np.array_equal(out[1].cpu().numpy(), rd.cpu().numpy())
            else:
                rl = jzt.fof(st["points"], st["b"], st["periodic_L"])
                assert np.array_equal(out.cpu().numpy(), rl.cpu().numpy())


@pytest.mark.parametrize("queue", [False, True])
def test_batch_small_jobs_match_oracle(queue):
    import paper_2604_05885_gb300 as jzt
    sets = [s for s in _sets(16, 9) if s["points"].shape[0] <= 3000]
    b = jzt.Batch(sets, n_lanes=3, graph=True, queue=queue)
    b.run()
    assert b.statuses() == [0] * len(sets)
    for st, out in zip(sets, b.outputs):
        x = st["host"]
        if st["op"] == "knn":
            ri, rd = oracle.knn_brute(x, st["k"], st["periodic_L"])
            parity.check_knn(x, np.arange(len(x)), out[0].cpu().numpy(), out[1].cpu().numpy(), ri, rd,
                             st["periodic_L"])
        else:
            s, lo = oracle.fof_bracket(x, st["b"], st["periodic_L"], cells=False)
            parity.check_fof(out.cpu().numpy(), s, lo)


def test_batch_rejects_bad_job():
    import paper_2604_05885_gb300 as jzt
    x = to_dev(workloads.uniform(10, 1))
    with pytest.raises(jzt.JztError):
        jzt.Batch([dict(points=x, op="knn", k=11)], n_lanes=1, graph=False)


def test_queue_rejects_shared_workspace_and_small_scratch():
    import ctypes
    import torch
    import paper_2604_05885_gb300 as jzt
    x = to_dev(workloads.uniform(500, 2))
    idx = torch.empty((500, 8), dtype=torch.int32, device="cuda")
    d2 = torch.empty((500, 8), dtype=torch.float32, device="cuda")
    jobs = (jzt.Job * 2)()
    for J in jobs:
        J.d_xyz, J.n, J.periodic_L, J.op, J.k, J.lane = x.data_ptr(), 500, 1.0, jzt.JZT_OP_KNN, 8, 0
        J.d_idx, J.d_dist2 = idx.data_ptr(), d2.data_ptr()
    ws = jzt.alloc_workspace(500, 8)
    ptrs = (ctypes.c_void_p * 2)(ws.data_ptr(), ws.data_ptr())
    sizes = (ctypes.c_size_t * 2)(ws.numel(), ws.numel())
    streams = (ctypes.c_void_p * 1)(torch.cuda.current_stream().cuda_stream)
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    qb = ctypes.c_size_t(0)
    assert jzt.lib.jzt_batch_queue_bytes(2, ctypes.byref(qb)) == 0
    scratch = torch.empty(int(qb.value), dtype=torch.uint8, device="cuda")
    rc = jzt.lib.jzt_batch_run_queue(jobs, 2, None, ptrs, sizes, streams, 1, None, scratch.data_ptr(),
                                     scratch.numel(), st.data_ptr())
    assert rc == jzt.JZT_ERR_INVALID and b"workspace of its own" in jzt.lib.jzt_last_error()
    rc = jzt.lib.jzt_batch_run_queue(jobs, 1, None, ptrs, sizes, streams, 1, None, scratch.data_ptr(), 16,
                                     st.data_ptr())
    assert rc == jzt.JZT_ERR_WORKSPACE


@pytest.mark.parametrize("queue", [False, True])
def test_per_job_leaf_capacity_leaves_results_unchanged(queue):
    """Each job may carry its own leaf capacity (chosen by size class); the rows and
    labels stay those of one call per set with the default tree."""
    import paper_2604_05885_gb300 as jzt
    from paper_2604_05885_gb300 import autotune
    sets = _sets(12, 21)
    b = jzt.Batch(sets, n_lanes=3, graph=True, queue=queue, nmax0_of=autotune.leaf_cap_fn([8, 16, 24]))
    assert sorted(set(b.job_nmax0)) == sorted({autotune.leaf_cap_fn([8, 16, 24])(int(s["points"].shape[0]))
                                                for s in sets})
    b.run()
    assert b.statuses() == [0] * len(sets)
    for st, out in zip(sets, b.outputs):
        if st["op"] == "knn":
            ri, rd = jzt.knn(st["points"], st["k"], st["periodic_L"])
            assert np.array_equal(out[0].cpu().numpy(), ri.cpu().numpy())
            assert np.array_equal(out[1].cpu().numpy(), rd.cpu().numpy())
        else:
            assert np.array_equal(out.cpu().numpy(), jzt.fof(st["points"], st["b"], st["periodic_L"]).cpu().numpy())
