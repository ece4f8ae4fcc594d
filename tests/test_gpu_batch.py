"""Batched jobs (jzt_batch_run): every job's result equals the one-call result
of the same set (jzt_knn / jzt_fof), eagerly and replayed from a CUDA graph,
and small jobs also match the oracle."""
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


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("n_lanes", [1, 5])
def test_batch_matches_one_call(graph, n_lanes):
    import paper_2604_05885_gb300 as jzt
    sets = _sets()
    b = jzt.Batch(sets, n_lanes=n_lanes, graph=graph)
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


def test_batch_small_jobs_match_oracle():
    import paper_2604_05885_gb300 as jzt
    sets = [s for s in _sets(16, 9) if s["points"].shape[0] <= 3000]
    b = jzt.Batch(sets, n_lanes=3, graph=True)
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
