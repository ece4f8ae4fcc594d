"""Host-side pieces of serving and batching that need no GPU: the latency
summary, and the shape of the synthetic request stream and batched sets."""
import math

import numpy as np
import pytest

import workloads


def test_latency_summary():
    pytest.importorskip("torch")
    from paper_2604_05885_gb300.serve import Request, latency_summary
    reqs = []
    for i in range(100):
        r = Request(i, i, 1000 + i, "knn", 8, t_arrival=0.01 * i)
        r.t_done = r.t_arrival + 0.001 * (i + 1)  # latencies 1..100 ms
        reqs.append(r)
    s = latency_summary(reqs)
    assert s["p50_ms"] == pytest.approx(50.5)
    assert s["p99_ms"] == pytest.approx(99.01)
    assert s["max_ms"] == pytest.approx(100.0)
    span = reqs[-1].t_done - reqs[0].t_arrival
    assert s["requests_per_s"] == pytest.approx(100 / span)
    assert s["particles_per_s"] == pytest.approx(sum(r.n for r in reqs) / span)


def test_serving_stream_shape():
    reqs = workloads.serving_stream(4000, 5, n_lo=1e4, n_hi=2 ** 24, repeat_frac=0.3, rate_hz=50.0)
    t = np.array([r["t_arrival"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(len(reqs) / t[-1] - 50.0) < 5.0  # Poisson rate
    n = np.array([r["n"] for r in reqs])
    assert n.min() >= 1e4 and n.max() < 2 ** 24
    # log-uniform sizes: the median of log n sits near the middle of the range
    assert abs(np.median(np.log(n)) - 0.5 * (math.log(1e4) + math.log(2 ** 24))) < 0.5
    seen, repeats = set(), 0
    for r in reqs:
        repeats += r["set_id"] in seen
        seen.add(r["set_id"])
    assert 0.25 < repeats / len(reqs) < 0.35
    for r in reqs:
        assert (r["op"] == "knn" and r["k"] in (8, 16, 32)) or (r["op"] == "fof" and r["b"] > 0)


def test_batched_specs_shape():
    specs = workloads.batched_specs(512, 4)
    n = np.array([s["n"] for s in specs])
    assert n.min() >= 1000 and n.max() < 2e6
    ops = [s["op"] for s in specs]
    assert 0.4 < ops.count("knn") / len(ops) < 0.6
    again = workloads.batched_specs(512, 4)
    assert specs == again  # seeded


def test_lane_assignment_longest_first():
    """Longest-processing-time order, each job to the least-loaded lane: every job
    placed once, and the largest lane load within Graham's bound (4/3 - 1/(3m))
    of the optimum, which brute force gives on small inputs."""
    import itertools
    pytest.importorskip("torch")
    from paper_2604_05885_gb300 import assign_lanes
    rng = np.random.default_rng(3)
    for trial in range(60):
        nj, m = int(rng.integers(1, 8)), int(rng.integers(1, 4))
        sizes = [int(v) for v in rng.integers(1, 50, nj)]
        lane_of = assign_lanes(sizes, m)
        assert len(lane_of) == nj and all(0 <= q < m for q in lane_of)
        load = [0] * m
        for j, q in enumerate(lane_of):
            load[q] += sizes[j]
        opt = min(max(sum(sizes[j] for j in range(nj) if a[j] == q) for q in range(m))
                  for a in itertools.product(range(m), repeat=nj))
        assert max(load) <= (4 / 3 - 1 / (3 * m)) * opt + 1e-9
    # equal jobs go round the lanes in job order; the largest job takes lane 0
    assert assign_lanes([5] * 6, 3) == [0, 1, 2, 0, 1, 2]
    assert assign_lanes([1, 9, 3], 2)[1] == 0
