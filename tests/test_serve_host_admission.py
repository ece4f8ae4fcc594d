"""Admission, memory accounting and eviction of serve.Server on the host, with
CUDA streams, events and trees replaced by fakes (no GPU): the budget is never
exceeded, repeated sets reuse their resident tree, the least recently used idle
tree is the one evicted, and a request larger than the budget raises."""
import contextlib

import pytest


@pytest.fixture
def fake_serve(monkeypatch):
    torch = pytest.importorskip("torch")
    from paper_2604_05885_gb300 import serve

    class FakeEvent:
        clock = [0]

        def __init__(self, enable_timing=False):
            self.t, self.polls = None, 0

        def record(self, stream=None):
            FakeEvent.clock[0] += 1
            self.t = FakeEvent.clock[0]

        def query(self):  # the work behind an event completes on its second poll
            self.polls += 1
            return self.polls >= 2

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return float(other.t - self.t)

    built = []

    class FakeTree:
        def __init__(self, pts, periodic_L, params, ws, stream=None):
            built.append(int(pts.shape[0]))

        def knn(self, k, out=None, stream=None):
            return out

        def fof(self, b, out=None, stream=None):
            return out

    monkeypatch.setattr(torch.cuda, "Stream", lambda device=None: object())
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: None)
    monkeypatch.setattr(serve, "Tree", FakeTree)

    def payload(set_id, n, stream):
        return torch.zeros((n, 3), dtype=torch.float32)

    return serve, payload, built


def _tree_cost(serve, n):
    s = serve.Server.__new__(serve.Server)
    s.params = None
    return s._tree_bytes(n) + n * 12


def test_lru_eviction_and_budget(fake_serve):
    serve, payload, built = fake_serve
    n = 1000
    out = n * 8 * 8  # kNN k = 8 outputs
    budget = 2 * _tree_cost(serve, n) + out  # two resident trees and one request's outputs
    srv = serve.Server(payload, n_lanes=1, hbm_budget=budget, device="cpu")
    R = serve.Request
    seq = [0, 1, 0, 2, 0, 1]  # set ids in arrival order
    reqs = [R(i, sid, n, "knn", 8, t_arrival=0.0) for i, sid in enumerate(seq)]
    srv.run(reqs, realtime=False, poll_sleep=0.0)
    assert all(r.t_done is not None for r in reqs)
    assert srv.peak_used <= budget
    # 0 and 1 built; 0 hit; 2 needs room: 1 is the least recently used idle tree;
    # 0 hit again; 1 is rebuilt and evicts 2 (0 was used more recently)
    assert [r.hit for r in reqs] == [False, False, True, False, True, False]
    assert srv.stats["evictions"] == 2 and srv.stats["builds"] == 4 and srv.stats["hits"] == 2
    assert list(srv.resident) == [0, 1]
    assert len(built) == 4


def test_request_larger_than_budget_raises(fake_serve):
    serve, payload, _ = fake_serve
    srv = serve.Server(payload, n_lanes=2, hbm_budget=_tree_cost(serve, 1000) // 2, device="cpu")
    with pytest.raises(RuntimeError, match="more than the budget"):
        srv.run([serve.Request(0, 0, 1000, "fof", b=0.01)], realtime=False, poll_sleep=0.0)


def test_busy_tree_is_not_evicted_and_requests_wait(fake_serve):
    serve, payload, built = fake_serve
    n = 1000
    budget = 3 * _tree_cost(serve, n) + 4 * n * 8 * 8
    srv = serve.Server(payload, n_lanes=4, hbm_budget=budget, device="cpu")
    R = serve.Request
    reqs = [R(i, i % 2, n, "knn", 8) for i in range(8)]  # two sets, four lanes
    srv.run(reqs, realtime=False, poll_sleep=0.0)
    assert all(r.t_done is not None for r in reqs)
    assert srv.peak_used <= budget
    # a set's tree serves one request at a time, so each set is built once and reused
    assert srv.stats["builds"] == 2 and srv.stats["hits"] == 6 and srv.stats["evictions"] == 0
    assert srv.stats["max_inflight"] == 2


def test_invalid_requests_are_rejected_before_any_work(fake_serve):
    serve, payload, built = fake_serve
    srv = serve.Server(payload, n_lanes=2, hbm_budget=1e12, device="cpu")
    R = serve.Request
    for bad in (R(0, 0, 1000, "knn", 64), R(1, 1, 10, "knn", 16), R(2, 2, 1000, "knn", 0),
                R(3, 3, 1000, "sort")):
        with pytest.raises(ValueError):
            srv.run([R(9, 9, 1000, "knn", 8), bad], realtime=False, poll_sleep=0.0)
    assert built == []  # nothing was started
