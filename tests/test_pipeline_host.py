"""Event ordering of pipeline.HostPipeline on the host, with CUDA streams, events
and trees replaced by logging fakes (no GPU).  With two slots, step i's upload
waits for the compute of step i - 2 (the last reader of its input slot), its
compute waits for its own upload and for the download of step i - 2 (the last
reader of its output slot), and its download waits for its compute."""
import contextlib

import pytest


@pytest.fixture
def fake_pipeline(monkeypatch):
    torch = pytest.importorskip("torch")
    from paper_2604_05885_gb300 import pipeline

    log = []

    class FakeStream:
        def __init__(self, device=None):
            self.name = None

        def wait_event(self, ev):
            log.append((self.name, "wait", ev.tag))

        def synchronize(self):
            pass

    class FakeEvent:
        def __init__(self, *a, **k):
            self.tag = None

        def record(self, stream):
            self.tag = (stream.name, sum(1 for e in log if e[1] == "record" and e[0] == stream.name))
            log.append((stream.name, "record", self.tag))

    class FakeTree:
        def __init__(self, pts, periodic_L, params, ws, stream=None):
            log.append((stream.name, "build", None))

        def knn(self, k, out=None, stream=None):
            log.append((stream.name, "knn", None))

        def fof(self, b, out=None, stream=None):
            log.append((stream.name, "fof", None))

    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(pipeline, "Tree", FakeTree)
    return torch, pipeline, log


def test_double_buffer_dependencies(fake_pipeline):
    torch, pipeline, log = fake_pipeline
    n, k = 64, 4
    pl = pipeline.HostPipeline(n, k, 0.01, 1.0, device="cpu", depth=2)
    pl.s_up.name, pl.s_comp.name, pl.s_down.name = "up", "comp", "down"
    host = [(torch.rand(n, 3), torch.empty(n, k, dtype=torch.int32), torch.empty(n, k), torch.empty(n, dtype=torch.int32))
            for _ in range(5)]
    for h in host:
        pl.submit(*h)
    # per stream, the i-th record belongs to step i
    waits = {}
    step = {"up": -1, "comp": -1, "down": -1}
    pending = {"up": [], "comp": [], "down": []}
    for s, what, tag in log:
        if what == "wait":
            pending[s].append(tag)
        elif what == "record":
            step[s] += 1
            waits[(s, step[s])] = sorted(pending[s])
            pending[s] = []
    for i in range(5):
        up = [("comp", i - 2)] if i >= 2 else []
        comp = sorted([("up", i)] + ([("down", i - 2)] if i >= 2 else []))
        assert waits[("up", i)] == up
        assert waits[("comp", i)] == comp
        assert waits[("down", i)] == [("comp", i)]
    # each step runs exactly one build, one kNN and one FoF on the compute stream
    assert [w for s, w, _ in log if s == "comp" and w in ("build", "knn", "fof")] == ["build", "knn", "fof"] * 5
