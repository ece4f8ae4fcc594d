"""Autotuner host logic with the batch and its timing faked (no GPU): the fastest
(lanes, parameters) pair wins, the winner is cached per batch signature, and a
cached entry is returned without timing anything."""
import json

import numpy as np
import pytest


def _sets(sizes_ops):
    return [{"points": np.zeros((n, 3), np.float32), "op": op, "k": k} for n, op, k in sizes_ops]


@pytest.fixture
def fake_tuner(monkeypatch):
    torch = pytest.importorskip("torch")
    from paper_2604_05885_gb300 import autotune

    class FakeBatch:
        def __init__(self, sets, n_lanes, params=None, graph=True, nmax0_of=None):
            self.n_lanes, self.params = n_lanes, dict(params or {})
            # the leaf capacity of each size class, read at one size per class
            self.caps = tuple(nmax0_of(n) if nmax0_of else 0 for n in (1000, 100_000, 1_000_000))

    cost = {}  # (lanes, sorted params) -> ms; anything unlisted is slow
    # (leaf capacity per size class) -> ms for the per-class trials; unlisted: slow

    def fake_time(batch, reps):
        if batch.caps != (0, 0, 0):
            return cost.get(("caps", batch.caps), 100.0)
        return cost.get((batch.n_lanes, tuple(sorted(batch.params.items()))), 100.0)

    monkeypatch.setattr(autotune, "Batch", FakeBatch)
    monkeypatch.setattr(autotune, "_time", fake_time)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a, **k: "FakeGPU")
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda: None)
    return autotune, cost


def test_fastest_configuration_wins_and_is_cached(fake_tuner, tmp_path):
    autotune, cost = fake_tuner
    cost[(8, (("n_target", 250),))] = 3.0
    cost[(16, ())] = 4.0
    sets = _sets([(1000, "knn", 8), (3000, "fof", 0), (70000, "knn", 16)])
    cache = str(tmp_path / "tune.json")
    seen = []
    lanes, params, caps = autotune.tune(sets, cache=cache, log=seen.append)
    assert (lanes, params, caps) == (8, {"n_target": 250}, [0, 0, 0])
    # every (lanes, params) candidate timed once, then 16 and 24 for the two size classes present
    assert len(seen) == len(autotune.LANES) * len(autotune.PARAMS) + 2 * 2
    table = json.load(open(cache))
    entry = table[autotune.signature(sets)]
    assert entry["n_lanes"] == 8 and entry["params"] == {"n_target": 250} and entry["ms"] == 3.0


def test_cached_entry_is_used_without_timing(fake_tuner, tmp_path, monkeypatch):
    autotune, cost = fake_tuner
    sets = _sets([(5000, "knn", 16), (5000, "knn", 16)])
    cache = str(tmp_path / "tune.json")
    cost[(4, (("ngr", 16),))] = 1.0
    first = autotune.tune(sets, cache=cache)

    def no_timing(batch, reps):
        raise AssertionError("a cached signature must not be timed again")

    monkeypatch.setattr(autotune, "_time", no_timing)
    assert autotune.tune(sets, cache=cache) == first == (4, {"ngr": 16}, [0, 0, 0])


def test_signature_groups_by_operation_and_size_octave(fake_tuner):
    autotune, _ = fake_tuner
    a = autotune.signature(_sets([(1100, "knn", 8), (3000, "fof", 0)]))
    b = autotune.signature(_sets([(1900, "knn", 8), (2100, "fof", 0)]))     # same octaves
    c = autotune.signature(_sets([(1100, "knn", 16), (3000, "fof", 0)]))    # another k
    d = autotune.signature(_sets([(2100, "knn", 8), (3000, "fof", 0)]))     # another octave
    e = autotune.signature(_sets([(1100, "knn", 8), (3000, "fof", 0), (3000, "fof", 0)]))  # more jobs
    assert a == b
    assert len({a, c, d, e}) == 4
    assert a.startswith("FakeGPU|2|")


def test_leaf_capacity_per_size_class(fake_tuner, tmp_path):
    """After the grid search the tuner tries a leaf capacity per size class, one class at
    a time, keeping what is faster; size classes follow N."""
    autotune, cost = fake_tuner
    cost[(16, ())] = 3.0
    cost[("caps", (16, 0, 0))] = 2.0      # small sets faster with 16-point leaves
    cost[("caps", (16, 0, 24))] = 2.5     # slower than the kept (16, 0, 0)
    sets = _sets([(1000, "knn", 8), (500_000, "fof", 0)])
    lanes, params, caps = autotune.tune(sets, cache=str(tmp_path / "t.json"))
    assert (lanes, params, caps) == (16, {}, [16, 0, 0])
    fn = autotune.leaf_cap_fn(caps)
    assert (fn(100), fn((1 << 14) - 1), fn(1 << 14), fn(1 << 20)) == (16, 16, 0, 0)
    assert [autotune.size_class(n) for n in (1, (1 << 14) - 1, 1 << 14, (1 << 18) - 1, 1 << 18)] == [0, 0, 1, 1, 2]
