"""Autotuner for batched jobs: picks the lane count and the tree parameters
(leaf capacity, super-node grouping, coarsening target) of a Batch by timing
candidate configurations on the batch itself, then a leaf capacity per set-size
class (small, medium, large sets), and caches the winner per batch signature
(device, job count, size histogram, operation mix) in a JSON file.  Results
never depend on these choices, only the time does.  The leaf capacity is also
the number of query points a LeafToLeaf warp takes at once (one warp per leaf).
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import Batch

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "jzt_gb300", "autotune.json")
LANES = (4, 8, 16)
PARAMS = ({}, {"ngr": 16}, {"n_target": 250}, {"nmax0": 24})
CLASS_BOUNDS = (1 << 14, 1 << 18)  # size classes: N < 2^14, N < 2^18, larger
LEAF_CAPS = (16, 24, 32)


def size_class(n: int) -> int:
    return 0 if n < CLASS_BOUNDS[0] else (1 if n < CLASS_BOUNDS[1] else 2)


def leaf_cap_fn(caps):
    """N -> the leaf capacity of N's size class (0: the batch parameters')."""
    caps = list(caps)
    return lambda n: caps[size_class(int(n))]


def signature(sets) -> str:
    hist = {}
    for st in sets:
        b = int(math.log2(max(1, int(st["points"].shape[0]))))
        key = f"{st['op']}{int(st.get('k', 0))}:{b}"
        hist[key] = hist.get(key, 0) + 1
    name = torch.cuda.get_device_name()
    return f"{name}|{len(sets)}|" + ",".join(f"{k}={v}" for k, v in sorted(hist.items()))


def _time(batch: Batch, reps: int) -> float:
    batch.run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        batch.run()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(sets, cache: str | None = DEFAULT_CACHE, lanes=LANES, params=PARAMS, reps: int = 3, log=None,
         leaf_caps=LEAF_CAPS):
    """Returns (n_lanes, params, caps) for these sets, from the cache or by timing;
    caps[c] is the leaf capacity of size class c (0 = that of params), for
    Batch(..., nmax0_of=leaf_cap_fn(caps))."""
    key = signature(sets)
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            table = json.load(fh)
    if key in table:
        e = table[key]
        return e["n_lanes"], e["params"], e.get("leaf_caps", [0, 0, 0])
    best = None
    for nl in lanes:
        for pr in params:
            b = Batch(sets, n_lanes=nl, params=pr or None, graph=True)
            ms = _time(b, reps)
            if log:
                log(f"autotune lanes={nl} params={pr} {ms:.2f} ms")
            if best is None or ms < best[0]:
                best = (ms, nl, pr)
            del b
            torch.cuda.empty_cache()
    # then one leaf capacity per size class present, one class at a time
    ms_best, nl, pr = best
    caps = [0, 0, 0]
    for c in sorted({size_class(int(st["points"].shape[0])) for st in sets}):
        for v in leaf_caps:
            if v == int(pr.get("nmax0", 32)):
                continue  # the class already runs at this capacity
            trial = list(caps)
            trial[c] = v
            b = Batch(sets, n_lanes=nl, params=pr or None, graph=True, nmax0_of=leaf_cap_fn(trial))
            ms = _time(b, reps)
            if log:
                log(f"autotune leaf capacities {trial} {ms:.2f} ms")
            if ms < ms_best:
                ms_best, caps = ms, trial
            del b
            torch.cuda.empty_cache()
    best = (ms_best, nl, pr)
    table[key] = {"n_lanes": best[1], "params": best[2], "leaf_caps": caps, "ms": best[0]}
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(table, fh, indent=1)
        os.replace(tmp, cache)
    return best[1], best[2], caps
