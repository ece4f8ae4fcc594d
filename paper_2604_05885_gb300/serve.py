"""Request serving for kNN / FoF jobs (no counterpart in the paper: a system
pattern on top of the method; results are those of one jzt_knn / jzt_fof call).

``Server`` is a continuous-batching loop.  Requests wait in a FIFO queue until
their arrival time has passed, a lane (a CUDA stream) is free and their memory
fits in the device-memory budget; every tick admits as many queued requests as
lanes and memory allow, so the work of requests that arrive while others run
overlaps on the GPU.  A request names a point set; the tree built for it stays
resident in its workspace (sized for any k <= 32), so a later request on the
same set runs only the walk.  Resident trees are evicted least-recently-used
when an admission needs their memory.

``PlainServer`` is the one-call-per-request path that the served form is
compared with: the same queue served in arrival order on one stream, each
request a full jzt_knn / jzt_fof call in one preallocated workspace.

Both record, per request, the device time at which its work ended (a CUDA event
read against an event recorded when the run started), so latency = completion
- arrival does not depend on how often the host polls.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import torch

from . import Tree, fof as _fof_call, knn as _knn_call, workspace_bytes

K_MAX = 32


@dataclass
class Request:
    """One kNN (op 'knn', k) or FoF (op 'fof', b) job on point set ``set_id``
    of ``n`` points; ``t_arrival`` is in seconds from the start of the run."""
    rid: int
    set_id: int
    n: int
    op: str
    k: int = 0
    b: float = 0.0
    periodic_L: float = 0.0
    t_arrival: float = 0.0
    # filled by the server
    t_done: float | None = None
    hit: bool = False
    result: object = None
    lane: int = -1
    _event: object = field(default=None, repr=False)  # completion event of the request's work
    _res: object = field(default=None, repr=False)    # the resident tree it runs on
    _pts: object = field(default=None, repr=False)    # its points, while a build needs them


def _check_requests(reqs):
    """Workspaces are sized for k <= K_MAX: reject anything else before any work."""
    for r in reqs:
        if r.op == "knn":
            if not 1 <= int(r.k) <= min(K_MAX, int(r.n)):
                raise ValueError(f"request {r.rid}: k = {r.k} outside 1..min({K_MAX}, n)")
        elif r.op != "fof":
            raise ValueError(f"request {r.rid}: op must be 'knn' or 'fof'")


def _out_bytes(r: Request) -> int:
    return r.n * r.k * 8 if r.op == "knn" else r.n * 4


def _alloc_out(r: Request, dev):
    if r.op == "knn":
        return (torch.empty((r.n, r.k), dtype=torch.int32, device=dev),
                torch.empty((r.n, r.k), dtype=torch.float32, device=dev))
    return torch.empty(r.n, dtype=torch.int32, device=dev)


class _Resident:
    __slots__ = ("tree", "bytes", "busy", "set_id")

    def __init__(self, set_id, tree, nbytes):
        self.set_id = set_id
        self.tree = tree
        self.bytes = nbytes
        self.busy = 0


class Server:
    """Continuous batching over ``n_lanes`` streams with a device-memory budget.

    payload(set_id, n, stream) must return the set's points (contiguous float32
    CUDA tensor n x 3) enqueued on ``stream``.
    """

    def __init__(self, payload, n_lanes: int = 8, hbm_budget: float = 150e9, params=None,
                 device=None, keep_trees: bool = True, keep_results: bool = False):
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.payload = payload
        self.params = params
        self.budget = int(hbm_budget)
        self.keep_trees = keep_trees
        self.keep_results = keep_results
        self.lanes = [torch.cuda.Stream(device=self.dev) for _ in range(max(1, int(n_lanes)))]
        self.lane_busy = [None] * len(self.lanes)
        self.resident: collections.OrderedDict[int, _Resident] = collections.OrderedDict()
        self.used = 0
        self.peak_used = 0
        self.stats = dict(admitted=0, hits=0, evictions=0, builds=0, max_inflight=0)

    # memory ------------------------------------------------------------------
    def _tree_bytes(self, n: int) -> int:
        return workspace_bytes(n, min(K_MAX, n), self.params)

    def _need(self, r: Request) -> int:
        need = _out_bytes(r)
        res = self.resident.get(r.set_id)
        if res is None:
            need += self._tree_bytes(r.n) + r.n * 12
        return need

    def _evict_for(self, need: int, keep_id: int) -> bool:
        while self.used + need > self.budget:
            victim = None
            for sid, res in self.resident.items():  # least recently used first
                if res.busy == 0 and sid != keep_id:
                    victim = sid
                    break
            if victim is None:
                return False
            res = self.resident.pop(victim)
            self.used -= res.bytes
            self.stats["evictions"] += 1
            del res
        return True

    # dispatch ----------------------------------------------------------------
    def _start(self, r: Request, lane: int):
        s = self.lanes[lane]
        res = self.resident.get(r.set_id)
        r.lane = lane
        # device memory comes from the dispatching stream's pool; it is released
        # only after the request's completion event has been observed
        out = _alloc_out(r, self.dev)
        if res is None:
            tb = self._tree_bytes(r.n)
            ws = torch.empty(tb, dtype=torch.uint8, device=self.dev)
            with torch.cuda.stream(s):
                pts = self.payload(r.set_id, r.n, s)
                tree = Tree(pts, r.periodic_L, self.params, ws, stream=s)
            res = _Resident(r.set_id, tree, tb)
            self.resident[r.set_id] = res  # busy until this request ends
            self.used += tb + r.n * 12
            self.stats["builds"] += 1
            r._pts = pts
        else:
            r.hit = True
            self.resident.move_to_end(r.set_id)
            self.stats["hits"] += 1
        res.busy += 1
        self.used += _out_bytes(r)
        if r.op == "knn":
            res.tree.knn(r.k, out=out, stream=s)
        else:
            res.tree.fof(r.b, out=out, stream=s)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(s)
        r._event = ev
        r._res = res
        r.result = out
        self.lane_busy[lane] = r
        self.peak_used = max(self.peak_used, self.used)
        self.stats["admitted"] += 1

    def _finish(self, r: Request, lane: int):
        res = r._res
        res.busy -= 1
        self.used -= _out_bytes(r)
        if not r.hit:
            self.used -= r.n * 12
            r._pts = None
        if not self.keep_trees and res.busy == 0 and self.resident.get(res.set_id) is res:
            del self.resident[res.set_id]
            self.used -= res.bytes
        if not self.keep_results:
            r.result = None
        r._res = None
        self.lane_busy[lane] = None

    def run(self, requests, realtime: bool = True, poll_sleep: float = 5e-5):
        """Serves ``requests`` (sorted by t_arrival).  realtime=False ignores the
        arrival times (all requests queued at t = 0).  Returns the requests with
        t_done set (seconds since the start of the run)."""
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        _check_requests(reqs)
        torch.cuda.synchronize(self.dev)
        t0_ev = torch.cuda.Event(enable_timing=True)
        t0_ev.record(torch.cuda.current_stream(self.dev))
        t0_ev.synchronize()
        t0 = time.perf_counter()
        pending = collections.deque()
        nxt = 0
        inflight = 0
        done = []
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and (not realtime or reqs[nxt].t_arrival <= now):
                pending.append(reqs[nxt])
                nxt += 1
            progressed = False
            for lane, r in enumerate(self.lane_busy):
                if r is not None and r._event.query():
                    self._finish(r, lane)
                    done.append(r)
                    inflight -= 1
                    progressed = True
            # admit in arrival order while a lane and memory are available
            while pending:
                lane = next((i for i, x in enumerate(self.lane_busy) if x is None), None)
                if lane is None:
                    break
                pick = None
                for i, r in enumerate(pending):
                    res = self.resident.get(r.set_id)
                    if res is not None and res.busy:
                        continue  # its tree is in use by a running request: keep it queued
                    pick = i
                    break
                if pick is None:
                    break
                r = pending[pick]
                need = self._need(r)
                if self.used + need > self.budget and not self._evict_for(need, r.set_id):
                    if inflight == 0:
                        raise RuntimeError(f"request {r.rid} needs {need} bytes, more than the budget allows")
                    break  # wait for memory to be released
                del pending[pick]
                self._start(r, lane)
                inflight += 1
                self.stats["max_inflight"] = max(self.stats["max_inflight"], inflight)
                progressed = True
            if not progressed:
                time.sleep(poll_sleep)
        for r in done:
            r.t_done = t0_ev.elapsed_time(r._event) / 1000.0
            r._event = None
        return reqs

    def clear(self):
        """Drops every resident tree."""
        torch.cuda.synchronize(self.dev)
        for res in self.resident.values():
            self.used -= res.bytes
        self.resident.clear()


class PlainServer:
    """One jzt_knn / jzt_fof call per request, in arrival order on one stream,
    in one workspace sized for the largest request."""

    def __init__(self, payload, max_n: int, device=None, out_budget: float = 150e9, keep_results: bool = False):
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.payload = payload
        self.ws = torch.empty(workspace_bytes(max_n, K_MAX), dtype=torch.uint8, device=self.dev)
        self.stream = torch.cuda.Stream(device=self.dev)
        self.out_budget = out_budget
        self.keep_results = keep_results

    def run(self, requests, realtime: bool = True, poll_sleep: float = 5e-5):
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        _check_requests(reqs)
        s = self.stream
        torch.cuda.synchronize(self.dev)
        t0_ev = torch.cuda.Event(enable_timing=True)
        t0_ev.record(torch.cuda.current_stream(self.dev))
        t0_ev.synchronize()
        t0 = time.perf_counter()
        outstanding = collections.deque()
        held = 0
        for r in reqs:
            if realtime:
                while time.perf_counter() - t0 < r.t_arrival:
                    time.sleep(poll_sleep)
            while outstanding and (held + _out_bytes(r) > self.out_budget or outstanding[0]._event.query()):
                q = outstanding.popleft()
                q._event.synchronize()
                held -= _out_bytes(q)
                if not self.keep_results:
                    q.result = None
            with torch.cuda.stream(s):
                pts = self.payload(r.set_id, r.n, s)
                if r.op == "knn":
                    r.result = _knn_call(pts, r.k, r.periodic_L, workspace=self.ws, stream=s, check=False)
                else:
                    r.result = _fof_call(pts, r.b, r.periodic_L, workspace=self.ws, stream=s, check=False)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(s)
            r._event = ev
            r.lane = 0
            held += _out_bytes(r)
            outstanding.append(r)
        torch.cuda.synchronize(self.dev)
        for r in reqs:
            r.t_done = t0_ev.elapsed_time(r._event) / 1000.0
            r._event = None
            if not self.keep_results:
                r.result = None
        return reqs


def latency_summary(reqs) -> dict:
    """p50 / p99 / mean latency (ms), throughput (requests/s, points/s) of a run."""
    import numpy as np
    lat = np.array([r.t_done - r.t_arrival for r in reqs])
    t_end = max(r.t_done for r in reqs)
    t_beg = min(r.t_arrival for r in reqs)
    span = max(t_end - t_beg, 1e-9)
    pts = sum(r.n for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3),
            "requests_per_s": len(reqs) / span, "particles_per_s": pts / span, "seconds": span}
