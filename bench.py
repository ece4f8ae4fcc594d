#!/usr/bin/env python
"""Throughput benchmark: exact kNN (k = 16) and FoF (b = 0.2 mean spacing) on
2^27 = 512^3 points (Zel'dovich-displaced lattice in a periodic unit box).

One step = build the tree (keys, radix sort, planes, nodes) + kNN walk + FoF
walk on device-resident points; value = particles per second for the whole job
(all ranks).  Multi-GPU runs are independent replicas (the workload does not
shard), so scaling is weak.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the only other implementation of this
path here) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "kNN(k=16) & FoF(b=0.2) particles/s at N=2^27 on 1 GB300; p50/p99 served latency"
UNIT = "particles/s"
FLOPS_PER_PAIR = 8        # dx, dy, dz, dx*dx, 2 fma (fma = 2 flops)
FP32_LANES_PER_SM = 128
SMS = 152
SORT_BYTES_PER_PT = 24    # one LSD pass: read key+value, write key+value (8+4 each way)
# bucket sort: scatter reads the key (8) and writes key+index (12); the bin sort reads
# key+index (12) and the point (12) and writes the key (8) and the float4 point (16)
BUCKET_SORT_BYTES_PER_PT = 68
BUILD_FLOOR_BYTES = 42    # read xyz 12 + sorted float4 16 + keys/perm 12 + tree ~2
# DRAM bytes per point of one k_l2l_knn launch (k = 16): 694 MB read + 2097 MB written
# on 2^24 points, from the ncu capture of this kernel version
L2L_TRAFFIC_BYTES_PER_PT = (693.5e6 + 2097.4e6) / (1 << 24)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-side", type=int, default=512)
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--b-frac", type=float, default=0.2)
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--ref-queries", type=int, default=1 << 18,
                    help="kNN rows per step of --impl reference (random points of the full set)")
    ap.add_argument("--ref-side", type=float, default=0.25,
                    help="side of the sub-cube whose FoF is timed per step by --impl reference")
    ap.add_argument("--cpu-queries", type=int, default=1 << 20,
                    help="kNN rows timed on the CPU for cpu_baseline")
    ap.add_argument("--cpu-side", type=float, default=0.5,
                    help="side of the sub-cube whose FoF is timed on the CPU for cpu_baseline")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--kdtree-side", type=float, default=0.5,
                    help="side of the sub-cube timed with scipy's k-d tree (context)")
    ap.add_argument("--nmax0", type=int, default=0, help="leaf capacity (0 = library default)")
    ap.add_argument("--cache", default=os.path.join(tempfile.gettempdir(), "jzt_bench_cache"))
    ap.add_argument("--batch-sets", type=int, default=512, help="batched sets (0 = skip the batched run)")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=20000, help="served requests (0 = skip serving)")
    ap.add_argument("--serve-sample", type=int, default=2000,
                    help="requests (the first ones of the stream) used to measure capacity and for the load sweep")
    ap.add_argument("--serve-lanes", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-load", type=float, default=0.8,
                    help="arrival rate as a fraction of the one-call server's measured capacity")
    ap.add_argument("--serve-sweep", default="0.5,1.0,1.5",
                    help="comma-separated extra loads to run both servers at (on the first --serve-sample requests)")
    return ap.parse_args()


def workload(n_side, cache):
    import numpy as np
    import workloads
    os.makedirs(cache, exist_ok=True)
    path = os.path.join(cache, f"zeldovich_{n_side}_seed3.npy")
    if os.path.exists(path):
        return np.load(path)
    x = workloads.zeldovich(n_side, 3)
    np.save(path + ".tmp.npy", x)
    os.replace(path + ".tmp.npy", path)
    return x


class Clocks:
    """nvidia-smi sampler over the timed region (SM clocks and throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [v.strip() for v in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None

        def num(v):
            try:
                return float(v)
            except ValueError:
                return float("nan")
        sm = sorted(num(r[1]) for r in rows)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(num(r[2]) for r in rows),
                "power_w_max": max(num(r[3]) for r in rows), "samples": len(rows),
                "reasons": sorted(reasons)}


def cpu_baseline(x, n_side, k, b, q_sample, fof_side, threads=0, seed=0):
    """The oracle (float64 cell lists, all host cores) on a bounded sample of the
    workload, scaled to a rate for the whole of it:

    * kNN: the rows of ``q_sample`` points drawn at random from the full periodic
      set (the same problem; every row costs about the same), time x N / q_sample;
    * FoF: the points of the sub-cube [0, fof_side)^3 as an open box (FoF needs
      the whole connected set, so a sub-volume stands in), time x N / its points.
    """
    import numpy as np
    import oracle
    n = x.shape[0]
    q = np.sort(np.random.default_rng(seed).choice(n, min(int(q_sample), n), replace=False))
    sel = np.all(x < np.float32(fof_side), axis=1)
    xs = np.ascontiguousarray(x[sel])
    cores = oracle.num_threads(threads)
    t0 = time.perf_counter()
    oracle.knn_cells(x, k, 1.0, queries=q, threads=threads)
    t1 = time.perf_counter()
    oracle.fof_cells(xs, b, 0.0, threads=threads)
    t2 = time.perf_counter()
    est = (t1 - t0) * n / len(q) + (t2 - t1) * n / xs.shape[0]
    return {"value": n / est, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"kNN k={k}: rows of {len(q)} random points of the full periodic {n_side}^3 Zel'dovich "
                      f"set ({t1 - t0:.1f} s); FoF b={b:.3g}: the {xs.shape[0]} points of the sub-cube "
                      f"[0,{fof_side})^3 as an open box ({t2 - t1:.1f} s); each part scaled to all {n} points",
            "seconds": t2 - t0, "seconds_full_estimate": est}


def batched_run(a, dev, log):
    """512 independent clustered sets (sizes log-uniform 1e3..2e6, per-set kNN k
    in {8,16,32} or FoF b in {0.15,0.2,0.25} x spacing), run as one Batch replayed
    from a CUDA graph with autotuned lanes and tree parameters, against one
    jzt_knn / jzt_fof call per set on one stream; outputs compared bitwise."""
    import torch

    import paper_2604_05885_gb300 as jzt
    import workloads
    from paper_2604_05885_gb300 import autotune

    t = time.perf_counter()
    host = workloads.batched_sets(a.batch_sets, 4, workers=min(16, os.cpu_count() or 1))
    gen_s = time.perf_counter() - t
    sets = [dict(points=torch.from_numpy(h["points"]).to(dev), op=h["op"], k=h["k"], b=h["b"],
                 periodic_L=h["periodic_L"]) for h in host]
    del host
    total = sum(int(st["points"].shape[0]) for st in sets)
    t = time.perf_counter()
    if a.no_autotune:
        n_lanes, params, caps = 8, {}, [0, 0, 0]
    else:
        n_lanes, params, caps = autotune.tune(sets, cache=os.path.join(a.cache, "autotune.json"), log=log)
    cap_fn = autotune.leaf_cap_fn(caps)
    tune_s = time.perf_counter() - t
    batch = jzt.Batch(sets, n_lanes=n_lanes, params=params or None, graph=True, nmax0_of=cap_fn)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        for _ in range(max(3, a.warmup)):
            fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    ms_batch = timed(batch.run, a.batch_steps)
    bad = [j for j, c in enumerate(batch.statuses()) if c != 0]
    # the same batch with the kNN LeafToLeaf of all jobs in persistent launches over a
    # device work queue (one workspace per job), also replayed from a CUDA graph
    qbatch = jzt.Batch(sets, n_lanes=n_lanes, params=params or None, graph=True, queue=True, nmax0_of=cap_fn)
    ms_queue = timed(qbatch.run, a.batch_steps)
    bad += [j for j, c in enumerate(qbatch.statuses()) if c != 0]
    # one call per set on one stream, one workspace sized for the largest set
    ws = jzt.alloc_workspace(max(int(st["points"].shape[0]) for st in sets), 32, None, dev)
    outs = []
    for st in sets:
        n = int(st["points"].shape[0])
        if st["op"] == "knn":
            outs.append((torch.empty((n, st["k"]), dtype=torch.int32, device=dev),
                         torch.empty((n, st["k"]), dtype=torch.float32, device=dev)))
        else:
            outs.append(torch.empty(n, dtype=torch.int32, device=dev))

    def one_call_per_set():
        for st, out in zip(sets, outs):
            if st["op"] == "knn":
                jzt.knn(st["points"], st["k"], st["periodic_L"], workspace=ws, check=False, out=out)
            else:
                jzt.fof(st["points"], st["b"], st["periodic_L"], workspace=ws, check=False, out=out)

    ms_plain = timed(one_call_per_set, a.batch_steps)
    jzt.status(ws, raise_on_error=True)
    same = True
    for st, ob, oq, op in zip(sets, batch.outputs, qbatch.outputs, outs):
        if st["op"] == "knn":
            same &= bool(torch.equal(ob[0], op[0]) and torch.equal(ob[1], op[1]))
            same &= bool(torch.equal(oq[0], op[0]) and torch.equal(oq[1], op[1]))
        else:
            same &= bool(torch.equal(ob, op)) and bool(torch.equal(oq, op))
    n_knn = sum(1 for st in sets if st["op"] == "knn")
    res = {"workload": f"{len(sets)} clustered sets, sizes log-uniform 1e3..2e6, seed 4",
           "points": total, "knn_sets": n_knn, "fof_sets": len(sets) - n_knn,
           "lanes": batch.n_lanes, "params": params or {}, "graph": True,
           "leaf_capacity_per_size_class": {"N < 2^14": caps[0] or "params", "2^14 <= N < 2^18": caps[1] or "params",
                                            "N >= 2^18": caps[2] or "params"},
           "value": total / (ms_batch / 1000.0), "unit": "particles/s", "ms_per_batch": ms_batch,
           "one_call_per_set": {"value": total / (ms_plain / 1000.0), "ms_per_batch": ms_plain},
           "persistent_queue": {"value": total / (ms_queue / 1000.0), "ms_per_batch": ms_queue,
                                "form": "per-job workspaces; kNN LeafToLeaf of all jobs in one persistent launch "
                                        "per (k class, boundary) over a device work queue; graph replay"},
           "speedup": ms_plain / ms_batch, "identical_results": same, "failed_jobs": bad,
           "steps": a.batch_steps, "autotune_s": tune_s, "generate_s": gen_s}
    del batch, qbatch, outs, ws, sets
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()
    return res


def serving_run(a, dev, log):
    """Poisson stream of kNN/FoF requests (sizes log-uniform 1e4..2^24, 30 % on an
    earlier set), served by the continuous-batching Server (lanes, HBM budget,
    resident trees) and by the one-call-per-request PlainServer, both at the same
    arrival rate: serve_load x the one-call server's measured capacity."""
    import torch

    import workloads
    from paper_2604_05885_gb300.serve import PlainServer, Request, Server, latency_summary

    spec = workloads.serving_stream(a.serve_requests, 5, rate_hz=1.0)
    seeds = {r["set_id"]: r["seed"] for r in spec}

    def payload(sid, n, stream):
        return workloads.clustered_device(n, seeds[sid], dev)

    def requests(rate, count=None):
        """The stream at ``rate`` requests/s (rate None: every request at t = 0);
        ``count``: only the first requests of the stream."""
        return [Request(i, r["set_id"], r["n"], r["op"], r["k"], r["b"], 1.0,
                        0.0 if rate is None else r["t_arrival"] / rate)
                for i, r in enumerate(spec[:count])]

    sample = min(a.serve_sample, len(spec)) if a.serve_sample > 0 else len(spec)

    max_n = max(r["n"] for r in spec)
    plain = PlainServer(payload, max_n, device=dev)
    warm = [Request(i, -1 - i, n, op, k, b, 1.0, 0.0)
            for i, (n, op, k, b) in enumerate([(20000, "knn", 16, 0.0), (300000, "fof", 0, 0.001),
                                               (20000, "fof", 0, 0.01), (300000, "knn", 32, 0.0)])]
    for sd in range(4):
        seeds[-1 - sd] = 99 + sd
    plain.run(warm, realtime=False)
    cap_plain = latency_summary(plain.run(requests(None, sample), realtime=False))
    rate = a.serve_load * cap_plain["requests_per_s"]
    log(f"one-call capacity {cap_plain['requests_per_s']:.1f} req/s; arrival rate {rate:.1f} req/s")
    plain_rt = latency_summary(plain.run(requests(rate), realtime=True))
    sweep = {}
    loads = [float(v) for v in a.serve_sweep.split(",") if v.strip()]
    for ld in loads:
        sweep[str(ld)] = {"one_call_per_request": latency_summary(
            plain.run(requests(ld * cap_plain["requests_per_s"], sample), realtime=True))}
    del plain
    torch.cuda.empty_cache()
    srv = Server(payload, n_lanes=a.serve_lanes, hbm_budget=a.serve_budget_gb * 1e9, device=dev)
    srv.run(warm, realtime=False)
    srv.clear()
    served_rt = latency_summary(srv.run(requests(rate), realtime=True))
    st_rt = dict(srv.stats)
    peak_rt = srv.peak_used
    srv.clear()
    for ld in loads:
        sweep[str(ld)]["served"] = latency_summary(srv.run(requests(ld * cap_plain["requests_per_s"], sample),
                                                           realtime=True))
        srv.clear()
    srv.stats = dict.fromkeys(srv.stats, 0)
    cap_served = latency_summary(srv.run(requests(None, sample), realtime=False))
    srv.clear()
    del srv
    torch.cuda.empty_cache()
    ns = sorted(r["n"] for r in spec)
    return {"workload": f"{len(spec)} requests, Poisson arrivals, sizes log-uniform 1e4..2^24, "
                        f"30% repeat an earlier set, seed 5",
            "points": sum(ns), "median_n": ns[len(ns) // 2], "arrival_rate_per_s": rate,
            "load_vs_one_call_capacity": a.serve_load, "lanes": a.serve_lanes,
            "hbm_budget_gb": a.serve_budget_gb, "served": served_rt, "served_stats": st_rt,
            "served_peak_bytes": peak_rt, "one_call_per_request": plain_rt,
            "capacity": {"served": cap_served, "one_call_per_request": cap_plain,
                         "requests": sample, "note": "every request of the first `requests` queued at t = 0"},
            "load_sweep": ({"requests": sample, "loads_vs_one_call_capacity": sweep} if sweep else None)}


def cpu_kdtree(x, n_side, k, side):
    """Context only: scipy's multithreaded k-d tree (build + kNN query, all host
    cores) on the points of the sub-cube [0, side)^3, treated as an open box."""
    import numpy as np
    try:
        from scipy.spatial import cKDTree
    except ImportError as exc:  # pragma: no cover
        return {"unavailable": str(exc)}
    sel = np.all(x < np.float32(side), axis=1)
    xs = np.ascontiguousarray(x[sel], dtype=np.float64)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    tr = cKDTree(xs)
    tr.query(xs, k, workers=-1)
    dt = time.perf_counter() - t0
    return {"value": xs.shape[0] / dt, "unit": UNIT, "cores": cores, "kind": "scipy cKDTree (kNN only)",
            "sample": f"{xs.shape[0]} points of the sub-cube [0,{side})^3 of the {n_side}^3 Zel'dovich set, "
                      f"open box; build + query k={k}", "seconds": dt}


def dist_env():
    """(rank, world size, local rank) from the torchrun environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def dist_setup(backend="nccl"):
    """One process per GPU: a process group when there is more than one rank.
    The ranks are independent replicas; the group only carries the barriers
    and the max-over-ranks timing."""
    rank, world, local = dist_env()
    pg = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
        pg = dist
    return rank, world, local, pg


def max_over_ranks(values, dist, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (identity for one rank)."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_rate(units_per_rank, world, ms_max):
    """Replicas: every rank processes units_per_rank; the job's rate uses the slowest rank."""
    return world * units_per_rank / (ms_max / 1000.0)


def catalogue_timing(x_dev, L, b, params, ws, lab, stream, dev, reps=3):
    """Build + FoF + catalogue (groups of at least 20 members) through
    jzt_tree_fof_catalogue, timed with CUDA events over ``reps`` calls."""
    import torch

    import paper_2604_05885_gb300 as jzt
    n = int(x_dev.shape[0])
    try:
        cap = n // 20 + 1
        order_c = torch.empty(n, dtype=torch.int32, device=dev)
        gbuf = torch.empty(cap * jzt.GROUP_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        ng = torch.zeros(1, dtype=torch.int64, device=dev)

        def cat_step():
            t2 = jzt.build(x_dev, periodic_L=L, workspace=ws, params=params)
            rc = jzt.lib.jzt_tree_fof_catalogue(t2._h, float(b), None, 20, 1.0, ctypes.c_void_p(lab.data_ptr()),
                                                ctypes.c_void_p(order_c.data_ptr()), ctypes.c_void_p(gbuf.data_ptr()),
                                                cap, ctypes.c_void_p(ng.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
            if rc != 0:
                raise RuntimeError(f"jzt_tree_fof_catalogue: {rc} {jzt.lib.jzt_last_error().decode()}")
            return t2
        t2 = cat_step()
        t2.status(raise_on_error=True)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(reps):
            t2 = cat_step()
        c1.record(stream)
        torch.cuda.synchronize(dev)
        t2.status(raise_on_error=True)
        ms_cat = c0.elapsed_time(c1) / reps
        out = {"ms_per_step": ms_cat, "value": n / (ms_cat / 1000.0), "unit": UNIT, "n": n, "min_count": 20,
               "groups": int(ng.item()), "step": "build + FoF + group order + catalogue reduction"}
        del order_c, gbuf, ng, t2
    except Exception as exc:  # noqa: BLE001  (reported, not fatal for the main line)
        out = {"error": str(exc)[:200]}
    jzt.profile_read()
    return out


def main():
    a = parse()
    if a.impl == "reference":
        rank, world, local = dist_env()
        dist = None  # rank 0 alone times the oracle; the other ranks exit without work
    else:
        rank, world, local, dist = dist_setup("nccl")
    n_side = a.n_side
    n = n_side ** 3
    k = a.k
    b = a.b_frac / n_side
    L = 1.0
    cfg = {"workload": f"zeldovich-{n_side}^3-periodic", "n": n, "k": k, "b": b, "periodic_L": L,
           "step": "build + kNN(k) + FoF(b) on device-resident points",
           "parallelism": f"replicas x{world}", "l2": "inputs (12 B/pt) larger than L2 (129 MB)"}

    if a.impl == "reference":
        if rank != 0:
            return
        x = workload(n_side, a.cache)
        import numpy as np  # noqa: F401
        vals = []
        for s in range(a.warmup + a.steps):
            cb = cpu_baseline(x, n_side, k, b, a.ref_queries, a.ref_side, seed=s)
            if s >= a.warmup:
                vals.append(cb)
        v = sorted(c["value"] for c in vals)[len(vals) // 2]
        cb = dict(vals[-1])
        cb["value"] = v
        cfg_ref = dict(cfg, step="oracle on a bounded sample per step, scaled to the whole workload",
                       sample=cb["sample"], parallelism=f"host cores x{cb['cores']}")
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": 1000.0 * sum(c["seconds"] for c in vals) / len(vals),
                "ms_per_step_full_workload_estimate": 1000.0 * sum(c["seconds_full_estimate"] for c in vals) / len(vals),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": cfg_ref, "cpu_baseline": cb,
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import numpy as np
    import torch

    import paper_2604_05885_gb300 as jzt
    import workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    x = workload(n_side, a.cache)
    x_dev = torch.from_numpy(x).to(dev)
    params = {"nmax0": a.nmax0} if a.nmax0 else None
    ws = jzt.alloc_workspace(n, k, params, dev)
    idx = torch.empty((n, k), dtype=torch.int32, device=dev)
    d2 = torch.empty((n, k), dtype=torch.float32, device=dev)
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(xd):
        tree = jzt.build(xd, periodic_L=L, workspace=ws, params=params)
        tree.knn(k, out=(idx, d2))
        tree.fof(b, out=lab)
        return tree

    tree = None
    for _ in range(a.warmup):
        tree = step(x_dev)
    if tree is not None:
        tree.status(raise_on_error=True)
    jzt.profile_read()  # discard warm-up records

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    clocks = Clocks(local)
    barrier()
    jzt.profile_enable(True)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        tree = step(x_dev)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    jzt.profile_enable(False)
    ms_total = e0.elapsed_time(e1)
    phase_ms, phase_cnt, launches = jzt.profile_read()
    st = tree.status(raise_on_error=True)
    ms_step = max_over_ranks([ms_total / a.steps], dist, dev)[0]
    value = whole_job_rate(n, world, ms_step)

    # kNN with rows in z order (Sec. III-G's benchmark output, no final reordering):
    # build + kNN, compared with the same in input order
    zo = {}
    for order in (1, 0):
        def knn_step():
            t3 = jzt.build(x_dev, periodic_L=L, workspace=ws, params=params)
            t3.knn(k, order=order, out=(idx, d2))
            return t3
        t3 = knn_step()
        z0 = torch.cuda.Event(enable_timing=True)
        z1 = torch.cuda.Event(enable_timing=True)
        z0.record(stream)
        for _ in range(3):
            t3 = knn_step()
        z1.record(stream)
        torch.cuda.synchronize(dev)
        t3.status(raise_on_error=True)
        zms = z0.elapsed_time(z1) / 3
        zo["z_order" if order else "input_order"] = {"ms_per_step": zms, "value": n / (zms / 1000.0), "unit": UNIT}
    del t3
    jzt.profile_read()

    # FoF catalogue (Sec. IV-B): build + FoF + group order + reductions, groups >= 20; on the
    # benchmark set (all singletons at b = 0.2 spacings) and on the 2^24 clustered periodic set.
    # The clustered set (4096 blobs, 7 M groups) also gets the plain rates: build + FoF and
    # build + kNN (k = 32), since FoF on the benchmark set links nothing.
    cat = catalogue_timing(x_dev, L, b, params, ws, lab, stream, dev)
    clu = {}
    try:
        wc, xc_h = workloads.config_clustered_16m()
        xc = torch.from_numpy(xc_h).to(dev)
        nc = xc.shape[0]
        wsc = jzt.alloc_workspace(nc, wc.k, params, dev)
        labc = torch.empty(nc, dtype=torch.int32, device=dev)
        cat_c = catalogue_timing(xc, wc.periodic_L, wc.b, params, wsc, labc, stream, dev)
        cat_c["workload"] = f"{wc.name}, seed 2, b = 0.2/256"
        ic = torch.empty((nc, wc.k), dtype=torch.int32, device=dev)
        dc = torch.empty((nc, wc.k), dtype=torch.float32, device=dev)
        for name, op in (("fof", lambda t: t.fof(wc.b, out=labc)), ("knn", lambda t: t.knn(wc.k, out=(ic, dc)))):
            def one():
                t = jzt.build(xc, periodic_L=wc.periodic_L, workspace=wsc, params=params)
                op(t)
                return t
            tc = one()
            tc.status(raise_on_error=True)
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            for _ in range(3):
                tc = one()
            c1.record(stream)
            torch.cuda.synchronize(dev)
            tc.status(raise_on_error=True)
            ms_c = c0.elapsed_time(c1) / 3
            clu[name] = {"workload": wc.name, "n": nc, "periodic_L": wc.periodic_L,
                         "k" if name == "knn" else "b": wc.k if name == "knn" else wc.b,
                         "step": f"build + {'kNN' if name == 'knn' else 'FoF'}", "ms_per_step": ms_c,
                         "value": nc / (ms_c / 1000.0), "unit": UNIT}
            if name == "fof":
                clu[name]["groups"] = int(torch.unique(labc).numel())
            del tc
        del xc, wsc, labc, ic, dc
    except Exception as exc:  # noqa: BLE001  (reported, not fatal for the main line)
        cat_c = cat_c if "cat_c" in locals() else {"error": str(exc)[:200]}
        clu["error"] = str(exc)[:200]
    jzt.profile_read()

    del ws, idx, d2, lab, tree
    torch.cuda.empty_cache()

    # end to end from pinned host buffers: every step uploads its points and reads
    # back kNN rows and FoF labels.  HostPipeline overlaps the transfers of one
    # step with the compute of its neighbours (double-buffered device buffers);
    # e2e_serial runs the same steps strictly one after another on one stream.
    e2e, e2e_serial = None, None
    if a.e2e_steps > 0:
        from paper_2604_05885_gb300.pipeline import HostPipeline
        try:
            x_host = torch.from_numpy(x).pin_memory()
            idx_h = torch.empty((n, k), dtype=torch.int32).pin_memory()
            d2_h = torch.empty((n, k), dtype=torch.float32).pin_memory()
            lab_h = torch.empty(n, dtype=torch.int32).pin_memory()
        except RuntimeError as exc:  # pinned allocation refused
            x_host = None
            e2e = {"value": None, "unit": UNIT, "error": str(exc)[:200]}
        if x_host is not None:
            h2d = x_host.numel() * 4
            d2h = idx_h.numel() * 4 + d2_h.numel() * 4 + lab_h.numel() * 4
            pipe = HostPipeline(n, k, b, L, params, dev)
            for _ in range(2):
                pipe.submit(x_host, idx_h, d2_h, lab_h)
            pipe.synchronize()
            barrier()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(pipe.s_up)
            for _ in range(a.e2e_steps):
                pipe.submit(x_host, idx_h, d2_h, lab_h)
            f1.record(pipe.s_down)
            pipe.synchronize()
            barrier()
            ms_e2e = f0.elapsed_time(f1) / a.e2e_steps
            pipe.status(raise_on_error=True)
            del pipe
            torch.cuda.empty_cache()
            # serial: one stream, upload -> compute -> download per step
            ws1 = jzt.alloc_workspace(n, k, params, dev)
            x_in = torch.empty((n, 3), dtype=torch.float32, device=dev)
            i1 = torch.empty((n, k), dtype=torch.int32, device=dev)
            d1 = torch.empty((n, k), dtype=torch.float32, device=dev)
            l1 = torch.empty(n, dtype=torch.int32, device=dev)
            barrier()
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            for _ in range(max(1, a.e2e_steps // 2)):
                x_in.copy_(x_host, non_blocking=True)
                t1 = jzt.build(x_in, periodic_L=L, workspace=ws1, params=params)
                t1.knn(k, out=(i1, d1))
                t1.fof(b, out=l1)
                idx_h.copy_(i1, non_blocking=True)
                d2_h.copy_(d1, non_blocking=True)
                lab_h.copy_(l1, non_blocking=True)
            g1.record(stream)
            barrier()
            ms_ser = g0.elapsed_time(g1) / max(1, a.e2e_steps // 2)
            t1.status(raise_on_error=True)
            del ws1, x_in, i1, d1, l1, t1
            torch.cuda.empty_cache()
            ms_e2e, ms_ser = max_over_ranks([ms_e2e, ms_ser], dist, dev)
            e2e = {"value": whole_job_rate(n, world, ms_e2e), "unit": UNIT, "ms_per_step": ms_e2e,
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "mode": "HostPipeline: transfers of neighbouring steps overlap the compute"}
            e2e_serial = {"value": whole_job_rate(n, world, ms_ser), "unit": UNIT, "ms_per_step": ms_ser,
                          "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        jzt.profile_read()

    # rooflines ----------------------------------------------------------------
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as fh:
            peaks = json.load(fh)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    alu_peak_tflops = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    steps = a.steps
    per = {ph: (phase_ms[ph] / phase_cnt[ph] if phase_cnt[ph] else 0.0) for ph in phase_ms}
    l2l_ms = per.get("knn_l2l", 0.0)
    pairs_per_launch = st["knn_pairs"]
    achieved = pairs_per_launch * FLOPS_PER_PAIR / (l2l_ms / 1000.0) / 1e12 if l2l_ms else 0.0
    roofline = {"kernel": "k_l2l_knn", "bound": "alu", "achieved": achieved, "peak": alu_peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / alu_peak_tflops if alu_peak_tflops else None,
                "traffic": L2L_TRAFFIC_BYTES_PER_PT * n if (n_side == 512 and k == 16) else None,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_l2l_knn on the 256^3 "
                                  "set (profiles/k_l2l_knn_zeldovich256.md), scaled by N", "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (median SM clock sampled)",
                "work": f"{pairs_per_launch} point pairs x {FLOPS_PER_PAIR} flops per launch",
                "ms_per_launch": l2l_ms}
    sort_ms = phase_ms.get("sort", 0.0) / max(1, phase_cnt.get("sort", 0))
    bucket = st.get("sort_path", 0) == 1
    sort_launch_ms = sort_ms if bucket else sort_ms / 8.0
    sort_bytes = BUCKET_SORT_BYTES_PER_PT if bucket else SORT_BYTES_PER_PT
    sort_gbs = sort_bytes * n / (sort_launch_ms / 1000.0) / 1e9 if sort_ms else 0.0
    build_ms = sum(per.get(ph, 0.0) for ph in ("box", "keys", "sort", "gather", "splits", "nodes"))
    build_floor_gbs = BUILD_FLOOR_BYTES * n / (build_ms / 1000.0) / 1e9 if build_ms else 0.0
    roof_sort = {"kernel": "k_bucket_scatter + k_bin_sort" if bucket else "k_onesweep", "bound": "hbm",
                 "achieved": sort_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": sort_gbs / hbm_peak,
                 "traffic": None, "peak_source": hbm_src,
                 "work": (f"{BUCKET_SORT_BYTES_PER_PT} B/pt x {n} (scatter into fine bins + per-bin sort)" if bucket
                          else f"{SORT_BYTES_PER_PT} B/pt x {n} per pass"),
                 "ms_per_launch": sort_launch_ms}
    roof_build = {"stage": "build (box, keys, sort, gather, splits, nodes)", "bound": "hbm",
                  "achieved": build_floor_gbs, "peak": hbm_peak, "unit": "GB/s",
                  "frac": build_floor_gbs / hbm_peak, "work": f"{BUILD_FLOOR_BYTES} B/pt algorithmic floor",
                  "ms": build_ms}
    knn_ms = sum(per.get(ph, 0.0) * phase_cnt.get(ph, 0) / steps for ph in ("knn_top", "knn_n2n", "knn_sort", "knn_l2l"))
    fof_ms = sum(per.get(ph, 0.0) * phase_cnt.get(ph, 0) / steps for ph in ("fof_top", "fof_n2n", "fof_l2l", "fof_labels"))

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "clocks": clk, "e2e": e2e, "e2e_serial": e2e_serial, "gpu_launches": launches,
            "fof_catalogue": cat, "fof_catalogue_clustered": cat_c, "fof_clustered": clu.get("fof"),
            "knn_clustered": clu.get("knn"), "knn_build_plus_walk": zo, "roofline": roofline,
            "roofline_sort": roof_sort, "roofline_build": roof_build,
            "phases_ms_per_step": {ph: phase_ms[ph] / steps for ph in phase_ms},
            "knn_particles_per_s": n / ((build_ms + knn_ms) / 1000.0) if knn_ms else None,
            "fof_particles_per_s": n / ((build_ms + fof_ms) / 1000.0) if fof_ms else None,
            "knn_pairs_per_point": st["knn_pairs"] / n, "fof_pairs_per_point": st["fof_pairs"] / n,
            "ilist_entries": st["ilist_entries"], "n_nodes": [v for v in st["n_nodes"] if v],
            "knn_plane_entries": [v for v in st["knn_plane_entries"] if v],
            "knn_l2l_entries_examined": st["knn_stats"][0], "knn_l2l_leaves_scanned": st["knn_stats"][1],
            "knn_l2l_candidates_queued": st["knn_stats"][2],
            "p50_p99_latency": None}
    del x_dev
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()

    def log(msg):
        print(f"[bench] {msg}", file=sys.stderr, flush=True)

    # the batched and serving runs describe one GPU; replicas (N > 1) skip them
    if a.batch_sets > 0 and world == 1:
        line["batched"] = batched_run(a, dev, log)
    if a.serve_requests > 0 and world == 1:
        sv = serving_run(a, dev, log)
        line["serving"] = sv
        line["p50_p99_latency"] = {"p50_ms": sv["served"]["p50_ms"], "p99_ms": sv["served"]["p99_ms"],
                                   "one_call_p50_ms": sv["one_call_per_request"]["p50_ms"],
                                   "one_call_p99_ms": sv["one_call_per_request"]["p99_ms"],
                                   "arrival_rate_per_s": sv["arrival_rate_per_s"]}
    if rank == 0 and not a.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(x, n_side, k, b, a.cpu_queries, a.cpu_side)
        line["cpu_kdtree"] = cpu_kdtree(x, n_side, k, a.kdtree_side)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
