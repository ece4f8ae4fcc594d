"""Multi-process paths of bench.py on CPU (gloo, world size 2): the replicas'
max-over-ranks timing and whole-job rate, and the reference arm under torchrun
(rank 0 alone runs the oracle and prints one line; the other rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w, local, pg = bench.dist_setup("gloo")
    assert (r, w, local) == (rank, world, rank)
    ms = [10.0 + 5.0 * rank, 3.0 - rank]
    got = bench.max_over_ranks(ms, pg)
    rate = bench.whole_job_rate(1000, w, got[0])
    pg.barrier()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"max": got, "rate": rate}, fh)
    pg.destroy_process_group()


def test_max_over_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r in res:
        assert r["max"] == [15.0, 3.0]
        assert r["rate"] == pytest.approx(2 * 1000 / 0.015)


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.0], None) == [1.5, 2.0]
    assert bench.whole_job_rate(10, 1, 1000.0) == pytest.approx(10.0)


def test_reference_arm_under_torchrun(tmp_path):
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--n-side", "32", "--steps", "1", "--warmup", "0",
           "--ref-side", "0.5", "--cache", str(tmp_path)]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
