"""The N > 1 benchmark path on CPU: two gloo ranks aggregate whole-job figures.

Each rank fits its own frame (weak scaling, no collective on the data path);
the only collective is the all-gather of (units, seconds) after the timed
region: units add, time is the slowest rank's.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [1000.0 * (rank + 1), 2.0 + rank, 10.0 * (rank + 1), 0.5 + rank]
    out[rank] = bench.aggregate(local, world)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        units, tmax, e2e_units, e2e_tmax = out[r]
        assert units == 3000.0 and tmax == 3.0 and e2e_units == 30.0 and e2e_tmax == 1.5


def test_single_rank_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate([5.0, 2.0, 3.0, 1.0], 1) == (5.0, 2.0, 3.0, 1.0)


def test_reference_arm_prints_one_json_line():
    """bench.py --impl reference: the FP64 oracle on the host, rank 0 only."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "point-component-iters/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], capture_output=True,
                       text=True, timeout=120, cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""
