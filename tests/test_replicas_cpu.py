"""Replica runs (one independent march per GPU, no collective on the data path): the
host-side bookkeeping of bench.py across ranks, on CPU with the gloo backend
(world size 2), and the reference arm launched by torchrun with two ranks."""
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


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        sec = bench.max_over_ranks(1.0 + 0.5 * rank, world)     # rank 1 is the slow one
        val = bench.job_throughput(1000, sec, world)
        with open(os.path.join(out_dir, "r%d.json" % rank), "w") as f:
            json.dump({"sec": sec, "value": val}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    got = [json.load(open(tmp_path / ("r%d.json" % r))) for r in range(2)]
    assert all(g["sec"] == 1.5 for g in got)                  # both see the slowest rank
    assert all(g["value"] == 2 * 1000 / 1.5 for g in got)     # units of all ranks / max time


def test_reference_arm_under_torchrun_two_ranks():
    """Rank 0 alone runs the oracle and prints one JSON line; rank 1 exits 0 silently."""
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle"
