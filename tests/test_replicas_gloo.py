"""The multi-process path of bench.py on CPU (gloo, world size 2): the
contraction needs no exchange between GPUs, so N > 1 runs independent
replicas; what the ranks share is the barrier around the timed region and the
max over ranks of the measured time, and only rank 0 prints."""
import json
import os
import socket
import subprocess
import sys

import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2", LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    ws, r, local = bench.dist_setup(None)
    assert (ws, r, local) == (2, rank, rank)
    bench.barrier(ws)
    # the slowest rank's time is the job's time
    out[rank] = bench.max_over_ranks(1.5 + rank, ws)
    bench.barrier(ws)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_max_over_ranks_and_barrier():
    port = free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(port, out), nprocs=2, join=True)
    assert dict(out) == {0: 2.5, 1: 2.5}


def test_reference_arm_under_torchrun_prints_once():
    # the launch the driver uses for N > 1, on CPU: rank 0 runs the oracle
    # arm and prints one line, rank 1 exits 0 without work
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--workload", "small_f64"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0
