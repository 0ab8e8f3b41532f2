"""The N > 1 path of bench.py on CPU: world size 2 over gloo (one process
per rank, rendezvous on 127.0.0.1).  The data path has no collective (the
replicas are independent sequences), so what is exercised is the host
logic: the max-over-ranks timing, the whole-job rate of weakly scaled
replicas, the per-rank workloads, and the reference arm, which only rank 0
runs and prints."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    t = bench.max_over_ranks([3.5, 7.25][rank], dist, device="cpu")
    rate = bench.job_rate(1000, dist.get_world_size(), t)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"t": t, "rate": rate}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_world_size_2(tmp_path):
    port = _free_port()
    torch.multiprocessing.spawn(_rank_main, args=(port, str(tmp_path)), nprocs=2, join=True)
    for r in (0, 1):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got["t"] == 7.25                 # the slowest replica's time
        assert got["rate"] == 2 * 1000 / 7.25   # both ranks' units over that time


def test_no_process_group_means_own_time():
    import bench

    assert bench.max_over_ranks(1.5, None) == 1.5
    assert bench.job_rate(10, 1, 2.0) == 5.0


def test_replicas_get_independent_sequences():
    import bench

    a, b = bench.workload(0), bench.workload(1)
    assert a.luma.shape == b.luma.shape and not np.array_equal(a.luma, b.luma)


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--scale-seqs", "1", "--scale-frames", "4"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
