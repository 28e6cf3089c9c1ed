"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2), as torchrun launches it.

The evaluation shards by independent problem (every rank runs its own replica; weak scaling), so
the only cross-rank steps are the barrier around the timed region and the max over ranks of the
step time; the reference arm runs on rank 0 alone and the other ranks exit 0 without work.
"""
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


def _rank_main(rank, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=2)
    bench.barrier(dist)
    v = bench.max_over_ranks(dist, 1.0 + 2.0 * rank)
    bench.barrier(dist)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(repr(v))
    dist.destroy_process_group()


def test_barrier_and_max_over_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=2,
                       start_method="spawn", join=True)
    vals = [float(open(tmp_path / f"r{r}.txt").read()) for r in range(2)]
    assert vals == [3.0, 3.0]   # the slower rank's time, on every rank


def test_reference_arm_under_torchrun_two_ranks():
    # what the driver runs for N = 2: rank 0 prints one JSON line, rank 1 exits 0 without work
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--ref-targets", "2", "--alphas", "10"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
