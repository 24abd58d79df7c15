"""The multi-rank (N > 1) path of bench.py, on CPU with the gloo backend (no GPU).

- the timing reduction: every rank ends with the slowest rank's time, and the whole-job value
  counts every rank's lattice against that time (weak scaling, replicas with no data-path
  collective);
- the reference arm under torchrun with two ranks: rank 0 alone runs the oracle and prints one
  JSON line; rank 1 exits 0 without work.
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


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    ms = [12.5, 19.75][rank]  # rank 1 is the slow one
    t = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (t, bench.aggregate_mlups(1000, world, 400, t * 1e-3))
    dist.barrier()
    dist.destroy_process_group()


def test_timing_reduction_takes_the_slowest_rank():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 19.75
    # 2 ranks x 1000 nodes x 400 updates in 19.75 ms
    assert res[0][1] == pytest.approx(2 * 1000 * 400 / 19.75e-3 / 1e6)
    assert res[0][1] == res[1][1]


def test_single_process_reduction_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.aggregate_mlups(2048 * 1024, 1, 100, 0.5) == pytest.approx(2048 * 1024 * 100 / 0.5 / 1e6)


@pytest.mark.slow
def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "3", "--warmup", "1", "--nx", "64", "--ny", "32"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1  # rank 0 only
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
