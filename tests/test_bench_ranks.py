"""The multi-rank (replicas) logic of bench.py on CPU with two gloo ranks:
every rank receives the slowest rank's time, the whole-job value counts the
work of all ranks over that time, and under torchrun only rank 0 of the
reference arm does work and prints."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = [0.75, 1.25][rank]  # per-rank durations (s)
        slowest = bench.max_over_ranks(mine, world)
        value = bench.whole_job_rate(world, 1000, 10, 3, slowest)
        dist.barrier()
        out[rank] = (slowest, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 1.25
    # 2 replicas x 1000 points x 10 steps x 3 runs in 1.25 s
    assert res[0][1] == res[1][1] == pytest.approx(2 * 1000 * 10 * 3 / 1.25 / 1e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.5, 1) == 0.5
    assert bench.whole_job_rate(1, 100, 2, 5, 2.0) == pytest.approx(100 * 2 * 5 / 2.0 / 1e9)


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_runs_on_rank_zero_only(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                        "--config", "star2d1r_f64_512"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stderr
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    if rank:
        assert lines == []
    else:
        rec = json.loads(lines[-1])
        assert rec["impl"] == "reference" and rec["value"] > 0 and rec["cpu_baseline"]["kind"] == "oracle"
