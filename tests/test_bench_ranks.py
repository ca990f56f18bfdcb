"""The multi-process path of bench.py on CPU: two gloo ranks (world size 2) go through the same
barrier and max-over-ranks helpers the NCCL run uses, the whole-job rate counts every rank's
units over the slowest rank's time, and the reference arm prints from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        # per-rank step times: rank 1 is the slower one
        ms = [40.0, 55.0][rank]
        ms_max = bench.max_over_ranks(world, ms)
        rate = bench.aggregate_rate(1000.0, 4, world, ms_max)
        bench.barrier(world)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"ms_max": ms_max, "rate": rate}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for g in got:
        assert g["ms_max"] == 55.0
        # 1000 units a step on each of 2 ranks, 4 steps, over 55 ms
        assert g["rate"] == pytest.approx(1000.0 * 4 * 2 / 0.055)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    bench.barrier(1)
    assert bench.max_over_ranks(1, 12.5) == 12.5
    assert bench.aggregate_rate(10.0, 3, 1, 2.0) == pytest.approx(10.0 * 3 / 0.002)


def test_reference_arm_prints_from_rank_zero_only():
    # a non-zero rank returns before it would run the oracle, printing nothing
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120,
                       cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
