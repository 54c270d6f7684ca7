"""The multi-rank (replicas only) path of bench.py on CPU: two gloo ranks, each with its own
step time; every rank must see the slowest one, and the whole-job throughput must count both
replicas at that time."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = [2.0, 3.5][rank]                                 # rank 1 is the slow one
        slowest = bench.max_over_ranks(ms, torch.device("cpu"))
        units = 1.0e6
        per_replica = units / (slowest * 1e-3) / 1e9              # Gpts/s at the slowest time
        tput = bench.whole_job_value(per_replica, ws, True)
        tmetric = bench.whole_job_value(slowest, ws, False)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
            fh.write(f"{slowest} {tput} {tmetric}\n")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    ws = 2
    mp.spawn(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    vals = [tuple(map(float, (tmp_path / f"rank{r}.txt").read_text().split())) for r in range(ws)]
    for slowest, tput, tmetric in vals:
        assert slowest == 3.5
        assert tput == pytest.approx(2 * 1.0e6 / 3.5e-3 / 1e9)
        assert tmetric == 3.5
