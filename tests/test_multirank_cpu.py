"""The N > 1 bench path on the CPU: two `gloo` ranks run the host logic that
`bench.py --gpus N` runs under torchrun (replicas only: every rank steps its own
copy of the workload, and no collective touches the data path). Checked here:
the max-over-ranks timing every rank agrees on, the whole-job rate (units of
all ranks over the slowest rank's time), and that only rank 0 runs the oracle
arm while the others return without work."""
from __future__ import annotations

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import json

    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (10 + r) ms for the whole run and (3 + 2 r) ms for the forward
        total, fwd = bench.max_over_ranks([10.0 + rank, 3.0 + 2.0 * rank], world, torch.device("cpu"))
        rate = bench.whole_job_rate(1000.0, world, total / 1e3)
        dist.barrier()

        class Args:
            steps, warmup, scale = 1, 0, 0.001

        ref = bench.run_reference(Args, rank) if rank != 0 else "skipped"
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"total": total, "fwd": fwd, "rate": rate, "ref_is_none": ref is None}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_whole_job_rate(tmp_path):
    import json

    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["total"] == 11.0 and r["fwd"] == 5.0
        # 1000 units per rank, 2 ranks, 11 ms per step
        assert r["rate"] == pytest.approx(2000.0 / 0.011)
    # non-zero ranks return from the oracle arm without running it
    assert res[1]["ref_is_none"]


def test_single_rank_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([4.0, 2.5], 1) == [4.0, 2.5]
    assert bench.whole_job_rate(500, 1, 0.5) == 1000.0
