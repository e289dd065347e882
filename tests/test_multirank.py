"""The multi-GPU path of the bench is independent replicas, one per rank (weak scaling): each rank's own
seed, the timed region's length the maximum over ranks, the attempts summed, and the reference arm run by
rank 0 alone. Its host logic is checked here with two gloo ranks on the CPU."""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out) -> None:
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, att = bench.reduce_over_ranks(10.0 + 3.0 * rank, 1000.0 * (rank + 1), world, "cpu")
    out.put((rank, ms, att, bench.replica_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_time_and_attempts():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [13.0, 13.0]  # the slowest rank's time
    assert [r[2] for r in res] == [3000.0, 3000.0]  # all ranks' attempts
    assert res[0][3] != res[1][3]  # independent replicas


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench
    args = argparse.Namespace(workload="8e8o", steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args, bench.WORKLOADS["8e8o"], 1, 2) is None
    assert capsys.readouterr().out == ""
