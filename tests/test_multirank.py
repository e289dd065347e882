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


def test_reference_arm_prints_one_contract_line(capsys):
    """Rank 0 times the oracle on a sample of the workload and prints one JSON line with the keys the
    benchmark contract asks of the reference arm."""
    import json
    import bench
    args = argparse.Namespace(workload="8e8o", steps=1, warmup=0, gpus=1)
    bench.run_reference(args, bench.WORKLOADS["8e8o"], 0, 1)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["workload"] == "8e8o"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["e2e"]["d2h_bytes_per_step"] == 0 and d["e2e"]["unit"] == d["unit"]
