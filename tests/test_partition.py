"""Host logic of hash-partitioned runs (Sec. V A) on the CPU: the owner of a determinant is its Algorithm 1
fingerprint mod the partition count, as the oracle computes the fingerprint; and the per-process exchange
step with two gloo ranks: every spawned entry reaches its owner exactly once, in source order, and the
counters and numerators are summed for the run's row."""
from __future__ import annotations

import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import bruteforce as bf
from oracle import oracle as O
from paper_1305_6981_gb300 import synth

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("which", ["8e8o", "24e60o"])
def test_owner_is_fingerprint_mod_partitions(which):
    from paper_1305_6981_gb300 import owners
    if which == "8e8o":
        s = synth.tiny_8e8o()
        dets = np.array([bf.to_words(d, 1) for d in bf.basis(8, 4, 4)[::7]], dtype=np.uint64)
    else:
        s = synth.large_24e60o()
        dets, _ = synth.walker_snapshot(s, 3000, seed=2)
    q = O.Oracle(s, tau=0.01)
    fps = np.array([q.fingerprint(d) for d in dets], dtype=object)
    for n_parts in (2, 3, 7):
        own = owners(s.n_orb, dets, n_parts)
        assert own.tolist() == [int(f % n_parts) for f in fps]
        assert len(set(own.tolist())) == n_parts  # every partition gets determinants
    with pytest.raises(Exception):
        owners(s.n_orb, dets, 0)


def _spawned_entries():
    s = synth.large_24e60o()
    keys, _ = synth.walker_snapshot(s, 20000, seed=5)
    rng = np.random.default_rng(8)
    amt = rng.integers(1, 6, len(keys)) * rng.choice([-1, 1], len(keys))
    vals = (rng.integers(0, 2, len(keys)) << 40) + amt  # (#initiator spawns << 40) + signed amount
    return s, keys, vals.astype(np.int64)


def _free_port() -> int:
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank: int, world: int, port: int, out) -> None:
    import torch.distributed as dist

    from paper_1305_6981_gb300 import owners
    from paper_1305_6981_gb300.partition import exchange, reduce_row, route
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s, keys, vals = _spawned_entries()
    mine = np.arange(len(keys)) % world == rank  # this rank's spawns
    dest = owners(s.n_orb, keys[mine], world)
    k, v, counts = route(keys[mine], vals[mine], dest, world)
    rk, rv = exchange(k, v, counts)
    row = {f: rank + 1 for f in ("nw_in", "nd_in", "c0_in", "nw_out", "nd_out", "attempts", "nulls", "spawn_events",
                                 "spawned_walkers", "death_walkers", "clone_walkers", "merged_entries",
                                 "aborted_walkers", "inserted_dets", "heavy_attempts")}
    row.update(iteration=7, shift=-0.25, num_in=0.1 + rank)
    out.put((rank, rk.tolist(), rv.tolist(), reduce_row(row)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_exchange_spawns_by_owner():
    from paper_1305_6981_gb300 import owners
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    s, keys, vals = _spawned_entries()
    own = owners(s.n_orb, keys, 2)
    src = np.arange(len(keys)) % 2
    for rank, rk, rv, row in res:
        # the entries owned by this rank, from source 0 then source 1, each in its original order
        expect = [(tuple(keys[i].tolist()), int(vals[i])) for srank in (0, 1)
                  for i in np.nonzero((own == rank) & (src == srank))[0]]
        assert list(zip(map(tuple, rk), rv)) == expect
        assert row["nw_in"] == 3 and row["heavy_attempts"] == 3 and row["iteration"] == 7
        assert row["num_in"] == 0.1 + 1.1 and row["shift"] == -0.25
    assert len(res[0][1]) + len(res[1][1]) == len(keys)
