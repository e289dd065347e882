"""The walker cycle at full size against the oracle: 24e/60o (two-word determinants, 8 irreps, initiator 3,
tau 0.001) grown on the GPU and settled to the steady state the benchmark times (~1.4e8 walkers on ~6e6
determinants), in its launch configuration (its workload table: 2e8-slot main list, 2^27-entry spawn table). From the grown list, one iteration
on the GPU and one in the oracle: diagonal elements of the loaded list bit-identical, walker lists
identical, every integer counter identical, the shift bit-identical, the projected-energy numerator within
1e-11 relative; the list loaded back through set_walkers gives the same iteration again. The oracle's
iteration takes a minute or two on the host cores. The same for the
active-space and spin-coupled workloads at 1e7 target walkers."""
from __future__ import annotations

import argparse

import numpy as np
import pytest

from oracle.oracle import Oracle
from parity import canonical, compare_rows, same_lists

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def one_iteration(workload: str, target: int = 0):
    """Grow the benchmark workload on the GPU, then one iteration on the GPU and in the oracle from the
    same list; returns the GPU row and the loaded list."""
    import bench
    wl = bench.WORKLOADS[workload]
    g, _, _, _ = bench.grow(argparse.Namespace(target=target, workload=workload), wl, 0)
    g.step(3)
    d, p, h = g.walkers()
    st = g.state()
    g.step(1)
    rows_g = g.history(1)
    after = g.walkers()
    # the same list loaded back through set_walkers (the copy in chunks, each chunk's keys inserted into the
    # index as it arrives): the same iteration again, with the same result
    g.set_walkers(d, p, h, iteration=st["iteration"], shift=st["shift"], vary=st["vary_shift"],
                  shift_counter=st["shift_counter"], nw_last_update=st["nw_last_update"])
    g.step(1)
    again = g.history(1)
    compare_rows(again, [dict(r, iter=r["iteration"]) for r in rows_g])
    assert again[0]["heavy_attempts"] == rows_g[0]["heavy_attempts"]
    assert same_lists(g.walkers(), after)
    g.close()

    q = Oracle(wl["system"](), tau=wl["tau"], initiator_threshold=wl["thr"], target_walkers=target or wl["target"],
               initial_population=wl["initial_population"], initial_shift=wl["initial_shift"],
               seed=bench.replica_seed(0), **wl.get("space", {}))
    q.set_walkers(d, p, iteration=st["iteration"], shift=st["shift"], vary=bool(st["vary_shift"]),
                  nw_prev=st["nw_last_update"], n_since=st["shift_counter"])
    dq, pq, hq = q.walkers()
    a, b = canonical(d, p, h), canonical(dq, pq, hq)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])  # H_ii - E0, bit-identical
    rows_q = q.iterate(1)
    compare_rows(rows_g, rows_q)
    assert same_lists(after, q.walkers())
    return rows_g[0], p


def test_one_iteration_at_1e8_walkers():
    r, p = one_iteration("24e60o")
    assert len(p) > 3_000_000 and int(np.abs(p.astype(np.int64)).sum()) > 80_000_000
    assert int(np.abs(p).max()) > 1_000_000  # millions of attempts from one determinant (heavy path)
    assert r["heavy_attempts"] > r["attempts"] // 2 and r["spawn_events"] > 100_000


@pytest.mark.parametrize("workload", ["24e60o-cas", "24e60o-hphf"])
def test_one_iteration_at_1e7_walkers_with_space_or_spin_coupling(workload):
    """The active-space and spin-coupled workloads of the benchmark at 1e7 target walkers."""
    r, p = one_iteration(workload, 10_000_000)
    assert int(np.abs(p.astype(np.int64)).sum()) > 5_000_000
    assert r["heavy_attempts"] > r["attempts"] // 2 and r["spawn_events"] > 10_000
    if workload.endswith("cas"):
        assert r["nulls"] > 0


def test_one_iteration_partitioned_at_1e7_walkers():
    """The grown 24e/60o list (1e7 target, settled) loaded into a run of three hash partitions: one iteration of
    the group against one oracle iteration from the same list, every counter, the shift and the union of the
    partitions' lists identical."""
    import bench
    from paper_1305_6981_gb300 import Partitioned
    wl = bench.WORKLOADS["24e60o"]
    g0, _, _, _ = bench.grow(argparse.Namespace(target=10_000_000, workload="24e60o"), wl, 0)
    d, p, h = g0.walkers()
    st = g0.state()
    g0.close()
    g = Partitioned(wl["system"](), wl["tau"], wl["thr"], n_partitions=3, target_walkers=10_000_000,
                    main_capacity=2 * len(p), spawn_capacity=1 << 23, outbox_capacity=1 << 20, seed=1)
    g.set_walkers(d, p, h, iteration=st["iteration"], shift=st["shift"], vary=st["vary_shift"],
                  shift_counter=st["shift_counter"], nw_last_update=st["nw_last_update"])
    g.step(1)
    rows_g = g.history(1)
    after = g.walkers()
    g.close()
    q = Oracle(wl["system"](), tau=wl["tau"], initiator_threshold=wl["thr"], target_walkers=10_000_000, seed=1)
    q.set_walkers(d, p, iteration=st["iteration"], shift=st["shift"], vary=bool(st["vary_shift"]),
                  nw_prev=st["nw_last_update"], n_since=st["shift_counter"])
    compare_rows(rows_g, q.iterate(1))
    assert same_lists(after, q.walkers())
    assert int(np.abs(p.astype(np.int64)).sum()) > 5_000_000 and rows_g[0]["spawn_events"] > 10_000


def test_one_iteration_hybrid_at_1e7_walkers():
    """The hybrid-walker workload of the benchmark (units of 1/16 walker) grown to a 1e7 target and settled: one
    iteration on the GPU and in the oracle from the same list, identical."""
    r, p = one_iteration("24e60o-real", 10_000_000)
    a = np.abs(p.astype(np.int64))
    assert a.sum() > 5_000_000 * 16 and np.all(a >= 16) and np.any(a % 16 != 0)
    assert r["heavy_attempts"] > r["attempts"] // 2
