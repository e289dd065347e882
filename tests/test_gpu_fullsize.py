"""The walker cycle at full size against the oracle: 24e/60o (two-word determinants, 8 irreps, initiator 3,
tau 0.001) grown on the GPU to ~1e8 walkers on ~4e6 determinants, in the launch configuration the benchmark
times (its workload table: 2e8-slot main list, 2^27-entry spawn table). From the grown list, one iteration
on the GPU and one in the oracle: diagonal elements of the loaded list bit-identical, walker lists
identical, every integer counter identical, the shift bit-identical, the projected-energy numerator within
1e-11 relative. The oracle's iteration takes a minute or two on the host cores."""
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


def test_one_iteration_at_1e8_walkers():
    import bench
    wl = bench.WORKLOADS["24e60o"]
    g, _, _, _ = bench.grow(argparse.Namespace(target=0, workload="24e60o"), wl, 0)
    g.step(3)
    d, p, h = g.walkers()
    st = g.state()
    assert len(p) > 3_000_000 and int(np.abs(p.astype(np.int64)).sum()) > 80_000_000
    assert int(np.abs(p).max()) > 1_000_000  # the reference: millions of attempts from one determinant
    g.step(1)
    rows_g = g.history(1)
    after = g.walkers()
    g.close()
    r = rows_g[0]
    assert r["heavy_attempts"] > r["attempts"] // 2 and r["spawn_events"] > 100_000

    q = Oracle(wl["system"](), tau=wl["tau"], initiator_threshold=wl["thr"], target_walkers=wl["target"],
               initial_population=wl["initial_population"], initial_shift=wl["initial_shift"],
               seed=bench.replica_seed(0))
    q.set_walkers(d, p, iteration=st["iteration"], shift=st["shift"], vary=bool(st["vary_shift"]),
                  nw_prev=st["nw_last_update"], n_since=st["shift_counter"])
    dq, pq, hq = q.walkers()
    a, b = canonical(d, p, h), canonical(dq, pq, hq)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])  # H_ii - E0, bit-identical
    rows_q = q.iterate(1)
    compare_rows(rows_g, rows_q)
    assert same_lists(after, q.walkers())
