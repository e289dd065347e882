"""Batched runs (one CUDA graph advancing several independent runs) give exactly the results of the same
runs advanced one at a time, each batched run matches the oracle, and the launch-shape options the autotuner
varies never change results."""
from __future__ import annotations

import numpy as np
import pytest

from oracle.oracle import Oracle
from parity import compare_rows, same_lists
from paper_1305_6981_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _same_rows(a, b):
    """Identical rows except the FP64 projected-energy numerator, which is summed in list order (slot order
    depends on the order of atomic slot claims) and agrees to rounding."""
    assert len(a) == len(b)
    for x, y in zip(a, b):
        for k in x:
            if k == "num_in":
                assert abs(x[k] - y[k]) <= 1e-12 * max(abs(y[k]), 1e-300)
            else:
                assert x[k] == y[k], (k, x[k], y[k])


def _runs(specs, **extra):
    from paper_1305_6981_gb300 import Fciqmc
    out = []
    for sp in specs:
        s = synth.make_system(sp["n_orb"], sp["n_elec"], seed=sp["sys_seed"] % 1000, n_chol=8)
        out.append(Fciqmc(s, 0.005, 3, target_walkers=sp["target"], initial_population=500, initial_shift=1.0,
                          seed=sp["seed"], main_capacity=1 << 16, spawn_capacity=1 << 14, **extra))
    return out


def test_batched_equals_one_at_a_time():
    from paper_1305_6981_gb300 import Batch
    specs = synth.batch_systems(6, seed=3)
    for sp in specs:
        sp["target"] = 5000
    a = _runs(specs)
    b = _runs(specs)
    batch = Batch(a, iterations_per_launch=7)
    batch.step(6)  # 42 iterations each
    for r in b:
        r.step(42)
    for ra, rb in zip(a, b):
        assert ra.sync() == 0 and rb.sync() == 0
        _same_rows(ra.history(42), rb.history(42))
        assert same_lists(ra.walkers(), rb.walkers())
        assert ra.state()["iteration"] == 42
    batch.close()
    for r in a + b:
        r.close()


def test_launch_shape_options_do_not_change_results():
    specs = synth.batch_systems(2, seed=5)
    for sp in specs:
        sp["target"] = 20000
    ref = _runs(specs)
    alt = _runs(specs, grid_blocks=7, index_load=0.2)
    for r in ref + alt:
        r.step(60)
    for r1, r2 in zip(ref, alt):
        _same_rows(r1.history(60), r2.history(60))
        assert same_lists(r1.walkers(), r2.walkers())
        r1.close()
        r2.close()


def test_batched_runs_match_the_oracle():
    """Four uneven runs advanced together by the batch graph: every run's history (counters, shift) and
    final walker list equal the oracle's for the same system and options."""
    from paper_1305_6981_gb300 import Batch
    specs = synth.batch_systems(4, seed=7)
    for sp in specs:
        sp["target"] = 4000
    runs = _runs(specs)
    batch = Batch(runs, iterations_per_launch=5)
    batch.step(6)  # 30 iterations each
    for sp, r in zip(specs, runs):
        assert r.sync() == 0
        s = synth.make_system(sp["n_orb"], sp["n_elec"], seed=sp["sys_seed"] % 1000, n_chol=8)
        q = Oracle(s, tau=0.005, initiator_threshold=3, target_walkers=sp["target"], initial_population=500,
                   initial_shift=1.0, seed=sp["seed"])
        rows_q = q.iterate(30)
        compare_rows(r.history(30), rows_q)
        assert same_lists(r.walkers(), q.walkers())
        assert rows_q[-1]["nd_out"] > 20
    batch.close()
    for r in runs:
        r.close()
