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
    """Sixteen uneven runs of the 64-run workload's kind (8e/16o to 16e/40o, targets 600 to 3000) advanced
    together by the batch graph for 150 iterations, the shift varying in most of them: every run's history
    (counters, shift) and final walker list equal the oracle's for the same system and options."""
    from paper_1305_6981_gb300 import Batch
    specs = synth.batch_systems(16, seed=7)
    rng = np.random.default_rng(3)
    for sp in specs:
        sp["target"] = int(np.exp(rng.uniform(np.log(600), np.log(3000))))
    runs = _runs(specs)
    batch = Batch(runs, iterations_per_launch=10)
    batch.step(15)  # 150 iterations each
    varied = 0
    for sp, r in zip(specs, runs):
        assert r.sync() == 0
        s = synth.make_system(sp["n_orb"], sp["n_elec"], seed=sp["sys_seed"] % 1000, n_chol=8)
        q = Oracle(s, tau=0.005, initiator_threshold=3, target_walkers=sp["target"], initial_population=500,
                   initial_shift=1.0, seed=sp["seed"])
        rows_q = q.iterate(150)
        compare_rows(r.history(150), rows_q)
        assert same_lists(r.walkers(), q.walkers())
        assert rows_q[-1]["nd_out"] > 20
        varied += q.state()["vary"]
    assert varied >= 8
    batch.close()
    for r in runs:
        r.close()


def test_tuner_chooses_a_candidate_whose_run_matches_the_oracle():
    """The autotuner times every candidate (block count, index load factor, spawn-table size) from one grown
    snapshot and returns the fastest one; a run created with its choice matches the oracle iteration for
    iteration (launch shapes never change results). Bucketed tuning gives each run its bucket's choice."""
    from paper_1305_6981_gb300 import Fciqmc
    from paper_1305_6981_gb300.autotune import DEFAULT_CANDIDATES, bucket_of, tune, tune_buckets
    s = synth.make_system(12, 6, seed=3, n_chol=8)
    r = tune(s, 0.005, 3, 5000, trial_iterations=5)
    n_cand = 1
    for v in DEFAULT_CANDIDATES.values():
        n_cand *= len(v)
    assert len(r["trials"]) == n_cand and all(t["status"] == 0 for t in r["trials"])
    best = r["best"]
    assert best["grid_blocks"] in DEFAULT_CANDIDATES["grid_blocks"]
    assert best["index_load"] in DEFAULT_CANDIDATES["index_load"]
    assert r["ms_per_iteration"] == min(t["ms_per_iteration"] for t in r["trials"])
    g = Fciqmc(s, 0.005, 3, target_walkers=5000, initial_population=300, initial_shift=1.0, seed=9, **best)
    q = Oracle(s, tau=0.005, initiator_threshold=3, target_walkers=5000, initial_population=300,
               initial_shift=1.0, seed=9)
    g.step(40)
    compare_rows(g.history(40), q.iterate(40))
    assert same_lists(g.walkers(), q.walkers())
    g.close()
    small = dict(grid_blocks=[0, 38], index_load=[0.5], spawn_factor=[0.5])
    targets = [3000, 3500, 9000]
    per_run, buckets = tune_buckets([s, s, s], targets, 0.005, 3, trial_iterations=3, candidates=small)
    assert set(buckets) == {bucket_of(t) for t in targets} and len(buckets) == 2
    assert per_run[0] == per_run[1] == buckets[bucket_of(3000)]["best"]
