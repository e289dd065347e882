"""The 12e/24o workload at its stated configuration (8 irreps, initiator threshold 3, tau 0.005, 1e6 target
walkers) on the GPU through the C ABI against the oracle, every iteration from the reference: the growth
phase, the shift starting to vary when N_w first reaches 1e6, and 300 iterations with the shift varying.
After every iteration the walker lists are identical; every integer counter and the shift are identical and
the projected-energy numerator agrees within 1e-11 relative (compared over the whole history at the end).
About 1550 iterations in all (the oracle takes a few minutes on 16 host cores)."""
from __future__ import annotations

import pytest

from oracle.oracle import Oracle
from parity import compare_rows, same_lists
from paper_1305_6981_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

VARY_ITERATIONS = 300


def test_12e24o_at_1e6_walkers_every_iteration():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1305_6981_gb300 import Fciqmc

    s = synth.init_12e24o()
    kw = dict(target_walkers=1_000_000, initial_population=2000, initial_shift=1.0, seed=7)
    g = Fciqmc(s, 0.005, 3, main_capacity=1 << 21, spawn_capacity=1 << 20, **kw)
    q = Oracle(s, tau=0.005, initiator_threshold=3, **kw)
    rows_q = []
    vary_at = None
    k = 0
    while k < 4000:
        g.step(1)
        rows_q += q.iterate(1)
        k += 1
        assert same_lists(g.walkers(), q.walkers()), f"walker lists differ after iteration {k}"
        if vary_at is None and q.state()["vary"]:
            vary_at = k
        if vary_at is not None and k >= vary_at + VARY_ITERATIONS:
            break
    assert vary_at is not None and k == vary_at + VARY_ITERATIONS
    rows = g.history(k)
    compare_rows(rows, rows_q)
    assert max(r["nw_out"] for r in rows) >= 1_000_000
    assert len({r["shift"] for r in rows[vary_at:]}) > 10  # the shift varies
    assert sum(r["aborted_walkers"] for r in rows) > 0  # the initiator rule acts
    g.close()
