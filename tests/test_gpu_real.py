"""Real/integer hybrid walkers on the GPU through the C ABI against the oracle: populations in units of
2^-b walkers, attempts rounded stochastically, spawns drawn in units, the occupation threshold applied
after annihilation. Walker lists identical after every iteration, every counter and the shift identical,
the numerator within 1e-11; no amplitude below the threshold survives an iteration."""
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


def _lockstep(system, tau, thr, n_iter, caps, bits, occ, n_parts=1, **kw):
    from paper_1305_6981_gb300 import Fciqmc, Partitioned
    opts = dict(walker_fraction_bits=bits, occupation_threshold=occ, **kw)
    g = (Fciqmc(system, tau, thr, **caps, **opts) if n_parts == 1
         else Partitioned(system, tau, thr, n_partitions=n_parts, **caps, **opts))
    q = Oracle(system, tau=tau, initiator_threshold=thr, **opts)
    occ_units = round(occ * (1 << bits))
    rows_q = []
    fractional = 0
    for k in range(n_iter):
        g.step(1)
        rows_q += q.iterate(1)
        d, p, _ = g.walkers()
        assert same_lists((d, p), q.walkers()), f"walker lists differ after iteration {k + 1}"
        a = np.abs(p.astype(np.int64))
        assert np.all(a >= occ_units)  # nothing below the occupation threshold
        fractional += int(np.sum(a % (1 << bits) != 0))
    rows = g.history(n_iter)
    compare_rows(rows, rows_q)
    assert fractional > 0  # amplitudes off the integer grid occur
    g.close()
    return rows


def test_hybrid_8e8o_plain():
    rows = _lockstep(synth.tiny_8e8o(), 0.01, -1, 300, dict(main_capacity=1 << 14), 8, 1.0,
                     target_walkers=1500, initial_population=500, initial_shift=0.5, seed=5)
    assert any(r["attempts"] * 256 != r["nw_in"] for r in rows)  # attempts are rounded walker counts


def test_hybrid_12e24o_initiator_threshold_two_walkers():
    _lockstep(synth.init_12e24o(), 0.005, 3, 100, dict(main_capacity=1 << 17), 6, 2.0,
              target_walkers=100000, initial_population=2000, initial_shift=1.0, seed=7)


def test_hybrid_24e60o_heavy_two_words():
    rows = _lockstep(synth.large_24e60o(), 0.001, 3, 30, dict(main_capacity=1 << 16), 4, 1.0,
                     initial_population=4000, initial_shift=2.0, seed=3)
    assert sum(r["heavy_attempts"] for r in rows) > 0


def test_hybrid_partitioned_8e8o():
    _lockstep(synth.tiny_8e8o(), 0.01, -1, 150, dict(main_capacity=1 << 14), 8, 1.0, n_parts=2,
              target_walkers=1500, initial_population=500, initial_shift=0.5, seed=5)
