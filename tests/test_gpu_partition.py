"""Hash-partitioned runs (Sec. V A) on the GPU through the C ABI (fciqmc_group_*), against the oracle's
unpartitioned run: the random numbers are keyed by determinant and iteration, not by partition, so the union
of the partitions' lists must equal the oracle's list after every iteration, the run's rows (counters summed
over partitions) must equal the oracle's rows, and each partition must hold only its own determinants."""
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


def _lockstep(system, tau, thr, n_parts, n_iter, caps, **kw):
    from paper_1305_6981_gb300 import Partitioned, owners
    g = Partitioned(system, tau, thr, n_partitions=n_parts, **caps, **kw)
    q = Oracle(system, tau=tau, initiator_threshold=thr, **kw)
    rows_q = []
    for k in range(n_iter):
        g.step(1)
        rows_q += q.iterate(1)
        assert same_lists(g.walkers(), q.walkers()), f"walker lists differ after iteration {k + 1}"
    assert g.sync() == 0
    rows = g.history(n_iter)
    compare_rows(rows, rows_q)
    for r, p in enumerate(g.parts):  # each partition holds exactly its own determinants
        d, _, _ = p.walkers()
        assert np.all(owners(system.n_orb, d, n_parts) == r)
    assert min(len(p.walkers()[1]) for p in g.parts) > 0
    e, est = g.estimates(), q.estimate()
    assert e["n_walkers"] == est["nw"] and e["n_dets"] == est["nd"] and e["c0"] == est["c0"]
    assert abs(e["proj_num"] - est["num"]) <= 1e-11 * max(abs(est["num"]), 1e-300)
    g.close()
    return rows


@pytest.mark.parametrize("n_parts", [2, 3])
def test_partitioned_8e8o_plain(n_parts):
    rows = _lockstep(synth.tiny_8e8o(), 0.01, -1, n_parts, 300, dict(main_capacity=1 << 14),
                     target_walkers=1500, initial_population=1000, initial_shift=0.5, seed=5)
    assert any(r["shift"] != rows[0]["shift"] for r in rows)  # the shift varied with the run's N_w


@pytest.mark.parametrize("n_parts", [2, 3])
def test_partitioned_12e24o_initiator(n_parts):
    rows = _lockstep(synth.init_12e24o(), 0.005, 3, n_parts, 120, dict(main_capacity=1 << 17),
                     target_walkers=200000, initial_population=3000, initial_shift=1.0, seed=7)
    assert sum(r["aborted_walkers"] for r in rows) > 0


def test_partitioned_24e60o_heavy_two_words():
    rows = _lockstep(synth.large_24e60o(), 0.001, 3, 3, 40, dict(main_capacity=1 << 16),
                     initial_population=5000, initial_shift=2.0, seed=3)
    assert sum(r["heavy_attempts"] for r in rows) > 0


@pytest.mark.parametrize("mode", ["spin-coupled", "cisd"])
def test_partitioned_with_spin_coupling_or_space(mode):
    """Spin-coupled functions are routed by the fingerprint of their stored determinant; excitations outside
    a permitted space stay null excitations in every partition."""
    kw = dict(hphf=True) if mode == "spin-coupled" else dict(max_excitation=2)
    rows = _lockstep(synth.init_12e24o(), 0.005, 3, 2, 80, dict(main_capacity=1 << 17),
                     target_walkers=100000, initial_population=3000, initial_shift=1.0, seed=11, **kw)
    if mode == "cisd":
        assert sum(r["nulls"] for r in rows) > 0


def test_partitioned_outbox_overflow_stops_every_partition():
    """An outbox too small for the iteration's routed spawns stops the iteration in every partition before
    any list changes, and the error stays set."""
    from paper_1305_6981_gb300 import Partitioned, _native
    s = synth.large_24e60o()
    g = Partitioned(s, 0.005, 3, n_partitions=2, main_capacity=1 << 18, outbox_capacity=8, seed=3)
    d0, p0 = synth.walker_snapshot(s, 100_000, seed=11)
    g.set_walkers(d0, p0)
    before = g.walkers()
    g.step(2)
    with pytest.raises(_native.FciqmcError) as err:
        g.sync()
    assert err.value.status == -2  # FCIQMC_ERR_CAPACITY
    assert all(p.estimates()["status"] == -2 for p in g.parts)
    assert same_lists(g.walkers(), before)
    assert g.history(10) == []
    g.close()


def test_partitioned_handles_refuse_single_stepping():
    from paper_1305_6981_gb300 import Fciqmc, _native
    s = synth.tiny_8e8o()
    h = Fciqmc(s, 0.01, -1, n_partitions=2, partition_index=1, main_capacity=1 << 12)
    with pytest.raises(_native.FciqmcError):
        h.step(1)
    with pytest.raises(_native.FciqmcError):  # a determinant of the other partition
        from paper_1305_6981_gb300 import owners
        d, p = synth.walker_snapshot(s, 2000, seed=1)
        own = owners(s.n_orb, d, 2)
        h.set_walkers(d[own == 0], p[own == 0])
    h.close()
