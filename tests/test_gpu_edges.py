"""Edge cases of the walker cycle on the GPU against the oracle, through the C ABI: the largest supported
size (64 electrons in 64 spatial orbitals: both words of every determinant full, 2016 electron pairs),
a single electron (no pairs, so every attempt is a single), two electrons in two orbitals (a four-
determinant space), and an empty walker list. Walker lists identical after every iteration, every
integer counter identical, the shift bit-identical."""
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


def make_pair(system, tau, thr, **kw):
    from paper_1305_6981_gb300 import Fciqmc
    caps = {k: kw.pop(k) for k in ("main_capacity", "spawn_capacity") if k in kw}
    g = Fciqmc(system, tau, thr, **kw, **caps)
    q = Oracle(system, tau=tau, initiator_threshold=thr, **kw)
    return g, q


def lockstep(g, q, n_iter):
    rows_q = []
    for k in range(n_iter):
        g.step(1)
        rows_q += q.iterate(1)
        assert same_lists(g.walkers(), q.walkers()), f"walker lists differ after iteration {k + 1}"
    compare_rows(g.history(n_iter), rows_q)
    return rows_q


def test_largest_supported_size_64e64o():
    """8 irreps, slowly decaying Cholesky vectors and a near-degenerate window at the Fermi level, so
    that the reference spawns onto hundreds of determinants per iteration."""
    s = synth.make_system(64, 64, seed=11, n_chol=64, symmetry=True, chol_decay_len=8.0,
                          energies=synth.frontier_energies(64, lo=28, hi=35), name="64e64o")
    g, q = make_pair(s, 0.002, 3, initial_population=3000, initial_shift=0.0, seed=4, main_capacity=1 << 16)
    info = g.info()
    assert info["words"] == 2 and info["reference_excitations"] > 0
    ref = info["reference"]
    assert int(ref[0]) == (1 << 64) - 1 and int(ref[1]) == 0  # 32 doubly occupied orbitals fill word 0
    rows = lockstep(g, q, 6)
    assert rows[-1]["nd_out"] > 100 and sum(r["spawn_events"] for r in rows) > 100
    g.close()


def test_one_electron_only_singles():
    s = synth.small_system(6, 1, seed=2)
    g, q = make_pair(s, 0.01, -1, ms2=1, initial_population=200, initial_shift=0.1, seed=8, main_capacity=1 << 10)
    assert g.info()["n_double_ref"] == 0 and g.info()["p_double"] == 0.0
    rows = lockstep(g, q, 200)
    d, _, _ = g.walkers()
    assert len(d) >= 3  # the electron has left the reference orbital
    assert sum(r["spawn_events"] for r in rows) > 0
    g.close()


def test_two_electrons_in_two_orbitals():
    s = synth.small_system(2, 2, seed=3)
    g, q = make_pair(s, 0.01, -1, initial_population=100, initial_shift=0.1, seed=6, main_capacity=1 << 10)
    lockstep(g, q, 200)
    d, _, _ = g.walkers()
    assert 1 < len(d) <= 4
    g.close()


def test_empty_walker_list():
    s = synth.tiny_8e8o()
    g, q = make_pair(s, 0.01, -1, initial_population=50, seed=2, main_capacity=1 << 10)
    none_d = np.zeros((0, 1), dtype=np.uint64)
    none_p = np.zeros(0, dtype=np.int32)
    g.set_walkers(none_d, none_p, iteration=7, shift=0.3, vary=0)
    q.set_walkers(none_d, none_p, iteration=7, shift=0.3)
    rows = lockstep(g, q, 3)
    assert all(r["nw_out"] == 0 and r["attempts"] == 0 for r in rows)
    assert len(g.walkers()[1]) == 0
    g.close()
