"""Invariants of the oracle's dynamics that hold for any correct FCIQMC iteration (CPU only).

Every determinant keeps the electron count, the M_s and the spatial symmetry of the reference; the list
holds distinct determinants with nonzero populations; the row's determinant count is the list's. The
walker count obeys two exact relations: annihilation only ever removes walkers, so
N_w(out) <= N_w(in) + deaths + clones + applied spawns, and since |C| and C have the same parity,
N_w(out) and N_w(in) + deaths + clones + applied spawns have the same parity (applied spawns = spawned
walkers minus those the initiator rule aborted).
"""
from __future__ import annotations

import numpy as np
import pytest

import bruteforce as bf
from oracle.oracle import Oracle
from paper_1305_6981_gb300 import synth


def _irrep_product(d: int, irrep: np.ndarray) -> int:
    g = 0
    k = 0
    while d:
        if d & 1:
            g ^= int(irrep[k >> 1])
        d >>= 1
        k += 1
    return g


@pytest.mark.parametrize("thr", [-1, 3])
def test_every_iteration_keeps_the_invariants(thr):
    s = synth.init_12e24o()
    q = Oracle(s, tau=0.05, initiator_threshold=thr, initial_population=2000, initial_shift=0.6, seed=17,
               target_walkers=6000)
    ref = int(q.info()["ref"][0])
    g_ref = _irrep_product(ref, s.irrep)
    alpha = sum(1 << (2 * p) for p in range(s.n_orb))
    n_iter = 120
    aborted = 0
    for k in range(n_iter):
        r = q.iterate(1)[0]
        d, p, _ = q.walkers()
        words = [bf.from_words(w) for w in d]
        assert len(set(words)) == len(words), k  # distinct determinants
        assert np.all(p != 0) and r["nd_out"] == len(words)
        assert r["nw_out"] == int(np.abs(p.astype(np.int64)).sum())
        for x in words:
            assert bin(x).count("1") == s.n_elec
            assert bin(x & alpha).count("1") == s.n_elec // 2  # M_s = 0
            assert _irrep_product(x, s.irrep) == g_ref
        bound = r["nw_in"] + r["death_walkers"] + r["clone_walkers"] + r["spawned_walkers"] - r["aborted_walkers"]
        assert r["nw_out"] <= bound, k
        assert (bound - r["nw_out"]) % 2 == 0, k
        aborted += r["aborted_walkers"]
    assert r["nd_out"] > 50 and r["iter"] == n_iter - 1
    assert (aborted > 0) == (thr >= 0)  # the initiator rule is active only when it is on
