"""Invariants of the oracle's dynamics that hold for any correct FCIQMC iteration (CPU only).

Every determinant keeps the electron count, the M_s and the spatial symmetry of the reference; the list
holds distinct determinants with nonzero populations; the row's determinant count is the list's. The
walker count obeys two exact relations: annihilation only ever removes walkers, so
N_w(out) <= N_w(in) + deaths + clones + applied spawns, and since |C| and C have the same parity,
N_w(out) and N_w(in) + deaths + clones + applied spawns have the same parity (applied spawns = spawned
walkers minus those the initiator rule aborted).
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import bruteforce as bf
from oracle import oracle as O
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


def test_thread_count_does_not_change_results():
    """The oracle splits a determinant's attempts into chunks spread over threads; one thread and several
    threads give identical lists and counters (the reference holds several chunks' worth of walkers)."""
    s = synth.init_12e24o()
    dets, pops = synth.walker_snapshot(s, 60_000, seed=3, ref_fraction=0.5)
    out = []
    for threads in (1, 6):
        O.set_threads(threads)
        q = O.Oracle(s, tau=0.005, initiator_threshold=3, seed=9)
        q.set_walkers(dets, pops, iteration=40, shift=0.3)
        rows = q.iterate(3)
        d, p, _ = q.walkers()
        out.append((rows, sorted(zip(map(tuple, d.tolist()), p.tolist()))))
    O.set_threads(os.cpu_count() or 1)
    assert max(abs(int(x)) for x in pops) > 4 * 4096
    assert out[0][1] == out[1][1]
    for a, b in zip(out[0][0], out[1][0]):
        assert {k: v for k, v in a.items() if k != "num_in"} == {k: v for k, v in b.items() if k != "num_in"}
        assert abs(a["num_in"] - b["num_in"]) <= 1e-12 * max(1.0, abs(a["num_in"]))
