"""Parity of the CUDA walker cycle with the CPU oracle, through the C ABI (GPU only).

Walker lists (determinant, population) must be identical after every iteration; every integer
counter of every iteration must be identical; the shift is bit-identical; the projected-energy
numerator agrees within 1e-11 relative (the GPU reduces it in a different order).
"""
from __future__ import annotations

import numpy as np
import pytest

import bruteforce as bf
from oracle.oracle import Oracle
from parity import canonical, compare_rows, same_lists
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


def run_lockstep(g, q, n_iter, every=1):
    """Advance both; compare walker lists every `every` iterations; return (gpu rows, oracle rows)."""
    rows_q = []
    for k in range(n_iter):
        g.step(1)
        rows_q += q.iterate(1)
        if (k + 1) % every == 0 or k + 1 == n_iter:
            assert same_lists(g.walkers(), q.walkers()), f"walker lists differ after iteration {k + 1}"
    return g.history(n_iter), rows_q


def test_setup_facts_match_oracle():
    for s in (synth.tiny_8e8o(), synth.init_12e24o(), synth.large_24e60o()):
        g, q = make_pair(s, 0.01, 3, main_capacity=1 << 12)
        gi, qi = g.info(), q.info()
        assert gi["e0"] == qi["E0"]
        assert gi["d53"] == qi["d53"] and gi["p_double"] == qi["p_double"]
        assert gi["n_single_ref"] == qi["n_single_ref"] and gi["n_double_ref"] == qi["n_double_ref"]
        assert np.array_equal(gi["reference"], qi["ref"])
        g.close()


def test_plain_8e8o_every_iteration():
    """8e/8o, no initiator, tau 0.01, 2^14 target walkers: every iteration of a 1000-iteration run."""
    s = synth.tiny_8e8o()
    g, q = make_pair(s, 0.01, -1, target_walkers=1 << 14, initial_population=1000, initial_shift=0.5, seed=5,
                     main_capacity=1 << 14)
    rows_q = []
    for k in range(1000):
        g.step(1)
        rows_q += q.iterate(1)
        assert same_lists(g.walkers(), q.walkers()), f"iteration {k + 1}"
    compare_rows(g.history(1000), rows_q)
    e = g.estimates()
    est = q.estimate()
    assert e["n_walkers"] == est["nw"] and e["c0"] == est["c0"] and e["n_dets"] == est["nd"]
    assert abs(e["proj_num"] - est["num"]) <= 1e-11 * abs(est["num"])
    assert e["vary_shift"] == 1
    g.close()


def test_initiator_12e24o_every_iteration():
    """12e/24o, 8 irreps, initiator threshold 3, tau 0.005."""
    s = synth.init_12e24o()
    g, q = make_pair(s, 0.005, 3, target_walkers=200000, initial_population=3000, initial_shift=1.0, seed=7,
                     main_capacity=1 << 17)
    rows, rows_q = run_lockstep(g, q, 150)
    compare_rows(rows, rows_q)
    assert sum(r["aborted_walkers"] for r in rows) > 0
    g.close()


def test_two_words_24e60o_heavy_reference():
    """24e/60o (two words), initiator 3, tau 0.001; 5000 walkers on the reference exercise the chunked
    heavy-determinant path."""
    s = synth.large_24e60o()
    g, q = make_pair(s, 0.001, 3, initial_population=5000, initial_shift=2.0, seed=3, main_capacity=1 << 16)
    # the reference's attempts read its tabulated doubles: one entry per choice path of the generator
    ref = q.info()["ref"]
    _, _, info = q.excite_ranks(ref, 2, 0, 0, 0)
    paths = 0
    for k1 in range(int(info[1])):
        _, _, i1 = q.excite_ranks(ref, 2, k1, 0, 0)
        for k2 in range(int(i1[2])):
            _, _, i2 = q.excite_ranks(ref, 2, k1, k2, 0)
            paths += int(i2[3])
    assert g.info()["reference_excitations"] == paths > 100_000
    rows_q = []
    for k in range(40):
        g.step(1)
        rows_q += q.iterate(1)
        assert same_lists(g.walkers(), q.walkers()), f"iteration {k + 1}"
    compare_rows(g.history(40), rows_q)
    g.close()


def test_heavy_path_one_word():
    s = synth.tiny_8e8o()
    g, q = make_pair(s, 0.01, 3, initial_population=20000, initial_shift=0.1, seed=9, main_capacity=1 << 13)
    assert g.info()["reference_excitations"] > 0
    rows_q = []
    for k in range(30):
        g.step(1)
        rows_q += q.iterate(1)
        assert same_lists(g.walkers(), q.walkers()), f"iteration {k + 1}"
    compare_rows(g.history(30), rows_q)
    g.close()


def test_snapshot_roundtrip_and_windows():
    """set_walkers from an oracle snapshot, then both advance identically (C ABI read/write path)."""
    s = synth.init_12e24o()
    g, q = make_pair(s, 0.005, 3, initial_population=2000, initial_shift=0.8, seed=21, main_capacity=1 << 16)
    q.iterate(60)
    d, p, hd = q.walkers()
    st = q.state()
    g.set_walkers(d, p, iteration=st["iteration"], shift=st["shift"], vary=st["vary"], shift_counter=st["n_since"],
                  nw_last_update=st["nw_prev"])
    dg, pg, hg = g.walkers()
    a = canonical(dg, pg, hg)
    b = canonical(d, p, hd)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])  # H_ii - E0 computed on the GPU, bit-identical
    rows_q = q.iterate(20)
    g.step(20)
    compare_rows(g.history(20), rows_q)
    assert same_lists(g.walkers(), q.walkers())
    g.close()


def _rejects_invalid_lists(g, dB, pB):
    """Invalid lists (wrong electron count, a bit beyond the basis, a zero population, a repeated
    determinant) are rejected on the device and leave the run's list as it was."""
    from paper_1305_6981_gb300._native import FciqmcError
    before = g.walkers()
    assert len(pB) > 8 and 2 * g.info()["n_orb"] < 64
    wrong_count, beyond_basis, zero_pop, repeated = dB.copy(), dB.copy(), pB.copy(), dB.copy()
    wrong_count[3, 0] ^= np.uint64(1 << 40)  # one electron more or fewer
    beyond_basis[5, 0] |= np.uint64(1 << 63)  # spin orbital 63 of a 48-spin-orbital basis
    zero_pop[7] = 0
    repeated[2] = repeated[len(pB) - 1]
    for dd, pp in ((wrong_count, pB), (beyond_basis, pB), (dB, zero_pop), (repeated, pB)):
        with pytest.raises(FciqmcError):
            g.set_walkers(dd, pp)
    assert same_lists(g.walkers(), before)


def test_reloads_and_invalid_lists():
    """Repeated set_walkers (the old list's index entries are located and emptied one by one before the new
    keys go in): after loading list A, running, and loading a different list B, both sides advance
    identically from B. Rejected lists leave the run as it was: the next iterations are the oracle's."""
    s = synth.init_12e24o()
    g, q = make_pair(s, 0.005, 3, initial_population=2000, initial_shift=0.8, seed=23, main_capacity=1 << 16)
    q.iterate(40)
    dA, pA, _ = q.walkers()
    g.set_walkers(dA, pA)
    g.step(5)
    q.iterate(40)
    dB, pB, hB = q.walkers()
    st = q.state()
    g.set_walkers(dB, pB, hB, iteration=st["iteration"], shift=st["shift"], vary=st["vary"],
                  shift_counter=st["n_since"], nw_last_update=st["nw_prev"])
    _rejects_invalid_lists(g, dB, pB)
    rows_q = q.iterate(25)
    g.step(25)
    compare_rows(g.history(25), rows_q)
    assert same_lists(g.walkers(), q.walkers())
    g.close()


def test_reloads_and_invalid_lists_dense_index():
    """The same with lists long against the index (more than 1/16 of its entries), where loading empties the
    whole index instead of the old list's entries one by one: synthetic lists of 1.9e3 and 2.6e3
    determinants, an index of 2^13 entries."""
    s = synth.init_12e24o()
    g, q = make_pair(s, 0.005, 3, seed=23, main_capacity=1 << 12)
    assert g.info()["index_capacity"] == 1 << 13
    dA, pA = synth.walker_snapshot(s, 6000, seed=3)
    g.set_walkers(dA, pA, iteration=10, shift=0.0, vary=0)
    g.step(5)
    dB, pB = synth.walker_snapshot(s, 8000, seed=4)
    assert len(pA) * 16 > 1 << 13 and len(pB) * 16 > 1 << 13
    g.set_walkers(dB, pB, iteration=20, shift=0.0, vary=0)
    q.set_walkers(dB, pB, iteration=20, shift=0.0)
    _rejects_invalid_lists(g, dB, pB)
    rows_q = q.iterate(25)
    g.step(25)
    compare_rows(g.history(25), rows_q)
    assert same_lists(g.walkers(), q.walkers())
    g.close()


@pytest.mark.parametrize("n_walkers,scale", [(30_000, 20), (900_000, 1)])
def test_short_and_long_lists_every_iteration(n_walkers, scale):
    """A list shorter than a quarter of the sweep's blocks in tiles (9.5e3 determinants with ~60 walkers each,
    so from the second iteration on the heavy path takes every determinant above 32 walkers) and a long one
    (2.9e5 determinants, threshold 256): both in lockstep with the oracle for 8 iterations."""
    s = synth.init_12e24o()
    g, q = make_pair(s, 0.005, 3, seed=31, main_capacity=1 << 21)
    d, p = synth.walker_snapshot(s, n_walkers, seed=6)
    p = (p.astype(np.int64) * scale).astype(np.int32)
    g.set_walkers(d, p, iteration=3, shift=0.3, vary=0)
    q.set_walkers(d, p, iteration=3, shift=0.3)
    rows_q = []
    for k in range(8):
        g.step(1)
        rows_q += q.iterate(1)
        assert same_lists(g.walkers(), q.walkers()), f"iteration {k + 1}"
    rows = g.history(8)
    compare_rows(rows, rows_q)
    if scale > 1:  # the lowered threshold sends most attempts to the heavy path after the first iteration
        assert rows[1]["heavy_attempts"] > 2 * rows[0]["heavy_attempts"]
    g.close()


def test_read_back_into_pinned_host_arrays():
    """get_walkers into page-locked host arrays (the benchmark's host-buffer path) gives the list read into
    pageable arrays, with or without the diagonal elements; arrays too small for the list give CAPACITY."""
    from paper_1305_6981_gb300._native import FciqmcError
    s = synth.init_12e24o()
    g, q = make_pair(s, 0.005, 3, seed=29, main_capacity=1 << 14)
    d0, p0 = synth.walker_snapshot(s, 8000, seed=4)
    g.set_walkers(d0, p0, iteration=5, shift=0.2, vary=0)
    q.set_walkers(d0, p0, iteration=5, shift=0.2)
    g.step(10)
    q.iterate(10)
    d, p, h = g.walkers()
    n = len(p)
    assert n > 1000
    W = d.shape[1]
    pd = torch.empty((n + 7, W), dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    pp = torch.empty(n + 7, dtype=torch.int32, pin_memory=True).numpy()
    ph = torch.empty(n + 7, dtype=torch.float64, pin_memory=True).numpy()
    assert g.walkers_into(pd, pp, ph) == n
    a, b = canonical(pd[:n], pp[:n], ph[:n]), canonical(d, p, h)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert same_lists((pd[:n], pp[:n]), q.walkers())
    pp[:] = 0
    assert g.walkers_into(pd, pp) == n
    assert same_lists((pd[:n], pp[:n]), (d, p))
    with pytest.raises(FciqmcError) as err:
        g.walkers_into(pd[: n - 1], pp[: n - 1], ph[: n - 1])
    assert err.value.status == -2
    assert same_lists(g.walkers(), (d, p))  # reading changes nothing
    g.close()


def test_duplicate_determinants_rejected():
    from paper_1305_6981_gb300._native import FciqmcError
    s = synth.tiny_8e8o()
    g, _ = make_pair(s, 0.01, -1, main_capacity=1 << 12)
    d = np.array([[0xFF], [0xFF]], dtype=np.uint64)
    with pytest.raises(FciqmcError):
        g.set_walkers(d, np.array([1, 2], dtype=np.int32))
    g.close()


def test_capacity_error_keeps_last_completed_state():
    """A main list too small for the run stops with CAPACITY; the list read back is the oracle's state
    at the last completed iteration."""
    from paper_1305_6981_gb300._native import FciqmcError
    s = synth.tiny_8e8o()
    g, q = make_pair(s, 0.02, -1, initial_population=3000, initial_shift=1.0, seed=2, main_capacity=1024)
    g.step(200)
    with pytest.raises(FciqmcError) as ei:
        g.sync()
    assert ei.value.status == -2
    done = g.state()["iteration"]
    assert 0 < done < 200
    q.iterate(done)
    assert same_lists(g.walkers(), q.walkers())
    g.close()


def test_gpu_run_is_deterministic():
    s = synth.init_12e24o()
    out = []
    for _ in range(2):
        from paper_1305_6981_gb300 import Fciqmc
        g = Fciqmc(s, 0.005, 3, initial_population=2000, initial_shift=1.0, seed=4, main_capacity=1 << 16)
        g.step(100)
        out.append(g.history(100))
        g.close()
    for a, b in zip(*out):
        for k in a:
            if k == "num_in":  # summed in slot order, which follows the order of atomic slot claims
                assert abs(a[k] - b[k]) <= 1e-12 * max(abs(b[k]), 1e-300)
            else:
                assert a[k] == b[k]


@pytest.mark.parametrize("cap", [1 << 13, 1 << 16])
def test_compaction_preserves_parity(cap):
    """A run with heavy determinant turnover triggers main-list compaction; parity holds across it. With
    2^16 slots (an index of 2^17 entries) the list is always short enough for the old entries to be
    emptied one by one; with 2^13 slots the longer lists clear the whole index."""
    s = synth.tiny_8e8o()
    g, q = make_pair(s, 0.05, 3, initial_population=3000, initial_shift=0.0, seed=13, main_capacity=cap)
    rows_q = []
    for k in range(150):
        g.step(1)
        rows_q += q.iterate(1)
    assert same_lists(g.walkers(), q.walkers())
    compare_rows(g.history(150), rows_q)
    assert g.estimates()["compactions"] > 0
    g.close()
