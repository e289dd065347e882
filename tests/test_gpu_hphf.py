"""Spin-coupled functions (Sec. VI C) on the GPU, through the C ABI, against the oracle: walker lists
(stored determinants and populations) identical after every iteration, every integer counter identical,
the shift bit-identical, the projected-energy numerator within 1e-11 relative."""
from __future__ import annotations

import numpy as np
import pytest

import bruteforce as bf
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
    g = Fciqmc(system, tau, thr, hphf=True, **kw, **caps)
    q = Oracle(system, tau=tau, initiator_threshold=thr, hphf=True, **kw)
    return g, q


def lockstep(g, q, n_iter):
    rows_q = []
    for k in range(n_iter):
        g.step(1)
        rows_q += q.iterate(1)
        assert same_lists(g.walkers(), q.walkers()), f"walker lists differ after iteration {k + 1}"
    compare_rows(g.history(n_iter), rows_q)
    # the estimators of the final list (fciqmc_estimators), open-shell functions with their sqrt(2)
    e, est = g.estimates(), q.estimate()
    assert e["n_walkers"] == est["nw"] and e["n_dets"] == est["nd"] and e["c0"] == est["c0"]
    assert abs(e["proj_num"] - est["num"]) <= 1e-11 * max(abs(est["num"]), 1e-300)
    return rows_q


def stored(d: int, n_orb: int) -> bool:
    f = 0
    for p in range(n_orb):
        f |= ((d >> (2 * p + 1)) & 1) << (2 * p) | ((d >> (2 * p)) & 1) << (2 * p + 1)
    return d <= f


def test_plain_8e8o():
    s = synth.tiny_8e8o()
    g, q = make_pair(s, 0.02, -1, initial_population=500, initial_shift=0.2, seed=5, main_capacity=1 << 12)
    rows = lockstep(g, q, 300)
    d, p, _ = g.walkers()
    assert all(stored(int(w[0]), 8) for w in d)
    assert sum(bin((int(w[0]) ^ (int(w[0]) >> 1)) & 0x5555).count("1") > 0 for w in d) > 10  # open-shell functions
    assert rows[-1]["nd_out"] > 50
    g.close()


def test_initiator_12e24o():
    s = synth.init_12e24o()
    g, q = make_pair(s, 0.005, 3, initial_population=3000, initial_shift=0.8, seed=9, main_capacity=1 << 16)
    lockstep(g, q, 100)
    g.close()


def test_heavy_path_24e60o():
    """24e/60o (two words): 5000 walkers on the reference exercise the heavy-determinant path."""
    s = synth.large_24e60o()
    g, q = make_pair(s, 0.001, 3, initial_population=5000, initial_shift=2.0, seed=7, main_capacity=1 << 16)
    # the closed-shell reference's attempts read its tabulated doubles (target function and p): one entry per
    # choice path of the generator
    ref = q.info()["ref"]
    _, _, info = q.excite_ranks(ref, 2, 0, 0, 0)
    paths = 0
    for k1 in range(int(info[1])):
        _, _, i1 = q.excite_ranks(ref, 2, k1, 0, 0)
        for k2 in range(int(i1[2])):
            _, _, i2 = q.excite_ranks(ref, 2, k1, k2, 0)
            paths += int(i2[3])
    assert g.info()["reference_excitations"] == paths > 100_000
    lockstep(g, q, 30)
    d, _, _ = g.walkers()
    assert all(stored(bf.from_words(w), 60) for w in d)
    g.close()


def test_with_permitted_space_8e8o():
    s = synth.tiny_8e8o()
    g, q = make_pair(s, 0.02, -1, initial_population=500, initial_shift=0.2, seed=6, main_capacity=1 << 12,
                     max_seniority=2)
    rows = lockstep(g, q, 200)
    assert sum(r["nulls"] for r in rows) > 0
    g.close()


def test_requirements_and_loaded_lists():
    from paper_1305_6981_gb300 import Fciqmc
    from paper_1305_6981_gb300._native import FciqmcError
    with pytest.raises(FciqmcError):
        Fciqmc(synth.small_system(8, 6, seed=5), 0.01, -1, ms2=2, hphf=True, main_capacity=1 << 10)
    s = synth.tiny_8e8o()
    g = Fciqmc(s, 0.01, -1, hphf=True, main_capacity=1 << 10)
    before = g.walkers()
    d = 0xFF ^ 0b1 ^ (1 << 10)  # spin orbital 0 -> 10: an open-shell pair
    f = 0
    for p in range(8):
        f |= ((d >> (2 * p + 1)) & 1) << (2 * p) | ((d >> (2 * p)) & 1) << (2 * p + 1)
    larger = max(d, f)
    with pytest.raises(FciqmcError):
        g.set_walkers(np.array([[0xFF], [larger]], dtype=np.uint64), np.array([5, 1], dtype=np.int32))
    assert same_lists(g.walkers(), before)
    g.set_walkers(np.array([[0xFF], [min(d, f)]], dtype=np.uint64), np.array([5, 1], dtype=np.int32))
    q = Oracle(s, tau=0.01, hphf=True)
    q.set_walkers(np.array([[0xFF], [min(d, f)]], dtype=np.uint64), np.array([5, 1], dtype=np.int32))
    _, _, hg = g.walkers()
    _, _, hq = q.walkers()
    assert np.array_equal(np.sort(hg), np.sort(hq))  # spin-coupled diagonal elements, bit-identical
    g.close()
