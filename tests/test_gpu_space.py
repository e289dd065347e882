"""Permitted spaces (Sec. VI: excitations outside the space are null excitations) on the GPU, through
the C ABI, against the oracle: walker lists identical after every iteration, every integer counter
(including the null excitations) identical, the shift bit-identical."""
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


def make_pair(system, tau, thr, space, **kw):
    from paper_1305_6981_gb300 import Fciqmc
    caps = {k: kw.pop(k) for k in ("main_capacity", "spawn_capacity") if k in kw}
    g = Fciqmc(system, tau, thr, **space, **kw, **caps)
    q = Oracle(system, tau=tau, initiator_threshold=thr, **space, **kw)
    return g, q


def lockstep(g, q, n_iter):
    rows_q = []
    for k in range(n_iter):
        g.step(1)
        rows_q += q.iterate(1)
        assert same_lists(g.walkers(), q.walkers()), f"walker lists differ after iteration {k + 1}"
    compare_rows(g.history(n_iter), rows_q)
    return rows_q


def test_seniority_zero_8e8o():
    s = synth.tiny_8e8o()
    g, q = make_pair(s, 0.02, -1, dict(max_seniority=0), initial_population=500, initial_shift=0.2, seed=4,
                     main_capacity=1 << 12)
    rows = lockstep(g, q, 300)
    assert sum(r["nulls"] for r in rows) > 0
    d, _, _ = g.walkers()
    assert all(bin((int(w[0]) ^ (int(w[0]) >> 1)) & 0x5555).count("1") == 0 for w in d)  # closed shells only
    g.close()


def test_truncated_ci_12e24o_initiator():
    """CISD (at most two electrons away from the reference) with the initiator rule."""
    s = synth.init_12e24o()
    g, q = make_pair(s, 0.005, 3, dict(max_excitation=2), initial_population=3000, initial_shift=0.8, seed=8,
                     main_capacity=1 << 16)
    rows = lockstep(g, q, 120)
    assert sum(r["nulls"] for r in rows) > 0
    ref = int(q.info()["ref"][0])
    d, _, _ = g.walkers()
    assert max(bin(ref & ~int(w[0])).count("1") for w in d) == 2
    g.close()


def test_active_space_24e60o_heavy_path():
    """24e/60o (two words): spatial orbitals 0..3 frozen doubly occupied, 52..59 deleted, at most six singly
    occupied spatial orbitals; 5000 walkers on the reference exercise the heavy-determinant path."""
    s = synth.large_24e60o()
    core = bf.to_words((1 << 8) - 1, 2)
    deleted = bf.to_words(((1 << 16) - 1) << 104, 2)
    space = dict(frozen_occupied=core, frozen_empty=deleted, max_seniority=6)
    g, q = make_pair(s, 0.001, 3, space, initial_population=5000, initial_shift=2.0, seed=6,
                     main_capacity=1 << 16)
    # the reference's attempts read its tabulated doubles, those leaving the space marked as null
    # excitations: one entry per choice path of the (unrestricted) generator
    ref = q.info()["ref"]
    _, _, info = q.excite_ranks(ref, 2, 0, 0, 0)
    paths = 0
    for k1 in range(int(info[1])):
        _, _, i1 = q.excite_ranks(ref, 2, k1, 0, 0)
        for k2 in range(int(i1[2])):
            _, _, i2 = q.excite_ranks(ref, 2, k1, k2, 0)
            paths += int(i2[3])
    assert g.info()["reference_excitations"] == paths > 100_000
    rows = lockstep(g, q, 30)
    assert sum(r["nulls"] for r in rows) > 0
    d, _, _ = g.walkers()
    for w in d:
        x = bf.from_words(w)
        assert x & 0xFF == 0xFF and (x >> 104) & 0xFFFF == 0
    g.close()


def test_reference_and_lists_outside_the_space_rejected():
    from paper_1305_6981_gb300 import Fciqmc
    from paper_1305_6981_gb300._native import FciqmcError
    s = synth.tiny_8e8o()
    with pytest.raises(FciqmcError):
        Fciqmc(s, 0.01, -1, frozen_empty=[0b1], main_capacity=1 << 10)
    g = Fciqmc(s, 0.01, -1, max_excitation=2, main_capacity=1 << 10)
    before = g.walkers()
    triple = 0xFF ^ 0b111 ^ (0b111 << 8)  # three electrons moved: outside CISD
    with pytest.raises(FciqmcError):
        g.set_walkers(np.array([[0xFF], [triple]], dtype=np.uint64), np.array([5, 1], dtype=np.int32))
    assert same_lists(g.walkers(), before)
    g.close()
