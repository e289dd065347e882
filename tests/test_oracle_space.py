"""Pins of the oracle's permitted spaces (CPU only).

Sec. VI: restrictions on the space are imposed by returning a null excitation whenever the excitation
generator produces a determinant outside the permitted space; the generation probabilities of the
excitations that remain are unchanged. The oracle's membership test is checked against the
definitions written out on Python integers (excitation level relative to the reference, seniority,
frozen spin orbitals), and one step of the dynamics against Eq. 1 with the Hamiltonian projected onto
the space; a truncated run reaches the lowest eigenvalue of the projected Hamiltonian.
"""
from __future__ import annotations

import numpy as np
import pytest

import bruteforce as bf
from oracle import oracle as O
from paper_1305_6981_gb300 import synth

REF = 0xFF  # 8e/8o reference: spatial orbitals 0..3 doubly occupied

SPACES = {
    "cisd": dict(max_excitation=2),
    "seniority0": dict(max_seniority=0),
    "seniority2_cisdt": dict(max_seniority=2, max_excitation=3),
    # active space: spatial orbital 0 frozen doubly occupied, spatial orbital 7 deleted
    "cas": dict(frozen_occupied=[0b11], frozen_empty=[0b11 << 14]),
}


def level(d: int, ref: int = REF) -> int:
    return bin(ref & ~d).count("1")


def seniority(d: int, n_orb: int) -> int:
    return sum(((d >> (2 * p)) & 1) != ((d >> (2 * p + 1)) & 1) for p in range(n_orb))


def allowed(d: int, space: dict, n_orb: int = 8) -> bool:
    if "max_excitation" in space and level(d) > space["max_excitation"]:
        return False
    if "max_seniority" in space and seniority(d, n_orb) > space["max_seniority"]:
        return False
    fo = space.get("frozen_occupied", [0])[0]
    fe = space.get("frozen_empty", [0])[0]
    return (d & fo) == fo and (d & fe) == 0


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_8e8o()


@pytest.fixture(scope="module")
def tiny_space(tiny):
    dets = bf.basis(8, 4, 4)
    return dets, bf.hamiltonian(8, tiny.h, tiny.eri_s8, dets)


@pytest.mark.parametrize("name", sorted(SPACES))
def test_membership_matches_definitions(tiny, tiny_space, name):
    dets, _ = tiny_space
    q = O.Oracle(tiny, tau=0.01, **SPACES[name])
    got = np.array([q.in_space(bf.to_words(d, 1)) for d in dets])
    want = np.array([allowed(d, SPACES[name]) for d in dets])
    assert np.array_equal(got, want)
    assert 0 < want.sum() < len(dets)


def test_membership_two_words():
    """24e/60o: random determinants across the word boundary against the same definitions."""
    s = synth.large_24e60o()
    ref = (1 << 24) - 1
    fo, fe = 0b1111, 0b11 << 118
    space = dict(max_excitation=4, max_seniority=6, frozen_occupied=bf.to_words(fo, 2),
                 frozen_empty=bf.to_words(fe, 2))
    q = O.Oracle(s, tau=0.001, **space)
    rng = np.random.default_rng(11)
    n_in = 0
    for _ in range(3000):
        k = int(rng.integers(0, 7))  # electrons moved out of the reference
        holes = rng.choice(24, k, replace=False)
        parts = rng.choice(np.arange(24, 120), k, replace=False)
        d = ref
        for x in holes:
            d ^= 1 << int(x)
        for x in parts:
            d ^= 1 << int(x)
        want = (bin(ref & ~d).count("1") <= 4 and seniority(d, 60) <= 6 and (d & fo) == fo and (d & fe) == 0)
        assert q.in_space(bf.to_words(d, 2)) == want
        n_in += want
    assert n_in > 100


def test_reference_outside_the_space_is_rejected(tiny):
    with pytest.raises(ValueError):
        O.Oracle(tiny, tau=0.01, frozen_empty=[0b1])  # spin orbital 0 is occupied in the reference


@pytest.mark.parametrize("name", ["cisd", "seniority0", "cas"])
def test_one_step_expectation_in_the_space(tiny, tiny_space, name):
    """E[C^(n+1)] over independent random keys equals Eq. 1 with H projected onto the space: no walker
    ever lands outside it, and inside it the expectation is that of the unrestricted dynamics."""
    dets, H = tiny_space
    space = SPACES[name]
    index = {d: i for i, d in enumerate(dets)}
    inside = np.array([allowed(d, space) for d in dets])
    rng = np.random.default_rng(7)
    cand = [d for d in dets if allowed(d, space) and d != REF]
    pick = rng.choice(len(cand), min(24, len(cand)), replace=False)
    chosen = [cand[i] for i in pick] + [REF]
    pops = rng.integers(1, 6, len(chosen)) * rng.choice([-1, 1], len(chosen))
    pops[-1] = 60
    # tau small enough that a spawn rarely carries more than one walker (the variance floor below assumes
    # outcomes of size one; a single excitation of 8e/8o can have tau |H| / P_gen of several at tau 0.05)
    tau, S = 0.02, -0.4
    q = O.Oracle(tiny, tau=tau, initial_shift=S, **space)
    E0 = q.info()["E0"]
    c = np.zeros(len(dets))
    for d, p in zip(chosen, pops):
        c[index[d]] = p
    off = (H - np.diag(np.diag(H))) * inside[:, None]
    expect = c - tau * ((np.diag(H) - E0 - S) * c) - tau * (off @ c)
    K = 6000
    acc = np.zeros(len(dets))
    acc2 = np.zeros(len(dets))
    words = np.array([bf.to_words(d, 1) for d in chosen])
    nulls = 0
    for k in range(K):
        q.set_walkers(words, pops, iteration=k, shift=S)
        nulls += q.iterate(1)[0]["nulls"]
        dd, pp, _ = q.walkers()
        v = np.zeros(len(dets))
        for w, p in zip(dd, pp):
            v[index[int(w[0])]] = p
        acc += v
        acc2 += v * v
    assert np.all(acc[~inside] == 0)
    mean = acc / K
    var = acc2 / K - mean ** 2
    touched = (var > 0) | (expect != 0)
    floor_var = np.abs(expect) * np.clip(1 - np.abs(expect), 0, 1)
    z = np.abs(mean - expect)[touched] / np.sqrt(np.maximum(var, floor_var)[touched] / K)
    assert np.all(np.isfinite(z))
    assert z.max() < 5.0, z.max()
    assert nulls > 0


@pytest.mark.slow
def test_truncated_dynamics_reach_projected_ground_state(tiny, tiny_space):
    """Plain FCIQMC restricted to the seniority-zero space of 8e/8o (closed shells only): the
    time-averaged projected energy agrees with the lowest eigenvalue of H projected onto that space,
    which lies 0.03 Eh above the FCI energy."""
    dets, H = tiny_space
    inside = np.array([allowed(d, SPACES["seniority0"]) for d in dets])
    e_sp = np.linalg.eigvalsh(H[np.ix_(inside, inside)])[0]
    e_fci = np.linalg.eigvalsh(H)[0]
    assert e_sp > e_fci + 0.02
    q = O.Oracle(tiny, tau=0.02, target_walkers=3000, initial_population=1500, initial_shift=0.1, seed=5,
                 max_seniority=0)
    E0 = q.info()["E0"]
    q.iterate(600)
    rows = q.iterate(4096)
    num = np.array([r["num_in"] for r in rows])
    c0 = np.array([r["c0_in"] for r in rows], dtype=float)
    B = 32
    nb = len(num) // B
    bn = num[: nb * B].reshape(B, nb).mean(1)
    bc = c0[: nb * B].reshape(B, nb).mean(1)
    jk = np.array([(bn.sum() - bn[i]) / (bc.sum() - bc[i]) for i in range(B)])
    ep = E0 + bn.sum() / bc.sum()
    eperr = np.sqrt((B - 1) / B * ((jk - jk.mean()) ** 2).sum())
    assert abs(ep - e_sp) < 4 * eperr + 1e-4, (ep, eperr, e_sp, e_fci)
    d, p, _ = q.walkers()
    assert all(allowed(int(w[0]), SPACES["seniority0"]) for w in d)
