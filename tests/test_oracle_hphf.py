"""Pins of the oracle's spin-coupled functions (Sec. VI C; CPU only).

Independent constructions: the spin-flip operator F built on the full M_s = 0 sector of 8e/8o from its
definition (exchange alpha and beta of every electron, then reorder the creation operators) must
commute with the brute-force Hamiltonian and square to one; the spin-coupled functions are the
F = sigma combinations of each determinant pair, U its matrix, and the oracle's matrix elements must
equal U^T H U. The closed-form generation probability of any target is checked against the exact
enumeration of every random path of the generator, and one step of the dynamics against Eq. 1 in the
spin-coupled basis.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import bruteforce as bf
from oracle import oracle as O
from paper_1305_6981_gb300 import synth

REF = 0xFF


def flip(d: int, n_orb: int) -> int:
    out = 0
    for p in range(n_orb):
        a, b = (d >> (2 * p)) & 1, (d >> (2 * p + 1)) & 1
        out |= (b << (2 * p)) | (a << (2 * p + 1))
    return out


def flip_phase(d: int, n_so: int) -> int:
    """Sign of sorting the creation operators of the flipped spin orbitals back into ascending order."""
    ks = [k ^ 1 for k in range(n_so) if (d >> k) & 1]
    inv = sum(1 for x in range(len(ks)) for y in range(x + 1, len(ks)) if ks[x] > ks[y])
    return -1 if inv % 2 else 1


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_8e8o()


@pytest.fixture(scope="module")
def sector(tiny):
    dets = bf.basis(8, 4, 4)
    H = bf.hamiltonian(8, tiny.h, tiny.eri_s8, dets)
    index = {d: i for i, d in enumerate(dets)}
    n = len(dets)
    F = np.zeros((n, n))
    for i, d in enumerate(dets):
        F[index[flip(d, 8)], i] = flip_phase(d, 16)
    sigma = flip_phase(REF, 16)
    reps = sorted({min(d, flip(d, 8)) for d in dets})
    U = np.zeros((n, len(reps)))
    for k, r in enumerate(reps):
        rb = flip(r, 8)
        if rb == r:
            U[index[r], k] = 1.0
        else:
            U[index[r], k] = 1.0 / np.sqrt(2.0)
            U[index[rb], k] = sigma * flip_phase(r, 16) / np.sqrt(2.0)
    return dets, H, F, U, reps, sigma


def test_spin_flip_is_a_symmetry(sector):
    dets, H, F, U, reps, sigma = sector
    assert np.abs(F @ F - np.eye(len(dets))).max() == 0
    assert np.abs(F @ H - H @ F).max() < 1e-12
    # the functions are orthonormal eigenvectors of F with eigenvalue sigma
    assert np.abs(U.T @ U - np.eye(len(reps))).max() < 1e-14
    assert np.abs(F @ U - sigma * U).max() < 1e-14
    # the sector holds the ground state: its lowest eigenvalue is the FCI energy
    e_sector = np.linalg.eigvalsh(U.T @ H @ U)[0]
    assert abs(e_sector - np.linalg.eigvalsh(H)[0]) < 1e-10


def test_matrix_elements_equal_the_projection(tiny, sector):
    dets, H, F, U, reps, sigma = sector
    Hs = U.T @ H @ U
    q = O.Oracle(tiny, tau=0.01, hphf=True)
    rng = np.random.default_rng(2)
    pick = sorted(set(rng.choice(len(reps), 160, replace=False)) | {reps.index(REF)})
    opened = sum(flip(reps[k], 8) != reps[k] for k in pick)
    assert 20 < opened < len(pick)
    for x in pick:
        a = bf.to_words(reps[x], 1)
        assert abs(q.hphf_hdiag(a) - Hs[x, x]) < 1e-12, hex(reps[x])
        for y in pick:
            if y != x:
                assert abs(q.hphf_hij(a, bf.to_words(reps[y], 1)) - Hs[x, y]) < 1e-12, (hex(reps[x]), hex(reps[y]))


def _enumerate(q, d, pd_num, pd_den):
    """Exact probability of every determinant one attempt from d can generate (all random paths)."""
    probs = {}
    for kind, ptype in ((1, Fraction(pd_den - pd_num, pd_den)), (2, Fraction(pd_num, pd_den))):
        _, _, info = q.excite_ranks(d, kind, 0, 0, 0)
        n1 = int(info[1])
        for k1 in range(n1):
            _, _, info = q.excite_ranks(d, kind, k1, 0, 0)
            n2 = int(info[2])
            for k2 in range(n2):
                if kind == 1:
                    paths = [(0, ptype / (n1 * n2))]
                else:
                    _, _, info = q.excite_ranks(d, kind, k1, k2, 0)
                    n3 = int(info[3])
                    paths = [(k3, ptype / (n1 * n2 * n3)) for k3 in range(n3)]
                for k3, pr in paths:
                    r, child, _ = q.excite_ranks(d, kind, k1, k2, k3)
                    c = bf.from_words(child)
                    probs[c] = probs.get(c, Fraction(0)) + pr
    return probs


@pytest.mark.parametrize("which", ["8e8o", "10e12o_sym"])
def test_generation_probability_of_any_target(tiny, which):
    s = tiny if which == "8e8o" else synth.small_system(12, 10, seed=6, symmetry=True)
    q = O.Oracle(s, tau=0.01)
    info = q.info()
    rng = np.random.default_rng(4)
    M, N = s.n_orb, s.n_elec
    sources = [int(info["ref"][0])]
    for _ in range(3):
        occ_a = sorted(rng.choice(M, N // 2, replace=False))
        occ_b = sorted(rng.choice(M, N // 2, replace=False))
        sources.append(sum(1 << (2 * p) for p in occ_a) | sum(1 << (2 * p + 1) for p in occ_b))
    for d in sources:
        probs = _enumerate(q, bf.to_words(d, 1), info["d53"], 2 ** 53)
        for c, p in probs.items():
            g = q.gen_prob(bf.to_words(d, 1), bf.to_words(c, 1))
            assert abs(g - float(p)) <= 4e-16 * float(p), (hex(d), hex(c), g, float(p))
        # targets the generator never produces: beyond doubles, spin- or symmetry-forbidden
        space = bf.basis(M, N // 2, N // 2)
        for c in rng.choice(len(space), 300, replace=False):
            t = space[int(c)]
            if t not in probs and t != d:
                assert q.gen_prob(bf.to_words(d, 1), bf.to_words(t, 1)) == 0.0


def test_one_step_expectation_in_spin_coupled_functions(tiny, sector):
    """E[C^(n+1)] over independent random keys equals Eq. 1 with the Hamiltonian of the spin-coupled
    functions U^T H U; walkers only ever sit on the stored determinant of a pair."""
    dets, H, F, U, reps, sigma = sector
    Hs = U.T @ H @ U
    index = {r: k for k, r in enumerate(reps)}
    rng = np.random.default_rng(8)
    cand = [r for r in reps if r != REF]
    pick = rng.choice(len(cand), 24, replace=False)
    chosen = [cand[i] for i in pick] + [REF]
    pops = rng.integers(1, 6, len(chosen)) * rng.choice([-1, 1], len(chosen))
    pops[-1] = 60
    # tau small enough that a spawn rarely carries more than one walker (the variance floor below assumes
    # outcomes of size one; a single excitation of 8e/8o can have tau |H| / P_gen of several at tau 0.05)
    tau, S = 0.01, -0.4
    q = O.Oracle(tiny, tau=tau, initial_shift=S, hphf=True)
    E0 = q.info()["E0"]
    c = np.zeros(len(reps))
    for r, p in zip(chosen, pops):
        c[index[r]] = p
    expect = c - tau * ((np.diag(Hs) - E0 - S) * c) - tau * ((Hs - np.diag(np.diag(Hs))) @ c)
    K = 12000
    acc = np.zeros(len(reps))
    acc2 = np.zeros(len(reps))
    words = np.array([bf.to_words(r, 1) for r in chosen])
    for k in range(K):
        q.set_walkers(words, pops, iteration=k, shift=S)
        q.iterate(1)
        dd, pp, _ = q.walkers()
        v = np.zeros(len(reps))
        for w, p in zip(dd, pp):
            v[index[int(w[0])]] = p  # KeyError if a walker sat on the larger determinant of a pair
        acc += v
        acc2 += v * v
    mean = acc / K
    var = acc2 / K - mean ** 2
    touched = (var > 0) | (expect != 0)
    floor_var = np.abs(expect) * np.clip(1 - np.abs(expect), 0, 1)
    z = np.abs(mean - expect)[touched] / np.sqrt(np.maximum(var, floor_var)[touched] / K)
    assert np.all(np.isfinite(z))
    assert z.max() < 5.0, z.max()
    assert touched.sum() > 100


def test_projected_energy_numerator(tiny, sector):
    """The Eq. 2 numerator of a state over spin-coupled functions equals sum_B <Phi_ref|H|Phi_B> C_B."""
    dets, H, F, U, reps, sigma = sector
    Hs = U.T @ H @ U
    index = {r: k for k, r in enumerate(reps)}
    rng = np.random.default_rng(12)
    pick = rng.choice(len(reps), 400, replace=False)
    chosen = [reps[i] for i in pick if reps[i] != REF] + [REF]
    pops = rng.integers(1, 9, len(chosen)) * rng.choice([-1, 1], len(chosen))
    q = O.Oracle(tiny, tau=0.01, hphf=True)
    q.set_walkers(np.array([bf.to_words(r, 1) for r in chosen]), pops)
    est = q.estimate()
    want = sum(Hs[index[REF], index[r]] * p for r, p in zip(chosen, pops) if r != REF)
    assert abs(est["num"] - want) < 1e-11 * max(1.0, abs(want))
    assert sum(flip(r, 8) != r and Hs[index[REF], index[r]] != 0 for r in chosen) > 5


def test_stored_form_and_requirements(tiny):
    q = O.Oracle(tiny, tau=0.01, hphf=True)
    d = 0xFF ^ 0b1 ^ (1 << 10)  # spin orbital 0 (alpha) -> 10 (alpha): one open pair
    db = flip(d, 8)
    big = max(d, db)
    with pytest.raises(ValueError):
        q.set_walkers(np.array([[0xFF], [big]], dtype=np.uint64), np.array([5, 1], dtype=np.int32))
    with pytest.raises(ValueError):
        O.Oracle(synth.small_system(8, 6, seed=5), tau=0.01, ms2=2, hphf=True)  # M_s != 0


@pytest.mark.slow
def test_dynamics_reach_fci_energy(tiny, sector):
    """Plain FCIQMC in spin-coupled functions on 8e/8o: the time-averaged projected energy agrees with
    the exact ground-state energy."""
    dets, H, F, U, reps, sigma = sector
    e_fci = np.linalg.eigvalsh(H)[0]
    q = O.Oracle(tiny, tau=0.02, target_walkers=2500, initial_population=1200, initial_shift=0.1, seed=3,
                 hphf=True)
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
    assert abs(ep - e_fci) < 4 * eperr + 1e-4, (ep, eperr, e_fci)
