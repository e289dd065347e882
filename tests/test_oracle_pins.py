"""Pins of the CPU oracle against things other than itself (CPU only).

Each test checks the oracle against a value the paper or the mathematics fixes:
published known answers, an independent second-quantised Hamiltonian, exact
enumeration of the excitation generator's random paths against the paper's
closed-form generation probabilities, the expectation of one step against
Eq. 1, exact diagonalisation, and the paper's worked storage numbers.
"""
from __future__ import annotations

import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import bruteforce as bf
from oracle import oracle as O
from paper_1305_6981_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_8e8o()


@pytest.fixture(scope="module")
def tiny_space(tiny):
    dets = bf.basis(8, 4, 4)
    H = bf.hamiltonian(8, tiny.h, tiny.eri_s8, dets)
    return dets, H


# ---------------------------------------------------------------------------- random numbers
def test_philox_known_answers():
    """Philox4x32-10 reproduces the published Random123 known-answer vectors."""
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            assert O.philox(v[0:4], v[4:6]) == v[6:10]
            n += 1
    assert n == 3


def _split(R: int, top: int = 0) -> tuple[int, int]:
    """Philox words (r0, r1) whose choice word is the 75-bit R; top fills the type bits of r0."""
    return (top << 11) | (R & 0x7FF), R >> 11


def test_choice_digits_are_the_mixed_radix_expansion():
    """The attempt's choices are the digits of the uniform fraction x = R / 2^75 in mixed radix
    (n1, n2, n3): the digits are (k1, k2, k3) exactly when x lies in [c, c + 1/(n1 n2 n3)) with
    c = ((k1 n2 + k2) n3 + k3) / (n1 n2 n3). Checked at the first R of every cell and the R just below
    it, with random type bits, in exact integer arithmetic."""
    rng = np.random.default_rng(21)
    for radices in ([3], [7, 5], [5, 1, 4], [276, 96, 47], [2016, 128, 64], [3, 2, 2, 5]):
        total = math.prod(radices)
        cells = range(total) if total <= 400 else rng.integers(0, total, 300)
        for cell in cells:
            cell = int(cell)
            want, rest = [], cell
            for n in reversed(radices):
                want.append(rest % n)
                rest //= n
            want = want[::-1]
            first = -((-cell << 75) // total)  # ceil(cell 2^75 / total)
            top = int(rng.integers(0, 1 << 53))
            assert O.digits(*_split(first, top), radices) == want, (radices, cell)
            if cell > 0:
                prev = cell - 1
                got = O.digits(*_split(first - 1, top), radices)
                exp, rest = [], prev
                for n in reversed(radices):
                    exp.append(rest % n)
                    rest //= n
                assert got == exp[::-1], (radices, cell)


def test_choice_digits_uniform_and_independent():
    """Over uniform Philox words the joint distribution of three digits is uniform (chi-square over
    105 cells), so successive choices neither repeat nor correlate."""
    rng = np.random.default_rng(5)
    radices = [7, 5, 3]
    counts = np.zeros(105, dtype=np.int64)
    n = 60_000
    words = rng.integers(0, 2**63, size=(n, 2), dtype=np.int64).astype(np.uint64) * np.uint64(2) \
        + rng.integers(0, 2, size=(n, 2), dtype=np.int64).astype(np.uint64)
    for r0, r1 in words:
        k = O.digits(int(r0), int(r1), radices)
        counts[(k[0] * 5 + k[1]) * 3 + k[2]] += 1
    e = n / 105
    chi2 = float(((counts - e) ** 2 / e).sum())
    assert chi2 < 180.0, chi2  # 104 degrees of freedom: p < 1e-5 beyond 180


def test_own_log_accuracy():
    """The shift's logarithm (atanh series) agrees with the correctly rounded ln to 2 ulp."""
    rng = np.random.default_rng(11)
    xs = np.concatenate([np.exp(rng.uniform(-700, 700, 3000)), rng.uniform(0.5, 2.0, 3000),
                         1.0 + rng.normal(0, 1e-6, 500), [1.0, 2.0, 0.5, 1e-310, 1.7976931348623157e308]])
    worst = 0.0
    for x in xs:
        x = float(x)
        ref = math.log(x)
        got = O.log(x)
        if ref == 0.0:
            assert got == 0.0
            continue
        worst = max(worst, abs(got - ref) / math.ulp(ref))
    assert worst <= 2.0, worst
    assert O.log(1.0) == 0.0


# ---------------------------------------------------------------------------- Hamiltonian
def test_hamiltonian_matches_second_quantisation(tiny, tiny_space):
    """All 4900^2 Slater-Condon elements of the 8e/8o space against the brute-force operator form."""
    dets, H = tiny_space
    q = O.Oracle(tiny, tau=0.01)
    Ho = q.hmatrix(np.array([bf.to_words(d, 1) for d in dets]))
    assert np.abs(Ho.T - H).max() < 1e-12


@pytest.mark.parametrize("n_alpha,n_beta", [(2, 2), (3, 1), (3, 2)])
def test_hamiltonian_with_symmetry_and_spin(n_alpha, n_beta):
    """Symmetry-adapted integrals and open-shell (ms2 != 0) spaces."""
    s = synth.small_system(6, n_alpha + n_beta, seed=21, symmetry=True)
    dets = bf.basis(6, n_alpha, n_beta)
    H = bf.hamiltonian(6, s.h, s.eri_s8, dets)
    q = O.Oracle(s, tau=0.01, ms2=n_alpha - n_beta)
    Ho = q.hmatrix(np.array([bf.to_words(d, 1) for d in dets]))
    assert np.abs(Ho.T - H).max() < 1e-12


def _embed(system, n_orb_big, offset):
    """Place `system`'s orbitals at spatial offset..offset+M-1 of a larger, otherwise empty basis."""
    M = system.n_orb
    h = np.zeros((n_orb_big, n_orb_big))
    h[offset:offset + M, offset:offset + M] = system.h
    V = bf.eri_full(M, system.eri_s8)
    big = np.zeros((n_orb_big,) * 4)
    sl = slice(offset, offset + M)
    big[sl, sl, sl, sl] = V
    ps, qs = synth.pack_pairs(n_orb_big)
    vp = big[ps[:, None], qs[:, None], ps[None, :], qs[None, :]]
    eri = vp[np.tril_indices(len(ps))]
    return synth.System(n_orb=n_orb_big, n_elec=system.n_elec, h=h, eri_s8=np.ascontiguousarray(eri), irrep=None)


def test_hamiltonian_two_words(tiny, tiny_space):
    """Two-word determinants: the 8e/8o problem embedded at spin orbitals 56..71, across the word boundary."""
    dets, H = tiny_space
    big = _embed(tiny, 40, 28)
    ref = sum(1 << (56 + k) for k in range(8))
    q = O.Oracle(big, tau=0.01, reference=bf.to_words(ref, 2))
    emb = np.array([bf.to_words(d << 56, 2) for d in dets])
    Ho = q.hmatrix(emb)
    assert np.abs(Ho.T - H).max() < 1e-12


def test_reference_energy_and_pdouble(tiny, tiny_space):
    """E0 = H_00 of the aufbau determinant; P_double from the reference's excitation counts (Sec. VI)."""
    for s in (tiny, synth.init_12e24o()):
        q = O.Oracle(s, tau=0.01)
        info = q.info()
        M, N = s.n_orb, s.n_elec
        ref = sum(1 << k for k in range(N))  # aufbau, interleaved spins
        assert int(info["ref"][0]) == ref
        singles, doubles = bf.allowed_excitations(ref, M, s.irrep)
        assert info["n_single_ref"] == len(singles)
        assert info["n_double_ref"] == len(doubles)
        pd = len(doubles) / (len(singles) + len(doubles))
        assert info["d53"] == math.floor(pd * 2 ** 53)
        assert info["p_double"] == info["d53"] / 2 ** 53
        if s is tiny:
            dets, H = tiny_space
            i = dets.index(ref)
            assert abs(H[i, i] - info["E0"]) < 1e-12
            assert H[i, i] == H.diagonal().min()


# ---------------------------------------------------------------------------- excitation generator
def _enumerate(q, d, pd_num, pd_den):
    """Exact probability of every outcome of the generator from d, by walking all rank paths."""
    probs = {}
    p_null = Fraction(0)
    pgen = {}
    for kind, ptype in ((1, Fraction(pd_den - pd_num, pd_den)), (2, Fraction(pd_num, pd_den))):
        _, _, info = q.excite_ranks(d, kind, 0, 0, 0)
        n1 = int(info[1])
        if n1 == 0:
            p_null += ptype
            continue
        for k1 in range(n1):
            _, _, info = q.excite_ranks(d, kind, k1, 0, 0)
            n2 = int(info[2])
            if n2 == 0:
                p_null += ptype / n1
                continue
            for k2 in range(n2):
                if kind == 1:
                    paths = [(k2, 0, ptype / (n1 * n2))]
                else:
                    _, _, info = q.excite_ranks(d, kind, k1, k2, 0)
                    n3 = int(info[3])
                    if n3 == 0:
                        p_null += ptype / (n1 * n2)
                        continue
                    paths = [(k2, k3, ptype / (n1 * n2 * n3)) for k3 in range(n3)]
                for kk2, kk3, pr in paths:
                    r, child, info = q.excite_ranks(d, kind, k1, kk2, kk3)
                    assert r == kind
                    c = bf.from_words(child)
                    probs[c] = probs.get(c, Fraction(0)) + pr
                    pg = ptype * Fraction(int(info[4]), int(info[5]))
                    if c in pgen:
                        assert pgen[c] == pg
                    pgen[c] = pg
    return probs, pgen, p_null


@pytest.mark.parametrize("which", ["8e8o", "6e8o_sym", "10e12o_sym", "12e24o"])
def test_excitation_generator_is_normalised_and_matches_pgen(which, tiny):
    """Sum over all random paths into each D_j equals the closed-form P_gen (Sec. VI A/B), probabilities
    sum to one with the nulls, and the support is exactly the spin/symmetry-allowed excitations."""
    if which == "8e8o":
        s = tiny
    elif which == "6e8o_sym":
        s = synth.small_system(8, 6, seed=5, symmetry=True)
    elif which == "10e12o_sym":
        s = synth.small_system(12, 10, seed=6, symmetry=True)
    else:
        s = synth.init_12e24o()
    q = O.Oracle(s, tau=0.01)
    info = q.info()
    pd_num, pd_den = info["d53"], 2 ** 53
    rng = np.random.default_rng(3)
    M, N = s.n_orb, s.n_elec
    sources = [int(info["ref"][0])]
    for _ in range(3 if M <= 12 else 1):
        occ_a = sorted(rng.choice(M, N // 2, replace=False))
        occ_b = sorted(rng.choice(M, N // 2, replace=False))
        sources.append(sum(1 << (2 * p) for p in occ_a) | sum(1 << (2 * p + 1) for p in occ_b))
    renormalised = False
    for d in sources:
        probs, pgen, p_null = _enumerate(q, bf.to_words(d, 1), pd_num, pd_den)
        for c, p in probs.items():
            assert p == pgen[c], (hex(d), hex(c))
        assert sum(probs.values()) + p_null == 1
        singles, doubles = bf.allowed_excitations(d, M, s.irrep)
        assert set(probs) == singles | doubles
        _, _, i1 = q.excite_ranks(bf.to_words(d, 1), 1, 0)
        renormalised = renormalised or 0 < i1[1] < N
    if which == "10e12o_sym":
        # some source has electrons without an allowed single (delta_s > 0 in Sec. VI A)
        assert renormalised


def test_excitation_generator_two_words():
    """The same exact enumeration for the 24e/60o reference (two words, 8 irreps)."""
    s = synth.large_24e60o()
    q = O.Oracle(s, tau=0.001)
    info = q.info()
    d = bf.from_words(info["ref"])
    probs, pgen, p_null = _enumerate(q, bf.to_words(d, 2), info["d53"], 2 ** 53)
    for c, p in probs.items():
        assert p == pgen[c]
    assert sum(probs.values()) + p_null == 1
    singles, doubles = bf.allowed_excitations(d, 60, s.irrep)
    assert set(probs) == singles | doubles


# ---------------------------------------------------------------------------- dynamics
def _random_state(rng, dets, n, ref):
    idx = rng.choice(len(dets), n, replace=False)
    chosen = [dets[i] for i in idx if dets[i] != ref][: n - 1] + [ref]
    pops = rng.integers(1, 6, len(chosen)) * rng.choice([-1, 1], len(chosen))
    pops[-1] = 60
    return chosen, pops


@pytest.mark.parametrize("S", [-0.4, 8.0])
def test_one_step_expectation_is_eq1(tiny, tiny_space, S):
    """E[C^(n+1)] over independent random keys equals [1 - tau (H_ii - E0 - S)] C - tau H_offdiag C (Eq. 1).
    With S = -0.4 every determinant of the sample has H_ii - E0 - S > 0 (death only); with S = 8 the reference
    and the sampled determinants with H_ii - E0 < 8 have r < 0 and clone (the second branch of Eq. 4)."""
    dets, H = tiny_space
    index = {d: i for i, d in enumerate(dets)}
    rng = np.random.default_rng(5)
    ref = 0xFF
    chosen, pops = _random_state(rng, dets, 25, ref)
    tau = 0.05
    q = O.Oracle(tiny, tau=tau, initial_shift=S)
    E0 = q.info()["E0"]
    c = np.zeros(len(dets))
    for d, p in zip(chosen, pops):
        c[index[d]] = p
    expect = c - tau * ((np.diag(H) - E0 - S) * c) - tau * ((H - np.diag(np.diag(H))) @ c)
    K = 6000
    acc = np.zeros(len(dets))
    acc2 = np.zeros(len(dets))
    words = np.array([bf.to_words(d, 1) for d in chosen])
    deaths = clones = 0
    for k in range(K):
        q.set_walkers(words, pops, iteration=k, shift=S)
        row = q.iterate(1)[0]
        deaths += row["death_walkers"]
        clones += row["clone_walkers"]
        dd, pp, _ = q.walkers()
        v = np.zeros(len(dets))
        for w, p in zip(dd, pp):
            v[index[int(w[0])]] = p
        acc += v
        acc2 += v * v
    mean = acc / K
    var = acc2 / K - mean ** 2
    touched = (var > 0) | (expect != 0)
    # outcomes are integers, so E[x^2] >= |E[x]|: a component never hit in K samples still has
    # variance of at least about |E[x]| (1 - |E[x]|), which bounds how far 0 may sit from a tiny mean
    floor_var = np.abs(expect) * np.clip(1 - np.abs(expect), 0, 1)
    var_eff = np.maximum(var, floor_var)
    z = np.abs(mean - expect)[touched] / np.sqrt(var_eff[touched] / K)
    assert np.all(np.isfinite(z))
    assert z.max() < 5.0, z.max()
    assert touched.sum() > 100
    assert deaths > 0 and (clones > 0) == (S > 0), (deaths, clones)


@pytest.mark.slow
def test_plain_dynamics_reach_fci_energy(tiny, tiny_space):
    """Plain FCIQMC (no initiator) on 8e/8o: time-averaged shift and projected energies agree with
    the exact ground-state energy of the brute-force Hamiltonian within statistical error."""
    dets, H = tiny_space
    e_fci = np.linalg.eigvalsh(H)[0]
    q = O.Oracle(tiny, tau=0.02, target_walkers=4000, initial_population=2000, initial_shift=0.1, seed=3)
    E0 = q.info()["E0"]
    rows = q.iterate(600)
    assert q.state()["vary"]
    rows = q.iterate(4096)
    shift = np.array([r["shift"] for r in rows]) + E0
    num = np.array([r["num_in"] for r in rows])
    c0 = np.array([r["c0_in"] for r in rows], dtype=float)
    ms, es = bf.blocking(shift)
    # projected energy: ratio of means, error by jackknife over 32 blocks
    B = 32
    nb = len(num) // B
    bn = num[: nb * B].reshape(B, nb).mean(1)
    bc = c0[: nb * B].reshape(B, nb).mean(1)
    ratio = bn.sum() / bc.sum()
    jk = np.array([(bn.sum() - bn[i]) / (bc.sum() - bc[i]) for i in range(B)])
    ep = E0 + ratio
    eperr = np.sqrt((B - 1) / B * ((jk - jk.mean()) ** 2).sum())
    assert abs(ep - e_fci) < 4 * eperr + 1e-4, (ep, eperr, e_fci)
    assert abs(ms - e_fci) < 4 * es + 2e-3, (ms, es, e_fci)
    # once varied, the shift holds the walker number constant (Sec. II)
    nw = np.array([r["nw_out"] for r in rows], dtype=float)
    half = len(nw) // 2
    assert abs(nw[half:].mean() / nw[:half].mean() - 1) < 0.2
    assert 4000 <= nw.mean() < 4 * 4000


def test_shift_holds_the_population():
    """Once the walker number reaches the target the shift is varied (Sec. II) and holds the population
    steady: over the last 300 of 800 iterations of 8e/8o it stays within a factor of two of the target and
    does not drift."""
    q = O.Oracle(synth.tiny_8e8o(), tau=0.02, target_walkers=2000, initial_population=500, initial_shift=0.1,
                 seed=5)
    rows = q.iterate(800)
    assert q.state()["vary"]
    nw = np.array([r["nw_out"] for r in rows[-300:]], dtype=float)
    assert 1000 <= nw.min() and nw.max() <= 4000
    assert abs(nw[150:].mean() / nw[:150].mean() - 1) < 0.2


def test_invariants_with_initiator():
    """12e/24o initiator run: every determinant keeps N, Sz and the reference's irrep; list has no
    duplicates or empty entries; aborted spawns only occur with the initiator approximation on."""
    s = synth.init_12e24o()
    q = O.Oracle(s, tau=0.02, initiator_threshold=3, target_walkers=20000, initial_population=200,
                 initial_shift=0.3, seed=9)
    ref_sym = 0  # closed-shell reference
    ref = bf.from_words(q.info()["ref"])
    _, doubles = bf.allowed_excitations(ref, 24, s.irrep)
    rng = np.random.default_rng(2)
    start = [ref] + [int(x) for x in rng.choice(sorted(doubles), 300, replace=False)]
    pops = [500] + [int(x) for x in rng.choice([-3, -2, -1, 1, 2, 3], 300)]
    q.set_walkers(np.array([bf.to_words(d, 1) for d in start]), pops, shift=0.3)
    aborted = 0
    for _ in range(40):
        row = q.iterate(1)[0]
        aborted += row["aborted_walkers"]
        dets, pops, hd = q.walkers()
        assert np.all(pops != 0)
        ints = [bf.from_words(w) for w in dets]
        assert len(set(ints)) == len(ints)
        for d in ints:
            assert bin(d).count("1") == 12
            assert bin(d & 0x555555555555).count("1") == 6
            g = 0
            for k in range(48):
                if (d >> k) & 1:
                    g ^= int(s.irrep[k >> 1])
            assert g == ref_sym
        assert row["nw_out"] == int(np.abs(pops).sum())
        assert row["nd_out"] == len(pops)
    assert aborted > 0
    # stored diagonal is H_ii - E0 of each determinant
    E0 = q.info()["E0"]
    for w, h in zip(dets[:50], hd[:50]):
        assert h == q.hdiag(w) - E0


def test_initiator_rule_on_one_step(tiny):
    """Sec. V B: a spawn onto a determinant unoccupied after death survives only if some contributing
    parent is an initiator (flags of merged spawns are OR-ed); spawns onto occupied determinants are
    always added. Spawns are enumerated attempt by attempt with the same random keys."""
    q = O.Oracle(tiny, tau=0.05, initiator_threshold=3, seed=4)
    ref = bf.from_words(q.info()["ref"])
    rng = np.random.default_rng(8)
    pool = [int(x) for x in rng.choice([d for d in bf.basis(8, 4, 4) if d != ref], 1500, replace=False)]
    dets = [ref] + pool
    pops = [3000] + [int(x) for x in rng.choice([-3, -2, -1, 1, 2, 3], len(pool))]
    words = np.array([bf.to_words(d, 1) for d in dets])
    mixed_seen = 0
    for it in range(6):
        q.set_walkers(words, pops, iteration=it)
        from_init, from_non = {}, {}
        for d, c in zip(dets, pops):
            init = d == ref or abs(c) > 3
            for a in range(abs(c)):
                amt, child, _ = q.attempt(bf.to_words(d, 1), c, a)
                if amt:
                    tgt = from_init if init else from_non
                    k = bf.from_words(child)
                    tgt[k] = tgt.get(k, 0) + amt
        row = q.iterate(1)[0]
        nd, npop, _ = q.walkers()
        after = {bf.from_words(w): int(p) for w, p in zip(nd, npop)}
        old = set(dets)
        for d in after:
            if d not in old:
                assert d in from_init, hex(d)
        for k, v in from_init.items():
            net = v + from_non.get(k, 0)
            if k not in old:
                assert after.get(k, 0) == net
                mixed_seen += k in from_non and net != 0
        assert row["merged_entries"] == len(set(from_init) | set(from_non))
        # aborted: non-initiator spawns onto determinants unoccupied after death; old determinants
        # may have died in this iteration's death step, so they can add to the count
        aborted = sum(abs(v) for k, v in from_non.items() if k not in old and k not in from_init)
        onto_old = sum(abs(v) for k, v in from_non.items() if k in old)
        assert aborted <= row["aborted_walkers"] <= aborted + onto_old
    assert mixed_seen > 0


def test_fingerprint_is_spread():
    """Algorithm 1 over the 4900 determinants of 8e/8o: no collisions and uniform low bits."""
    q = O.Oracle(synth.tiny_8e8o(), tau=0.01)
    fps = [q.fingerprint(bf.to_words(d, 1)) for d in bf.basis(8, 4, 4)]
    assert len(set(fps)) == len(fps)
    counts = np.bincount(np.array(fps, dtype=np.uint64) & np.uint64(63), minlength=64)
    chi2 = ((counts - len(fps) / 64) ** 2 / (len(fps) / 64)).sum()
    assert chi2 < 130  # 63 degrees of freedom, p ~ 1e-6


def _fingerprint_golden():
    maps, cases = {}, []
    with open(os.path.join(GOLDEN, "fingerprint_alg1.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = line.split()
            if v[0] == "map":
                maps[int(v[1])] = int(v[2], 16)
            else:
                cases.append(([int(x) for x in v[1].split(",")], [int(x, 16) for x in v[2:]]))
    return maps, cases


@pytest.mark.parametrize("n_orb", [16, 64])
def test_fingerprint_is_algorithm1(n_orb):
    """Algorithm 1 (Sec. V) against values worked step by step from its recurrence (tests/golden): the orbital
    map is the keyed Philox of the random-number contract, a one-electron determinant hashes to its map value,
    and every prefix of the occupied list (ascending, electrons counted from 1) gives the listed hash."""
    maps, cases = _fingerprint_golden()
    q = O.Oracle(synth.make_system(n_orb, 4, seed=0, n_chol=1), tau=0.01)
    m = q.map1()
    for k, v in maps.items():
        if k < 2 * n_orb:
            assert int(m[k]) == v, k
    W = 1 if n_orb <= 32 else 2
    checked = 0
    for orbs, steps in cases:
        if max(orbs) >= 2 * n_orb:
            continue
        for n in range(1, len(orbs) + 1):
            d = sum(1 << k for k in orbs[:n])
            assert q.fingerprint(bf.to_words(d, W)) == steps[n - 1], (orbs[:n], hex(steps[n - 1]))
            checked += 1
        assert steps[0] == maps[orbs[0]]
    assert checked == (10 if n_orb == 16 else 18)


def test_paper_storage_numbers():
    """Sec. III and Sec. VII worked numbers: words per determinant and memory estimates."""
    g = {}
    with open(os.path.join(GOLDEN, "paper_storage.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            g[k] = int(v)
    so = g["spin_orbitals"]
    M = so // 2
    q = O.Oracle(synth.make_system(M, 4, seed=0, n_chol=1), tau=0.01)
    assert q.W + 1 == g["words_per_det"]
    assert g["memory_bytes"] // (8 * g["words_per_det"]) > g["min_dets"]
    n = math.comb(g["cr2_n_orb"], g["cr2_n_elec"] // 2) ** 2
    assert abs(n * 8 / 1e12 / g["cr2_fci_terabytes"] - 1) < 0.01
    assert abs(g["cr2_walkers"] * 16 / 1e9 / g["cr2_gigabytes"] - 1) < 0.1
