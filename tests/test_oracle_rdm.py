"""Pins of the oracle's energy functional E(h, V; c) = c^T H c / c^T c and its gradient (CPU only).

The oracle computes E from its Slater-Condon elements and the gradient from density matrices built
by applying a+ a and a+ a+ a a to each pair of determinants. Here both are checked against an
independent construction: the spin-summed excitation operators E_pq of the full 8e/8o sector
(tests/bruteforce.py), with gamma_PQ = c^T E_PQ c and Gamma_PQRS = c^T (E_PQ E_RS - delta_QR E_PS) c,
against exact diagonalisation, and against finite differences (E is linear in h and V, so central
differences are exact up to rounding).
"""
from __future__ import annotations

import numpy as np
import pytest

import bruteforce as bf
from oracle import oracle as O
from paper_1305_6981_gb300 import synth


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_8e8o()


@pytest.fixture(scope="module")
def ops(tiny):
    """Maps of E^sigma_PQ over the full 8e/8o sector, and H."""
    dets = bf.basis(8, 4, 4)
    index = {d: i for i, d in enumerate(dets)}
    n, M = len(dets), 8
    maps = {}
    for p in range(M):
        for q in range(M):
            for sig in (0, 1):
                m = np.full(n, -1, dtype=np.int64)
                s = np.zeros(n)
                for y, d in enumerate(dets):
                    r = bf.hop(d, 2 * p + sig, 2 * q + sig)
                    if r is not None:
                        m[y] = index[r[0]]
                        s[y] = r[1]
                maps[p, q, sig] = (m, s)
    H = bf.hamiltonian(8, tiny.h, tiny.eri_s8, dets)
    return dets, maps, H


def _apply(maps, P, Q, v):
    """(E_PQ v) with E_PQ = sum_sigma a+_{P sigma} a_{Q sigma}."""
    out = np.zeros_like(v)
    for sig in (0, 1):
        m, s = maps[P, Q, sig]
        ok = m >= 0
        np.add.at(out, m[ok], s[ok] * v[ok])
    return out


def brute_rdm(maps, c, M=8):
    norm = c @ c
    g1 = np.zeros((M, M))
    Ev = {}
    for R in range(M):
        for S in range(M):
            Ev[R, S] = _apply(maps, R, S, c)
    for P in range(M):
        for Q in range(M):
            g1[P, Q] = c @ Ev[P, Q]
    npair = M * (M + 1) // 2
    ge = np.zeros(npair * (npair + 1) // 2)

    def pidx(a, b):
        return max(a, b) * (max(a, b) + 1) // 2 + min(a, b)

    for P in range(M):
        for Q in range(M):
            EPQt_c = _apply(maps, Q, P, c)  # E_PQ^T c = E_QP c
            for R in range(M):
                for S in range(M):
                    g2 = EPQt_c @ Ev[R, S] - (c @ Ev[P, S] if Q == R else 0.0)
                    a, b = pidx(P, Q), pidx(R, S)
                    ge[pidx(a, b)] += 0.5 * g2
    return g1 / norm, ge / norm


def test_energy_functional_at_the_ground_state(tiny, ops):
    """FCI vector of 8e/8o: E equals the lowest eigenvalue, E = sum h grad_h + sum V grad_eri, and the
    gradients equal the brute-force density matrices."""
    dets, maps, H = ops
    w, v = np.linalg.eigh(H)
    c = v[:, 0]
    q = O.Oracle(tiny, tau=0.01)
    E, gh, ge = q.rdm_energy(np.array([bf.to_words(d, 1) for d in dets]), c)
    assert abs(E - w[0]) < 1e-10
    assert abs(E - (np.sum(tiny.h * gh) + np.sum(tiny.eri_s8 * ge))) < 1e-10
    g1, g2 = brute_rdm(maps, c)
    assert np.abs(gh - g1).max() < 1e-12
    assert np.abs(ge - g2).max() < 1e-12
    assert abs(np.trace(gh) - 8.0) < 1e-12  # particle number


def test_energy_functional_on_a_subset(tiny, ops):
    """A random subset of the sector with random amplitudes (zero elsewhere)."""
    dets, maps, H = ops
    rng = np.random.default_rng(17)
    sel = np.sort(rng.choice(len(dets), 700, replace=False))
    c_sub = rng.normal(size=len(sel))
    c_full = np.zeros(len(dets))
    c_full[sel] = c_sub
    q = O.Oracle(tiny, tau=0.01)
    E, gh, ge = q.rdm_energy(np.array([bf.to_words(dets[i], 1) for i in sel]), c_sub)
    assert abs(E - c_full @ H @ c_full / (c_full @ c_full)) < 1e-11
    g1, g2 = brute_rdm(maps, c_full)
    assert np.abs(gh - g1).max() < 1e-12
    assert np.abs(ge - g2).max() < 1e-12


def _embed(system, n_orb_big, offset):
    M = system.n_orb
    h = np.zeros((n_orb_big, n_orb_big))
    h[offset:offset + M, offset:offset + M] = system.h
    V = bf.eri_full(M, system.eri_s8)
    big = np.zeros((n_orb_big,) * 4)
    sl = slice(offset, offset + M)
    big[sl, sl, sl, sl] = V
    ps, qs = synth.pack_pairs(n_orb_big)
    vp = big[ps[:, None], qs[:, None], ps[None, :], qs[None, :]]
    return synth.System(n_orb=n_orb_big, n_elec=system.n_elec, h=h,
                        eri_s8=np.ascontiguousarray(vp[np.tril_indices(len(ps))]), irrep=None)


def test_energy_functional_two_words(tiny, ops):
    """Two-word determinants: 8e/8o embedded at spin orbitals 56..71 of a 40-orbital basis."""
    dets, maps, H = ops
    rng = np.random.default_rng(4)
    sel = np.sort(rng.choice(len(dets), 300, replace=False))
    c = rng.normal(size=len(sel))
    q8 = O.Oracle(tiny, tau=0.01)
    E8, gh8, ge8 = q8.rdm_energy(np.array([bf.to_words(dets[i], 1) for i in sel]), c)
    big = _embed(tiny, 40, 28)
    q40 = O.Oracle(big, tau=0.01, reference=bf.to_words(sum(1 << (56 + k) for k in range(8)), 2))
    E40, gh40, ge40 = q40.rdm_energy(np.array([bf.to_words(dets[i] << 56, 2) for i in sel]), c)
    assert abs(E40 - E8) < 1e-12
    assert np.abs(gh40[28:36, 28:36] - gh8).max() < 1e-13
    V40 = bf.eri_full(40, ge40)
    V8 = bf.eri_full(8, ge8)
    assert np.abs(V40[28:36, 28:36, 28:36, 28:36] - V8).max() < 1e-13


def test_energy_functional_finite_differences():
    """16e/40o (two words, no symmetry): central differences of E against the gradient."""
    s = synth.rdm_16e40o()
    dets, c = synth.sampled_vector(s, 250, seed=5)
    q = O.Oracle(s, tau=0.01)
    E, gh, ge = q.rdm_energy(dets, c)
    eps = 1e-6
    rng = np.random.default_rng(2)
    for p, r in [(0, 0), (3, 3), (0, 1), (2, 17), (7, 30)]:
        d = np.zeros_like(s.h)
        d[p, r] += eps
        if p != r:
            d[r, p] += eps
        qp = O.Oracle(synth.System(s.n_orb, s.n_elec, s.h + d, s.eri_s8, None), tau=0.01)
        qm = O.Oracle(synth.System(s.n_orb, s.n_elec, s.h - d, s.eri_s8, None), tau=0.01)
        fd = (qp.rdm_energy(dets, c)[0] - qm.rdm_energy(dets, c)[0]) / (2 * eps)
        an = gh[p, r] + (gh[r, p] if p != r else 0.0)
        assert abs(fd - an) < 1e-8, (p, r, fd, an)
    for k in rng.choice(len(s.eri_s8), 6, replace=False):
        v = s.eri_s8.copy()
        v[k] += eps
        ep = O.Oracle(synth.System(s.n_orb, s.n_elec, s.h, v, None), tau=0.01).rdm_energy(dets, c)[0]
        v[k] -= 2 * eps
        em = O.Oracle(synth.System(s.n_orb, s.n_elec, s.h, v, None), tau=0.01).rdm_energy(dets, c)[0]
        assert abs((ep - em) / (2 * eps) - ge[k]) < 1e-8, k
