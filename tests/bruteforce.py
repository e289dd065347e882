"""Independent brute-force references used to pin the oracle.

Nothing here uses the Slater-Condon rules: the Hamiltonian is assembled from
its second-quantised form

    H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps),
    E_pq = sum_sigma a+_{p sigma} a_{q sigma},

by applying creation/annihilation operators to occupation-number bit strings
with the Jordan-Wigner sign (-1)^(number of occupied spin orbitals below the
one acted on). Spin orbital k holds spatial orbital k >> 1 with spin k & 1.
"""
from __future__ import annotations

import itertools

import numpy as np


def eri_full(n_orb: int, eri_s8: np.ndarray) -> np.ndarray:
    """Unpack an 8-fold packed ERI vector into the full (pq|rs) tensor."""
    npair = n_orb * (n_orb + 1) // 2
    v = np.zeros((npair, npair))
    iu = np.tril_indices(npair)
    v[iu] = eri_s8
    v = v + v.T - np.diag(np.diag(v))
    pair = np.zeros((n_orb, n_orb), dtype=np.int64)
    for p in range(n_orb):
        for q in range(p + 1):
            pair[p, q] = pair[q, p] = p * (p + 1) // 2 + q
    return v[pair[:, :, None, None], pair[None, None, :, :]]


def basis(n_orb: int, n_alpha: int, n_beta: int) -> list[int]:
    """All determinants (Python ints) with n_alpha / n_beta electrons, in ascending order."""
    dets = []
    for a in itertools.combinations(range(n_orb), n_alpha):
        for b in itertools.combinations(range(n_orb), n_beta):
            d = 0
            for p in a:
                d |= 1 << (2 * p)
            for p in b:
                d |= 1 << (2 * p + 1)
            dets.append(d)
    return sorted(dets)


def _popcount_below(d: int, k: int) -> int:
    return bin(d & ((1 << k) - 1)).count("1")


def hop(d: int, create: int, annihilate: int):
    """a+_create a_annihilate |d>: returns (new det, sign) or None."""
    if not (d >> annihilate) & 1:
        return None
    s = _popcount_below(d, annihilate)
    d1 = d ^ (1 << annihilate)
    if (d1 >> create) & 1:
        return None
    s += _popcount_below(d1, create)
    return d1 | (1 << create), (-1) ** s


def hamiltonian(n_orb: int, h: np.ndarray, eri_s8: np.ndarray, dets: list[int]) -> np.ndarray:
    """Dense H[x, y] = <dets[x]|H|dets[y]> (no core energy).

    `dets` must be a complete (N, S_z) sector, such as basis() returns: the
    product E_pq E_rs passes through intermediate determinants of the sector."""
    n = len(dets)
    index = {d: i for i, d in enumerate(dets)}
    V = eri_full(n_orb, eri_s8)
    # E^sigma_pq as maps y -> x with signs
    maps, sgns = {}, {}
    for p in range(n_orb):
        for q in range(n_orb):
            for sig in (0, 1):
                m = np.full(n, -1, dtype=np.int64)
                s = np.zeros(n)
                for y, d in enumerate(dets):
                    r = hop(d, 2 * p + sig, 2 * q + sig)
                    if r is not None and r[0] in index:
                        m[y] = index[r[0]]
                        s[y] = r[1]
                maps[p, q, sig], sgns[p, q, sig] = m, s
    rows, cols, vals = [], [], []
    ys = np.arange(n)

    def add(m, s, coef):
        ok = m >= 0
        rows.append(m[ok])
        cols.append(ys[ok])
        vals.append(coef * s[ok])

    for p in range(n_orb):
        for q in range(n_orb):
            c1 = h[p, q] - 0.5 * sum(V[p, r, r, q] for r in range(n_orb))
            if c1 != 0.0:
                for sig in (0, 1):
                    add(maps[p, q, sig], sgns[p, q, sig], c1)
    for p, q, r, s in itertools.product(range(n_orb), repeat=4):
        c2 = 0.5 * V[p, q, r, s]
        if c2 == 0.0:
            continue
        for sig in (0, 1):
            for tau in (0, 1):
                m_rs, s_rs = maps[r, s, tau], sgns[r, s, tau]
                m_pq, s_pq = maps[p, q, sig], sgns[p, q, sig]
                ok = m_rs >= 0
                mid = np.where(ok, m_rs, 0)
                m = np.where(ok, m_pq[mid], -1)
                sg = np.where(ok, s_rs * s_pq[mid], 0.0)
                add(m, sg, c2)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    H = np.bincount(rows * n + cols, weights=vals, minlength=n * n).reshape(n, n)
    return H


def to_words(d: int, W: int) -> np.ndarray:
    d = int(d)
    return np.array([(d >> (64 * w)) & 0xFFFFFFFFFFFFFFFF for w in range(W)], dtype=np.uint64)


def from_words(words) -> int:
    return sum(int(w) << (64 * i) for i, w in enumerate(words))


def allowed_excitations(d: int, n_orb: int, irrep) -> tuple[set[int], set[int]]:
    """All spin- and symmetry-allowed single and double excitations of d, by enumeration."""
    n_so = 2 * n_orb
    g = (lambda k: 0) if irrep is None else (lambda k: int(irrep[k >> 1]))
    occ = [k for k in range(n_so) if (d >> k) & 1]
    vir = [k for k in range(n_so) if not (d >> k) & 1]
    singles, doubles = set(), set()
    for i in occ:
        for a in vir:
            if (i & 1) == (a & 1) and g(i) == g(a):
                singles.add(d ^ (1 << i) ^ (1 << a))
    for i, j in itertools.combinations(occ, 2):
        for a, b in itertools.combinations(vir, 2):
            if (i & 1) + (j & 1) != (a & 1) + (b & 1):
                continue
            if g(i) ^ g(j) != g(a) ^ g(b):
                continue
            doubles.add(d ^ (1 << i) ^ (1 << j) ^ (1 << a) ^ (1 << b))
    return singles, doubles


def blocking(x: np.ndarray) -> tuple[float, float]:
    """Mean and standard error by Flyvbjerg-Petersen blocking (plateau = max over levels)."""
    x = np.asarray(x, dtype=np.float64)
    mean = x.mean()
    errs = []
    while len(x) >= 32:
        errs.append(np.sqrt(x.var(ddof=1) / len(x)))
        n = len(x) // 2
        x = 0.5 * (x[0:2 * n:2] + x[1:2 * n:2])
    return mean, max(errs) if errs else float("nan")
