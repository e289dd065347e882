"""Seeded synthetic inputs for the FCIQMC walker cycle.

This module only draws inputs: one- and two-electron integral tables, orbital
symmetry labels and the multi-system batches built from them. It holds none of
the method's arithmetic (no matrix elements, excitations or walker dynamics),
so both the CUDA path and the CPU oracle may take their inputs from it.

The paper's own molecules (Be2 cc-pVQZ, Cr2 SV basis; Sec. VI-VII) need
quantum-chemistry integral files that are not available, so the integrals are
synthetic real tables with the shapes, permutational symmetry (8-fold, Sec. II
footnote on double-triangular packing) and abelian point-group structure
(Sec. II, XOR product of D2h-like irreps) of those workloads:

* orbital energies e_p (optionally with a near-degenerate frontier window),
  read as the diagonal Fock energies of the aufbau reference (n_elec/2 lowest
  spatial orbitals doubly occupied), which is what "orbital energy" means in
  the Hartree-Fock picture the paper's reference determinant comes from:
  h_pp = e_p - sum_{j occ} [2 (pp|jj) - (pj|jp)], so f_pp = e_p,
* h_pq = (the diagonal above) + sym(N(0, sigma_h) exp(-|p-q|/2)),
* (pq|rs) = sum_k L^k_pq L^k_rs with L^k symmetric, which makes the ERI
  tensor 8-fold symmetric and positive semidefinite.

With symmetry labels Gamma_p, h_pq is zero unless Gamma_p == Gamma_q and
Cholesky vector k carries irrep k mod 8 (L^k_pq = 0 unless
Gamma_p ^ Gamma_q == k mod 8), so (pq|rs) vanishes unless
Gamma_p ^ Gamma_q == Gamma_r ^ Gamma_s.
"""
from __future__ import annotations

import dataclasses
import hashlib

import numpy as np


@dataclasses.dataclass
class System:
    """A synthetic Hamiltonian in the layout the C ABI takes."""
    n_orb: int
    n_elec: int
    h: np.ndarray            # (n_orb, n_orb) float64, symmetric, row-major
    eri_s8: np.ndarray       # packed (pq|rs), length npair*(npair+1)/2
    irrep: np.ndarray | None  # (n_orb,) int32 labels 0..7, or None (no symmetry)
    e_core: float = 0.0
    name: str = ""

    @property
    def npair(self) -> int:
        return self.n_orb * (self.n_orb + 1) // 2

    def digest(self) -> str:
        m = hashlib.sha256()
        m.update(self.h.tobytes())
        m.update(self.eri_s8.tobytes())
        if self.irrep is not None:
            m.update(self.irrep.tobytes())
        return m.hexdigest()[:16]


def pack_pairs(n_orb: int) -> tuple[np.ndarray, np.ndarray]:
    """Lists (p, q) with p >= q in packed order pq = p(p+1)/2 + q."""
    ps, qs = [], []
    for p in range(n_orb):
        for q in range(p + 1):
            ps.append(p)
            qs.append(q)
    return np.array(ps), np.array(qs)


def _sym(x: np.ndarray) -> np.ndarray:
    return 0.5 * (x + x.T)


def make_system(n_orb: int, n_elec: int, *, seed: int, n_chol: int,
                symmetry: bool = False, sigma_h: float = 0.1,
                chol_amp: float = 0.3, chol_decay_len: float = 1.0,
                chol_k_decay: float | None = None,
                energies: np.ndarray | None = None, fock_diagonal: bool = True,
                name: str = "") -> System:
    """Draw h and packed ERIs from Generator(PCG64(seed)).

    chol_decay_len: L^k_pq ~ N(0, chol_amp) exp(-|p-q| / chol_decay_len).
    chol_k_decay:   optional extra factor exp(-k / chol_k_decay) per vector.
    energies:       orbital energies e_p (default -2 + 0.5 p).
    fock_diagonal:  shift h_pp so that the aufbau reference's diagonal Fock energies are e_p.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    p = np.arange(n_orb)
    dist = np.abs(p[:, None] - p[None, :])
    e = (-2.0 + 0.5 * p) if energies is None else np.asarray(energies, dtype=np.float64)
    irrep = (p % 8).astype(np.int32) if symmetry else None

    noise = _sym(rng.normal(0.0, sigma_h, size=(n_orb, n_orb)) * np.exp(-dist / 2.0))
    h = np.diag(e) + noise
    if irrep is not None:
        h = h * (irrep[:, None] == irrep[None, :])
    h = _sym(h)  # exact symmetry

    ps, qs = pack_pairs(n_orb)
    lp = np.zeros((n_chol, len(ps)))
    for k in range(n_chol):
        x = _sym(rng.normal(0.0, chol_amp, size=(n_orb, n_orb))) * np.exp(-dist / chol_decay_len)
        if chol_k_decay is not None:
            x = x * np.exp(-k / chol_k_decay)
        if irrep is not None:
            x = x * ((irrep[:, None] ^ irrep[None, :]) == (k % 8))
        lp[k] = x[ps, qs]
    v = lp.T @ lp                      # (npair, npair), symmetric PSD
    iu = np.tril_indices(len(ps))      # row >= col: packed index pq(pq+1)/2 + rs
    eri = np.ascontiguousarray(v[iu])
    if fock_diagonal:
        def pidx(a, b):
            return max(a, b) * (max(a, b) + 1) // 2 + min(a, b)
        n_occ = n_elec // 2
        for q in range(n_orb):
            mf = 0.0
            for j in range(n_occ):
                mf += 2.0 * v[pidx(q, q), pidx(j, j)] - v[pidx(q, j), pidx(q, j)]
            h[q, q] -= mf
    return System(n_orb=n_orb, n_elec=n_elec, h=np.ascontiguousarray(h), eri_s8=eri,
                  irrep=irrep, name=name)


def frontier_energies(n_orb: int, lo: int = 8, hi: int = 15, gap: float = 0.05) -> np.ndarray:
    """Orbital energies -2 + 0.5 p with a near-degenerate window [lo, hi] of spacing `gap`."""
    e = np.empty(n_orb)
    for p in range(n_orb):
        if p < lo:
            e[p] = -2.0 + 0.5 * p
        elif p <= hi:
            e[p] = (-2.0 + 0.5 * lo) + gap * (p - lo)
        else:
            e[p] = (-2.0 + 0.5 * lo) + gap * (hi - lo) + 0.5 * (p - hi)
    return e


# Workloads with the shapes of the five benchmark configurations.

def tiny_8e8o() -> System:
    """8 electrons in 8 spatial orbitals, no symmetry, 16 Cholesky vectors (Hilbert dim 4900)."""
    return make_system(8, 8, seed=0, n_chol=16, name="8e8o")


def init_12e24o() -> System:
    """12 electrons in 24 spatial orbitals, 8 irreps round-robin, 32 Cholesky vectors."""
    return make_system(24, 12, seed=1, n_chol=32, symmetry=True, name="12e24o")


def large_24e60o() -> System:
    """24 electrons in 60 spatial orbitals (two uint64 words), 8 irreps, decaying Cholesky
    vectors and a near-degenerate frontier window around the Fermi level (HOMO = spatial 11)."""
    return make_system(60, 24, seed=2, n_chol=120, symmetry=True, chol_decay_len=4.0,
                       chol_k_decay=24.0, energies=frontier_energies(60), name="24e60o")


def rdm_16e40o() -> System:
    """16 electrons in 40 spatial orbitals, no symmetry, 32 Cholesky vectors."""
    return make_system(40, 16, seed=4, n_chol=32, name="16e40o")


def small_system(n_orb: int, n_elec: int, seed: int, symmetry: bool = False, n_chol: int = 8) -> System:
    """Small random systems for exhaustive checks."""
    return make_system(n_orb, n_elec, seed=seed, n_chol=n_chol, symmetry=symmetry,
                       name=f"{n_elec}e{n_orb}o-s{seed}")


def batch_systems(n_runs: int = 64, seed: int = 3) -> list[dict]:
    """Uneven independent runs: n_elec even in [8, 16], n_orb in [max(16, n_elec), 40],
    no symmetry, target walkers log-uniform in [1e4, 2e6], Philox seed 1000 + r."""
    rng = np.random.Generator(np.random.PCG64(seed))
    runs = []
    for r in range(n_runs):
        n_elec = int(rng.integers(4, 9)) * 2
        n_orb = int(rng.integers(max(16, n_elec), 41))
        target = int(round(10 ** rng.uniform(4.0, np.log10(2e6))))
        runs.append(dict(n_elec=n_elec, n_orb=n_orb, target=target, seed=1000 + r,
                         sys_seed=int(rng.integers(0, 2**31))))
    return runs


def walker_snapshot(system: System, n_walkers: int, seed: int = 0, ref_fraction: float = 0.05,
                    max_level: int = 4) -> tuple[np.ndarray, np.ndarray]:
    """A synthetic walker list with the structure of an FCIQMC snapshot of a closed-shell system: the
    aufbau reference holds `ref_fraction` of the walkers; the others sit on distinct determinants
    reached from it by 1..max_level random same-spin substitutions (level L drawn with weight 2^-L)
    that keep the reference's spatial symmetry, with random signs and geometric magnitudes (mean 3).
    A space too small to hold n_walkers that way yields fewer. Returns (dets (n, W) uint64, pops (n,) int32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    M, N = system.n_orb, system.n_elec
    nh = N // 2
    W = (2 * M + 63) // 64
    irr = np.asarray(system.irrep if system.irrep is not None else np.zeros(M), dtype=np.int64)
    levels = np.arange(1, max_level + 1)
    wl = 0.5 ** levels
    wl = wl / wl.sum()
    n_ref = max(1, int(ref_fraction * n_walkers))
    ref_bits = np.zeros(64 * W, dtype=bool)
    ref_bits[:N] = True
    seen = {np.packbits(ref_bits, bitorder="little").tobytes()}
    rows, pops = [ref_bits], [n_ref]
    total = n_ref
    B = 4096
    while total < n_walkers:
        occ = [np.tile(np.arange(nh), (B, 1)) for _ in range(2)]
        vir = [np.tile(np.arange(nh, M), (B, 1)) for _ in range(2)]
        g = np.zeros(B, dtype=np.int64)
        L = rng.choice(levels, size=B, p=wl)
        r = np.arange(B)
        for step in range(max_level):
            act = L > step
            spin = rng.integers(0, 2, size=B)
            pi = rng.integers(0, nh, size=B)
            pa = rng.integers(0, M - nh, size=B)
            for sp in (0, 1):
                sel = r[act & (spin == sp)]
                i = occ[sp][sel, pi[sel]]
                a = vir[sp][sel, pa[sel]]
                occ[sp][sel, pi[sel]] = a
                vir[sp][sel, pa[sel]] = i
                g[sel] ^= irr[i] ^ irr[a]
        keep = r[g == 0]
        bits = np.zeros((len(keep), 64 * W), dtype=bool)
        kk = np.repeat(np.arange(len(keep)), nh)
        bits[kk, 2 * occ[0][keep].reshape(-1)] = True
        bits[kk, 2 * occ[1][keep].reshape(-1) + 1] = True
        packed = np.packbits(bits, axis=1, bitorder="little")
        mags = rng.geometric(1.0 / 3.0, size=len(keep))
        sgns = np.where(rng.random(len(keep)) < 0.5, 1, -1)
        added = 0
        for k in range(len(keep)):
            key = packed[k].tobytes()
            if key in seen:
                continue
            seen.add(key)
            rows.append(bits[k])
            pops.append(int(mags[k] * sgns[k]))
            total += int(mags[k])
            added += 1
            if total >= n_walkers:
                break
        if added == 0 and B >= 1 << 16:
            break  # a small space is exhausted: fewer walkers than asked for
        B = min(1 << 20, 2 * B)
    bits = np.array(rows)
    dets = np.packbits(bits, axis=1, bitorder="little").view("<u8").astype(np.uint64)
    return dets.reshape(len(rows), W), np.array(pops, dtype=np.int32)


def stored_pairs(dets: np.ndarray, pops: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """A snapshot on spin-coupled functions: each determinant of (dets, pops) is replaced by the smaller (last
    word most significant) of itself and its spin flip (bits 2p and 2p + 1 exchanged), populations of a pair
    are added, and entries that cancel are dropped. The determinants must have M_s = 0."""
    dets = np.ascontiguousarray(dets, dtype=np.uint64).reshape(len(pops), -1)
    even = np.uint64(0x5555555555555555)
    flip = ((dets & even) << np.uint64(1)) | ((dets >> np.uint64(1)) & even)
    merged: dict = {}
    for k, fk, c in zip(map(tuple, dets[:, ::-1].tolist()), map(tuple, flip[:, ::-1].tolist()), pops.tolist()):
        m = min(k, fk)
        merged[m] = merged.get(m, 0) + int(c)
    items = [(k, c) for k, c in merged.items() if c != 0]
    out = np.array([k[::-1] for k, _ in items], dtype=np.uint64).reshape(-1, dets.shape[1])
    return out, np.array([c for _, c in items], dtype=np.int32)


def sampled_vector(system: System, n_dets: int, seed: int = 5, max_level: int = 6) -> tuple[np.ndarray, np.ndarray]:
    """A fixed amplitude vector with the structure of a time-averaged FCIQMC wavefunction: the aufbau
    reference (amplitude 1) plus distinct S_z-conserving excitations of it whose level L (electrons
    moved) is uniform on 1..max_level, amplitude exp(-L) with a random sign. Returns
    (dets (n, W) uint64, c (n,) float64), the reference first."""
    rng = np.random.Generator(np.random.PCG64(seed))
    M, N = system.n_orb, system.n_elec
    na, nb = (N + 1) // 2, N // 2
    W = (2 * M + 63) // 64
    nv = (M - na, M - nb)
    ref = np.zeros(64 * W, dtype=bool)
    ref[:N] = True
    seen = {np.packbits(ref, bitorder="little").tobytes()}
    rows, amps = [ref], [1.0]
    while len(rows) < n_dets:
        B = min(1 << 18, 2 * (n_dets - len(rows)) + 1024)
        L = rng.integers(1, max_level + 1, size=B)
        lo = np.maximum(0, L - min(nb, nv[1]))
        hi = np.minimum(L, min(na, nv[0]))
        ok = lo <= hi
        La = lo + (rng.random(B) * (hi - lo + 1)).astype(np.int64)
        La = np.minimum(La, hi)
        Lb = L - La
        bits = np.zeros((B, 64 * W), dtype=bool)
        for spin, nocc, cnt in ((0, na, La), (1, nb, Lb)):
            occ_rank = np.argsort(rng.random((B, nocc)), axis=1).argsort(axis=1)
            vir_rank = np.argsort(rng.random((B, M - nocc)), axis=1).argsort(axis=1)
            keep_occ = occ_rank >= cnt[:, None]           # occupied orbitals that stay
            take_vir = vir_rank < cnt[:, None]            # virtual orbitals that get an electron
            occ_orbs = 2 * np.arange(nocc) + spin
            vir_orbs = 2 * np.arange(nocc, M) + spin
            r_o, c_o = np.nonzero(keep_occ)
            bits[r_o, occ_orbs[c_o]] = True
            r_v, c_v = np.nonzero(take_vir)
            bits[r_v, vir_orbs[c_v]] = True
        bits = bits[ok]
        Lk = L[ok]
        packed = np.packbits(bits, axis=1, bitorder="little")
        sg = np.where(rng.random(len(Lk)) < 0.5, 1.0, -1.0)
        for k in range(len(Lk)):
            key = packed[k].tobytes()
            if key in seen:
                continue
            seen.add(key)
            rows.append(bits[k])
            amps.append(float(np.exp(-Lk[k])) * sg[k])
            if len(rows) >= n_dets:
                break
    bits = np.array(rows)
    dets = np.packbits(bits, axis=1, bitorder="little").view("<u8").astype(np.uint64)
    return dets.reshape(len(rows), W), np.array(amps)
