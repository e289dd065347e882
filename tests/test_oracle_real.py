"""Pins of the oracle's real/integer hybrid walkers (populations in units of 2^-b walkers, attempts rounded
stochastically, spawns drawn in units, an occupation threshold below which amplitudes are rounded to
+-threshold or removed). Every step is unbiased, so one iteration must follow Eq. 1 in expectation, as for
integer walkers; the attempt count must average to N_w; no amplitude below the threshold may survive."""
from __future__ import annotations

import numpy as np
import pytest

import bruteforce as bf
from oracle import oracle as O
from paper_1305_6981_gb300 import synth

BITS = 6
R = 1 << BITS


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_8e8o()


@pytest.fixture(scope="module")
def tiny_space(tiny):
    dets = bf.basis(8, 4, 4)
    return dets, bf.hamiltonian(8, tiny.h, tiny.eri_s8, dets)


def _state(dets, n, seed):
    """n determinants (the reference among them) with amplitudes between 0.2 and 5 walkers, some below the
    occupation threshold of one walker, in units of 2^-BITS."""
    rng = np.random.default_rng(seed)
    ref = 0xFF
    idx = rng.choice(len(dets), n, replace=False)
    chosen = [dets[i] for i in idx if dets[i] != ref][: n - 1] + [ref]
    units = rng.integers(int(0.2 * R), 5 * R, len(chosen)) * rng.choice([-1, 1], len(chosen))
    units[-1] = 40 * R + 17
    return chosen, units.astype(np.int32)


@pytest.mark.parametrize("S", [-0.4, 8.0])
def test_hybrid_one_step_expectation_is_eq1(tiny, tiny_space, S):
    """E[C^(n+1)] = [1 - tau (H_ii - E0 - S)] C - tau H_offdiag C (Eq. 1) with C in walkers, over 6000 keys."""
    dets, H = tiny_space
    index = {d: i for i, d in enumerate(dets)}
    chosen, units = _state(dets, 25, 5)
    tau = 0.05
    q = O.Oracle(tiny, tau=tau, initial_shift=S, walker_fraction_bits=BITS, occupation_threshold=1.0)
    E0 = q.info()["E0"]
    c = np.zeros(len(dets))
    for d, u in zip(chosen, units):
        c[index[d]] = u / R
    expect = R * (c - tau * ((np.diag(H) - E0 - S) * c) - tau * ((H - np.diag(np.diag(H))) @ c))  # in units
    K = 6000
    acc = np.zeros(len(dets))
    acc2 = np.zeros(len(dets))
    words = np.array([bf.to_words(d, 1) for d in chosen])
    below = 0
    for k in range(K):
        q.set_walkers(words, units, iteration=k, shift=S)
        q.iterate(1)
        dd, pp, _ = q.walkers()
        below += int(np.sum(np.abs(pp) < R))
        v = np.zeros(len(dets))
        for w, p in zip(dd, pp):
            v[index[int(w[0])]] = p
        acc += v
        acc2 += v * v
    assert below == 0  # the occupation threshold leaves nothing between 0 and one walker
    mean = acc / K
    var = acc2 / K - mean ** 2
    touched = (var > 0) | (expect != 0)
    # every nonzero outcome has at least one walker (R units) after the occupation threshold, so
    # E[x^2] >= R |E[x]|: a component rarely hit still has variance of at least R |E[x]| - E[x]^2
    floor_var = np.clip(np.abs(expect) * R - expect ** 2, 0, None)
    var_eff = np.maximum(var, floor_var)
    z = np.abs(mean - expect)[touched] / np.sqrt(var_eff[touched] / K)
    assert np.all(np.isfinite(z))
    assert z.max() < 5.0, z.max()
    assert touched.sum() > 100


def test_hybrid_attempts_average_to_walkers(tiny, tiny_space):
    """A determinant with |C| walkers makes floor(|C|) or floor(|C|) + 1 attempts, |C| on average."""
    dets, _ = tiny_space
    chosen, units = _state(dets, 40, 9)
    words = np.array([bf.to_words(d, 1) for d in chosen])
    q = O.Oracle(tiny, tau=0.01, walker_fraction_bits=BITS)
    nw = float(np.abs(units).sum()) / R
    lo = int(np.sum(np.abs(units) // R))
    att = []
    for k in range(3000):
        q.set_walkers(words, units, iteration=k)
        r = q.iterate(1)[0]
        assert lo <= r["attempts"] <= lo + len(units)
        att.append(r["attempts"])
    att = np.array(att, dtype=float)
    sd = np.sqrt(0.25 * len(units) / len(att))  # each rounding has variance at most 1/4
    assert abs(att.mean() - nw) < 5 * sd


def test_hybrid_options_are_checked(tiny):
    with pytest.raises(ValueError):
        O.Oracle(tiny, tau=0.01, walker_fraction_bits=21)
    with pytest.raises(ValueError):
        O.Oracle(tiny, tau=0.01, walker_fraction_bits=4, occupation_threshold=0.01)  # below one unit


@pytest.mark.slow
def test_hybrid_dynamics_reach_fci_energy(tiny, tiny_space):
    """Plain dynamics with hybrid walkers on 8e/8o: the time-averaged projected energy agrees with the
    lowest eigenvalue of the brute-force Hamiltonian within its statistical error."""
    _, H = tiny_space
    e_fci = float(np.linalg.eigvalsh(H)[0])
    q = O.Oracle(tiny, tau=0.01, target_walkers=300, initial_population=20, initial_shift=0.3, seed=4,
                 walker_fraction_bits=BITS, occupation_threshold=1.0)
    q.iterate(1500)
    num, c0 = [], []
    for _ in range(40):
        rows = q.iterate(100)
        num += [r["num_in"] for r in rows]
        c0 += [r["c0_in"] for r in rows]
    e0 = q.info()["E0"]
    blocks = [(np.mean(num[i:i + 400]), np.mean(c0[i:i + 400])) for i in range(0, len(num), 400)]
    e_blocks = np.array([e0 + n / c for n, c in blocks])
    err = e_blocks.std(ddof=1) / np.sqrt(len(e_blocks))
    assert abs(e_blocks.mean() - e_fci) < 4 * err + 2e-3, (e_blocks.mean(), e_fci, err)
