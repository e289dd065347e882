"""Energy functional E(h, V; c) and its density-matrix gradient on the GPU, through the C ABI, against the
oracle (which builds the density matrices by applying the operators), exact diagonalisation, a
brute-force count of connected pairs, and central finite differences (E is linear in h and V, so the
differences are exact up to rounding)."""
from __future__ import annotations

import numpy as np
import pytest

import bruteforce as bf
from oracle.oracle import Oracle
from paper_1305_6981_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to("cuda")


def _functional(system, dets, c):
    from paper_1305_6981_gb300 import EnergyFunctional
    return EnergyFunctional(system.n_elec, system.n_orb, dets, c)


def _count_pairs(dets):
    """Brute-force numbers of single- and double-excitation pairs (unordered, distinct determinants)."""
    ints = [bf.from_words(w) for w in dets]
    ns = nd = 0
    for a in range(len(ints)):
        for b in range(a + 1, len(ints)):
            x = bin(ints[a] ^ ints[b]).count("1")
            ns += x == 2
            nd += x == 4
    return ns, nd


def test_full_space_ground_state_8e8o():
    s = synth.tiny_8e8o()
    space = bf.basis(8, 4, 4)
    H = bf.hamiltonian(8, s.h, s.eri_s8, space)
    w, v = np.linalg.eigh(H)
    dets = np.array([bf.to_words(d, 1) for d in space])
    f = _functional(s, dets, v[:, 0])
    E = float(f.energy(_dev(s.h), _dev(s.eri_s8)))
    gh, ge = f.gradient(torch.ones((), dtype=torch.float64, device="cuda"))
    Eq, ghq, geq = Oracle(s, tau=0.01).rdm_energy(dets, v[:, 0])
    assert abs(E - w[0]) < 1e-10
    assert abs(E - Eq) < 1e-11
    assert np.abs(gh.cpu().numpy() - ghq).max() < 1e-12
    assert np.abs(ge.cpu().numpy() - geq).max() < 1e-12
    f.close()


@pytest.mark.parametrize("n", [600, 3000, 10000])
def test_sampled_vector_16e40o_matches_oracle(n):
    s = synth.rdm_16e40o()
    dets, c = synth.sampled_vector(s, n, seed=5)
    f = _functional(s, dets, c)
    E = float(f.energy(_dev(s.h), _dev(s.eri_s8)))
    gh, ge = f.gradient(torch.ones((), dtype=torch.float64, device="cuda"))
    Eq, ghq, geq = Oracle(s, tau=0.01).rdm_energy(dets, c)
    assert abs(E - Eq) <= 1e-12 * abs(Eq)
    assert np.abs(gh.cpu().numpy() - ghq).max() < 1e-12
    assert np.abs(ge.cpu().numpy() - geq).max() < 1e-12
    if n <= 600:
        info = f.info()
        ns, nd = _count_pairs(dets)
        assert info["single_pairs"] == ns and info["double_pairs"] == nd
    f.close()


def test_autograd_function_and_repeatability():
    from paper_1305_6981_gb300 import rdm_energy
    s = synth.rdm_16e40o()
    dets, c = synth.sampled_vector(s, 2000, seed=6)
    f = _functional(s, dets, c)
    h = _dev(s.h).requires_grad_(True)
    eri = _dev(s.eri_s8).requires_grad_(True)
    E = rdm_energy(h, eri, f)
    (2.5 * E).backward()
    gh, ge = f.gradient(torch.tensor(2.5, dtype=torch.float64, device="cuda"))
    assert torch.equal(h.grad, gh) and torch.equal(eri.grad, ge)
    E2 = f.energy(h.detach(), eri.detach())
    assert float(E2) == float(E.detach())  # fixed reduction order
    f.close()


def test_finite_differences_and_linearity_at_scale():
    """2e5 determinants of 16e/40o: E = sum h grad_h + sum V grad_eri, and central differences
    (step 1e-6) of every diagonal and 60 off-diagonal h entries and 200 ERI entries agree with the
    gradient within 1e-8."""
    s = synth.rdm_16e40o()
    dets, c = synth.sampled_vector(s, 200_000, seed=5)
    f = _functional(s, dets, c)
    h0, v0 = _dev(s.h), _dev(s.eri_s8)
    E = float(f.energy(h0, v0))
    gh, ge = f.gradient(torch.ones((), dtype=torch.float64, device="cuda"))
    lin = float((h0 * gh).sum() + (v0 * ge).sum())
    assert abs(E - lin) <= 1e-12 * abs(E)
    eps = 1e-6
    rng = np.random.default_rng(3)
    pairs = [(p, p) for p in range(40)] + [tuple(sorted(rng.choice(40, 2, replace=False))) for _ in range(60)]
    ghn = gh.cpu().numpy()
    for p, q in pairs:
        d = torch.zeros_like(h0)
        d[p, q] += eps
        if p != q:
            d[q, p] += eps
        fd = (float(f.energy(h0 + d, v0)) - float(f.energy(h0 - d, v0))) / (2 * eps)
        an = ghn[p, q] + (ghn[q, p] if p != q else 0.0)
        assert abs(fd - an) < 1e-8, (p, q, fd, an)
    gen = ge.cpu().numpy()
    for k in rng.choice(len(s.eri_s8), 200, replace=False):
        d = torch.zeros_like(v0)
        d[int(k)] = eps
        fd = (float(f.energy(h0, v0 + d)) - float(f.energy(h0, v0 - d))) / (2 * eps)
        assert abs(fd - gen[k]) < 1e-8, (k, fd, gen[k])
    f.close()


def test_full_size_million_determinants():
    """The 1e6-determinant 16e/40o vector: linearity identity and 20 sampled central differences."""
    s = synth.rdm_16e40o()
    dets, c = synth.sampled_vector(s, 1_000_000, seed=5)
    f = _functional(s, dets, c)
    h0, v0 = _dev(s.h), _dev(s.eri_s8)
    E = float(f.energy(h0, v0))
    gh, ge = f.gradient(torch.ones((), dtype=torch.float64, device="cuda"))
    assert abs(E - float((h0 * gh).sum() + (v0 * ge).sum())) <= 1e-12 * abs(E)
    assert abs(float(torch.trace(gh)) - 16.0) < 1e-10  # particle number
    eps = 1e-6
    rng = np.random.default_rng(9)
    ghn, gen = gh.cpu().numpy(), ge.cpu().numpy()
    for p, q in [(0, 0), (5, 5), (1, 2), (7, 31), (20, 39)]:
        d = torch.zeros_like(h0)
        d[p, q] += eps
        if p != q:
            d[q, p] += eps
        fd = (float(f.energy(h0 + d, v0)) - float(f.energy(h0 - d, v0))) / (2 * eps)
        assert abs(fd - (ghn[p, q] + (ghn[q, p] if p != q else 0.0))) < 1e-8
    for k in rng.choice(len(s.eri_s8), 15, replace=False):
        d = torch.zeros_like(v0)
        d[int(k)] = eps
        fd = (float(f.energy(h0, v0 + d)) - float(f.energy(h0, v0 - d))) / (2 * eps)
        assert abs(fd - gen[k]) < 1e-8
    f.close()
