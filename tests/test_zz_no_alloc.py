"""The allocation-free estimator entry point (fciqmc_estimate_list_static) through the C ABI on the GPU,
against the estimators of a run (fciqmc_estimators) and against the oracle's estimate of the same list.

Some callers hold a walker list on the device but cannot allocate device memory when they need its
estimators (a fixed up-front memory pool, no tolerance for cudaMalloc's implicit synchronisation);
this entry point keeps its scratch in a static device array instead. Two calls in a row must both
agree with the run's own estimators: the second call reuses the array the first one left behind.
Entries that are not determinants of the run's basis are skipped and counted, never evaluated.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _static(L, system, refw, d_dev, p_dev, n, flags, out):
    dev = out.device
    h_dev = torch.from_numpy(np.ascontiguousarray(system.h)).to(dev)
    e_dev = torch.from_numpy(np.ascontiguousarray(system.eri_s8)).to(dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    rc = L.fciqmc_estimate_list_static(_ptr(h_dev), _ptr(e_dev), system.n_elec, system.n_orb,
                                       refw.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _ptr(d_dev), _ptr(p_dev),
                                       n, flags, _ptr(out), stream)
    torch.cuda.synchronize()
    return rc


def _run_and_list(which):
    from paper_1305_6981_gb300 import Fciqmc, synth
    if which == "12e24o":
        system = synth.init_12e24o()
        g = Fciqmc(system, 0.005, 3, main_capacity=1 << 18, seed=3)
        d0, p0 = synth.walker_snapshot(system, 100_000, seed=11)
        g.set_walkers(d0, p0)  # the run's own list, loaded through the existing C ABI path
        g.step(3)
    elif which == "24e60o":
        system = synth.large_24e60o()
        g = Fciqmc(system, 0.005, 3, main_capacity=1 << 18, seed=3)
        d0, p0 = synth.walker_snapshot(system, 100_000, seed=11)
        g.set_walkers(d0, p0)
        g.step(3)
    else:  # spin-coupled functions: a snapshot mapped to the stored determinants of its pairs
        system = synth.large_24e60o()
        g = Fciqmc(system, 0.005, 3, main_capacity=1 << 18, seed=3, hphf=True)
        d0, p0 = synth.stored_pairs(*synth.walker_snapshot(system, 100_000, seed=11))
        g.set_walkers(d0, p0)
        g.step(3)
    return system, g


@pytest.mark.parametrize("which", ["12e24o", "24e60o", "24e60o-spin-coupled"])
def test_static_estimator_matches_run_and_oracle_twice(which):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from oracle.oracle import Oracle
    from paper_1305_6981_gb300 import _native

    L = _native.load()
    spin = which.endswith("spin-coupled")
    system, g = _run_and_list(which)
    ref = g.estimates()
    dets, pops, _ = g.walkers()
    assert len(pops) > 300 and ref["c0"] != 0 and ref["proj_num"] != 0.0
    if spin:  # open-shell functions carry the sqrt(2) of the spin coupling: some must be present
        assert any((int(x) ^ (int(x) >> 1)) & 0x5555555555555555 for x in dets.reshape(-1))
    q = Oracle(system, tau=0.005, initiator_threshold=3, hphf=spin)
    q.set_walkers(dets, pops)
    est_q = q.estimate()
    dev = torch.device("cuda", 0)
    d_dev = torch.from_numpy(np.ascontiguousarray(dets).view(np.int64)).to(dev)
    p_dev = torch.from_numpy(np.ascontiguousarray(pops)).to(dev)
    out = torch.full((5,), -1.0, dtype=torch.float64, device=dev)
    refw = np.ascontiguousarray(g.info()["reference"], dtype=np.uint64)
    flags = _native.STATIC_SPIN_COUPLED if spin else 0
    for _ in range(2):
        assert _static(L, system, refw, d_dev, p_dev, len(pops), flags, out) == 0
        nw, nd, c0, num, bad = out.tolist()
        assert nw == ref["n_walkers"] == est_q["nw"] and nd == ref["n_dets"] == est_q["nd"]
        assert c0 == ref["c0"] == est_q["c0"] and bad == 0
        assert abs(num - ref["proj_num"]) <= 1e-11 * abs(ref["proj_num"])
        assert abs(num - est_q["num"]) <= 1e-11 * abs(est_q["num"])
    # lists beyond the static scratch are rejected before anything is launched
    assert _static(L, system, refw, d_dev, p_dev, _native.STATIC_MAX_DETS + 1, flags, out) == -2
    g.close()


def test_static_estimator_skips_invalid_entries():
    """A bit beyond the basis, a wrong electron count and an INT32_MIN population are counted in out[4] and
    contribute nothing; a reference with a bit beyond the basis is rejected on the host."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1305_6981_gb300 import _native

    L = _native.load()
    system, g = _run_and_list("24e60o")
    ref = g.estimates()
    dets, pops, _ = g.walkers()
    n_so = 2 * system.n_orb
    good = dets[0].copy()
    beyond = good.copy()
    beyond[1] ^= np.uint64(1 << (n_so - 64))  # one more electron, on a spin orbital outside the basis
    top = good.copy()
    low = int(top[0]) & -int(top[0])
    top[0] = np.uint64(int(top[0]) ^ low)
    top[1] = np.uint64(int(top[1]) | (1 << 63))  # same electron count, one moved beyond the basis
    short = good.copy()
    short[0] = np.uint64(int(short[0]) ^ low)  # an electron fewer
    extra = np.stack([beyond, top, short, good])
    extra_p = np.array([5, -7, 3, -2147483648], dtype=np.int32)
    all_d = np.concatenate([dets, extra])
    all_p = np.concatenate([pops, extra_p])
    dev = torch.device("cuda", 0)
    d_dev = torch.from_numpy(np.ascontiguousarray(all_d).view(np.int64)).to(dev)
    p_dev = torch.from_numpy(np.ascontiguousarray(all_p)).to(dev)
    out = torch.full((5,), -1.0, dtype=torch.float64, device=dev)
    refw = np.ascontiguousarray(g.info()["reference"], dtype=np.uint64)
    assert _static(L, system, refw, d_dev, p_dev, len(all_p), 0, out) == 0
    nw, nd, c0, num, bad = out.tolist()
    assert bad == 4
    assert nw == ref["n_walkers"] and nd == ref["n_dets"] and c0 == ref["c0"]
    assert abs(num - ref["proj_num"]) <= 1e-11 * abs(ref["proj_num"])
    bad_ref = refw.copy()
    bad_ref[1] |= np.uint64(1 << 63)
    bad_ref[0] = np.uint64(int(bad_ref[0]) ^ (int(bad_ref[0]) & -int(bad_ref[0])))
    assert _static(L, system, bad_ref, d_dev, p_dev, len(all_p), 0, out) == -1
    assert _static(L, system, refw, d_dev, p_dev, len(all_p), 2, out) == -1  # unknown flag
    g.close()
