"""The allocation-free estimator entry point (fciqmc_estimate_list_static) against the estimators of
a run (fciqmc_estimators), through the C ABI on the GPU.

Some callers hold a walker list on the device but cannot allocate device memory when they need its
estimators (a fixed up-front memory pool, no tolerance for cudaMalloc's implicit synchronisation);
this entry point keeps its scratch in a static device array instead. Two calls in a row must both
agree with the run's own estimators: the second call reuses the array the first one left behind.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("which", ["12e24o", "24e60o"])
def test_static_estimator_matches_run_estimators_twice(which):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1305_6981_gb300 import Fciqmc, _native, synth

    L = _native.load()
    system = synth.init_12e24o() if which == "12e24o" else synth.large_24e60o()
    g = Fciqmc(system, 0.005, 3, main_capacity=1 << 18, seed=3)
    d0, p0 = synth.walker_snapshot(system, 100_000, seed=11)
    g.set_walkers(d0, p0)  # the run's own list, loaded through the existing C ABI path
    g.step(3)
    ref = g.estimates()
    dets, pops, _ = g.walkers()
    assert len(pops) > 300 and ref["c0"] != 0 and ref["proj_num"] != 0.0
    dev = torch.device("cuda", 0)
    d_dev = torch.from_numpy(np.ascontiguousarray(dets).view(np.int64)).to(dev)
    p_dev = torch.from_numpy(np.ascontiguousarray(pops)).to(dev)
    h_dev = torch.from_numpy(np.ascontiguousarray(system.h)).to(dev)
    e_dev = torch.from_numpy(np.ascontiguousarray(system.eri_s8)).to(dev)
    out = torch.full((4,), -1.0, dtype=torch.float64, device=dev)
    refw = np.ascontiguousarray(g.info()["reference"], dtype=np.uint64)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for _ in range(2):
        rc = L.fciqmc_estimate_list_static(_ptr(h_dev), _ptr(e_dev), system.n_elec, system.n_orb,
                                           refw.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _ptr(d_dev),
                                           _ptr(p_dev), len(pops), _ptr(out), stream)
        assert rc == 0
        torch.cuda.synchronize()
        nw, nd, c0, num = out.tolist()
        assert nw == ref["n_walkers"] and nd == ref["n_dets"] and c0 == ref["c0"]
        assert abs(num - ref["proj_num"]) <= 1e-11 * abs(ref["proj_num"])
    # lists beyond the static scratch are rejected before anything is launched
    rc = L.fciqmc_estimate_list_static(_ptr(h_dev), _ptr(e_dev), system.n_elec, system.n_orb,
                                       refw.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _ptr(d_dev), _ptr(p_dev),
                                       _native.STATIC_MAX_DETS + 1, _ptr(out), stream)
    assert rc == -2
    g.close()
