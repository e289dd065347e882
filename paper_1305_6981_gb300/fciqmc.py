"""Python front end of the CUDA FCIQMC walker cycle.

Argument marshalling only: PyTorch supplies the device workspace and the CUDA
stream; every step of the walker cycle runs in libfciqmc.so (include/fciqmc.h).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import Estimates, Info, Options, Row, ROW_FIELDS, State, check


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def words_for(n_orb: int) -> int:
    """uint64 words per determinant: ceil(2 n_orb / 64)."""
    return (2 * n_orb + 63) // 64


class Fciqmc:
    """One FCIQMC run on one GPU.

    system: object with n_orb, n_elec, h (n_orb x n_orb), eri_s8 (packed), irrep (or None), e_core.
    Options are the fields of fciqmc_options (shift_damping, shift_period, initial_population,
    initial_shift, target_walkers, seed, p_double, main_capacity, spawn_capacity, history_capacity,
    grid_blocks, index_load). The permitted space (Sec. VI) is given by max_excitation, max_seniority
    (None: no limit), frozen_occupied and frozen_empty (W words or None); hphf=True puts the walkers
    on spin-coupled functions (Sec. VI C).
    """

    def __init__(self, system, tau: float, initiator_threshold: int = -1, *, ms2: int = 0, reference=None,
                 device=None, stream=None, max_excitation=None, max_seniority=None, frozen_occupied=None,
                 frozen_empty=None, hphf=False, **options):
        import torch

        self._L = L = _native.load()
        self.n_orb, self.n_elec = int(system.n_orb), int(system.n_elec)
        self.W = words_for(self.n_orb)
        o = Options()
        L.fciqmc_default_options(ctypes.byref(o))
        for k, v in options.items():
            if not hasattr(o, k) or k in ("reference", "space_flags", "max_excitation", "max_seniority",
                                          "frozen_occupied", "frozen_empty", "hphf"):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        o.hphf = 1 if hphf else 0
        if max_excitation is not None:
            o.space_flags |= 1
            o.max_excitation = int(max_excitation)
        if max_seniority is not None:
            o.space_flags |= 2
            o.max_seniority = int(max_seniority)
        self._frozen = []
        for name, mask in (("frozen_occupied", frozen_occupied), ("frozen_empty", frozen_empty)):
            if mask is not None:
                m = np.zeros(2, dtype=np.uint64)
                m[:self.W] = np.asarray(mask, dtype=np.uint64).reshape(-1)[:self.W]
                self._frozen.append(m)
                setattr(o, name, _ptr(m, ctypes.c_uint64))
        self._ref = None
        if reference is not None:
            self._ref = np.zeros(2, dtype=np.uint64)
            self._ref[:self.W] = np.asarray(reference, dtype=np.uint64).reshape(-1)[:self.W]
            o.reference = _ptr(self._ref, ctypes.c_uint64)
        self.options = o
        nbytes = L.fciqmc_workspace_bytes(self.n_elec, self.n_orb, ctypes.byref(o))
        if nbytes == 0:
            raise ValueError("unsupported problem size")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
        h = np.ascontiguousarray(system.h, dtype=np.float64)
        eri = np.ascontiguousarray(system.eri_s8, dtype=np.float64)
        irr = None
        if getattr(system, "irrep", None) is not None:
            self._irr = np.ascontiguousarray(system.irrep, dtype=np.int32)
            irr = _ptr(self._irr, ctypes.c_int32)
        handle = ctypes.c_void_p()
        with torch.cuda.device(dev):
            rc = L.fciqmc_create(_ptr(h, ctypes.c_double), _ptr(eri, ctypes.c_double),
                                 float(getattr(system, "e_core", 0.0)), self.n_elec, self.n_orb, ms2, irr,
                                 float(tau), int(initiator_threshold), ctypes.byref(o),
                                 ctypes.c_void_p(self.workspace.data_ptr()), int(nbytes),
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle))
        check(rc, "fciqmc_create")
        self.handle = handle

    # ------------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "handle", None):
            self._L.fciqmc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ iteration
    def step(self, n: int = 1):
        check(self._L.fciqmc_step(self.handle, int(n)), "fciqmc_step")

    def sync(self) -> int:
        return check(self._L.fciqmc_sync(self.handle), "fciqmc_sync")

    # ------------------------------------------------------------------ read-back
    def estimates(self) -> dict:
        """Estimators of the current list; a sticky device error is reported in ["status"]."""
        e = Estimates()
        rc = self._L.fciqmc_estimators(self.handle, ctypes.byref(e))
        if rc != e.status:
            check(rc, "fciqmc_estimators")
        return {f: getattr(e, f) for f, _ in Estimates._fields_}

    def profile(self, n: int = 1) -> dict:
        """Runs n iterations kernel by kernel between CUDA events; milliseconds summed per kernel."""
        ms = np.zeros(_native.N_KERNELS)
        check(self._L.fciqmc_profile(self.handle, int(n), _ptr(ms, ctypes.c_double)), "fciqmc_profile")
        return dict(zip(_native.KERNEL_NAMES, ms.tolist()))

    def walkers_into(self, dets: np.ndarray, pops: np.ndarray, hdiag: np.ndarray | None = None) -> int:
        """Reads the walker list into caller-provided host arrays (e.g. pinned); returns the count."""
        n = ctypes.c_int64()
        hd_ptr = _ptr(hdiag, ctypes.c_double) if hdiag is not None else None
        rc = self._L.fciqmc_get_walkers(self.handle, _ptr(dets, ctypes.c_uint64), _ptr(pops, ctypes.c_int32),
                                        hd_ptr, len(pops), ctypes.byref(n))
        check(rc, "fciqmc_get_walkers")
        return n.value

    def history(self, max_rows: int = 1 << 16) -> list[dict]:
        rows = (Row * max_rows)()
        n = ctypes.c_int64()
        check(self._L.fciqmc_history(self.handle, rows, max_rows, ctypes.byref(n)), "fciqmc_history")
        return [{f: getattr(rows[k], f) for f in ROW_FIELDS} for k in range(n.value)]

    def walkers(self):
        """(dets (n, W) uint64, pops (n,) int32, H_ii - E0 (n,) float64), in unspecified order."""
        n = ctypes.c_int64()
        cap = 1024
        while True:
            dets = np.zeros((cap, self.W), dtype=np.uint64)
            pops = np.zeros(cap, dtype=np.int32)
            hd = np.zeros(cap)
            rc = self._L.fciqmc_get_walkers(self.handle, _ptr(dets, ctypes.c_uint64), _ptr(pops, ctypes.c_int32),
                                            _ptr(hd, ctypes.c_double), cap, ctypes.byref(n))
            if rc == _native_capacity() and n.value > cap:
                cap = n.value
                continue
            check(rc, "fciqmc_get_walkers")
            return dets[:n.value], pops[:n.value], hd[:n.value]

    def set_walkers(self, dets, pops, hdiag=None, *, iteration=None, shift=None, vary=None, shift_counter=0,
                    nw_last_update=0):
        dets = np.ascontiguousarray(np.asarray(dets, dtype=np.uint64).reshape(-1, self.W))
        pops = np.ascontiguousarray(pops, dtype=np.int32)
        hd_ptr = None
        if hdiag is not None:
            hd = np.ascontiguousarray(hdiag, dtype=np.float64)
            hd_ptr = _ptr(hd, ctypes.c_double)
        st = None
        if iteration is not None:
            cur = self.state()
            st = State(int(iteration), float(cur["shift"] if shift is None else shift),
                       int(cur["vary_shift"] if vary is None else vary), int(shift_counter), int(nw_last_update))
        rc = self._L.fciqmc_set_walkers(self.handle, _ptr(dets, ctypes.c_uint64), _ptr(pops, ctypes.c_int32),
                                        hd_ptr, len(pops), ctypes.byref(st) if st is not None else None)
        check(rc, "fciqmc_set_walkers")

    def state(self) -> dict:
        s = State()
        check(self._L.fciqmc_get_state(self.handle, ctypes.byref(s)), "fciqmc_get_state")
        return {f: getattr(s, f) for f, _ in State._fields_}

    def info(self) -> dict:
        i = Info()
        check(self._L.fciqmc_get_info(self.handle, ctypes.byref(i)), "fciqmc_get_info")
        d = {f: getattr(i, f) for f, _ in Info._fields_}
        d["reference"] = np.array(list(i.reference), dtype=np.uint64)[:self.W]
        return d


def _native_capacity() -> int:
    return -2  # FCIQMC_ERR_CAPACITY


class Batch:
    """Several independent runs advanced together by one CUDA graph (fciqmc_batch_*): each launch advances
    every run by `iterations_per_launch` iterations, the runs' kernels executing concurrently."""

    def __init__(self, runs: list, iterations_per_launch: int = 10, stream=None):
        import torch

        self._L = L = _native.load()
        self.runs = list(runs)
        self.iterations_per_launch = int(iterations_per_launch)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.runs[0].device)
        arr = (ctypes.c_void_p * len(self.runs))(*[r.handle.value for r in self.runs])
        h = ctypes.c_void_p()
        check(L.fciqmc_batch_create(arr, len(self.runs), self.iterations_per_launch, ctypes.byref(h)),
              "fciqmc_batch_create")
        self.handle = h

    def step(self, n_launches: int = 1):
        check(self._L.fciqmc_batch_step(self.handle, int(n_launches), ctypes.c_void_p(self.stream.cuda_stream)),
              "fciqmc_batch_step")

    def close(self):
        if getattr(self, "handle", None):
            self._L.fciqmc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rng_throughput(n_blocks: int = 1 << 31, stream=None) -> float:
    """Philox4x32-10 blocks per second on the current device, keyed like spawning attempts
    (fciqmc_rng_throughput): the rate no walker cycle's attempts/s can exceed."""
    import torch

    L = _native.load()
    s = stream if stream is not None else torch.cuda.current_stream()
    out = ctypes.c_double()
    check(L.fciqmc_rng_throughput(int(n_blocks), ctypes.c_void_p(s.cuda_stream), ctypes.byref(out)),
          "fciqmc_rng_throughput")
    return out.value
