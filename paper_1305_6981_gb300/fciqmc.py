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
            cur = self.state() if shift is None or vary is None else {}
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


def owners(n_orb: int, dets, n_partitions: int) -> np.ndarray:
    """Partition of each determinant in a run of n_partitions partitions (fciqmc_owner: the Algorithm 1
    fingerprint mod n_partitions); host only."""
    W = words_for(n_orb)
    d = np.ascontiguousarray(np.asarray(dets, dtype=np.uint64).reshape(-1, W))
    out = np.zeros(len(d), dtype=np.int32)
    check(_native.load().fciqmc_owner(int(n_orb), _ptr(d, ctypes.c_uint64), len(d), int(n_partitions),
                                      _ptr(out, ctypes.c_int32)), "fciqmc_owner")
    return out


class Partitioned:
    """One run divided among n_partitions hash partitions on one GPU (Sec. V A; fciqmc_group_*): each
    partition is an Fciqmc handle holding the determinants that fciqmc_owner assigns to it, and an
    iteration spawns in every partition, exchanges the spawns onto other partitions' determinants, annihilates
    and takes one shift update from the run's N_w. Arguments as for Fciqmc (options apply to every
    partition); outbox_capacity sets the entries of each per-destination outbox."""

    def __init__(self, system, tau: float, initiator_threshold: int = -1, *, n_partitions: int = 2,
                 history_capacity: int = 1 << 16, stream=None, **kw):
        import torch

        self._L = L = _native.load()
        self.n_orb = int(system.n_orb)
        self.n = int(n_partitions)
        self.parts = [Fciqmc(system, tau, initiator_threshold, n_partitions=self.n, partition_index=r,
                             stream=stream, **kw) for r in range(self.n)]
        self.stream = self.parts[0].stream
        nbytes = L.fciqmc_group_workspace_bytes(self.n, int(history_capacity))
        if nbytes == 0:
            raise ValueError("unsupported number of partitions")
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=self.parts[0].device)
        arr = (ctypes.c_void_p * self.n)(*[p.handle.value for p in self.parts])
        h = ctypes.c_void_p()
        check(L.fciqmc_group_create(arr, self.n, int(history_capacity), ctypes.c_void_p(self.workspace.data_ptr()),
                                    int(nbytes), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
              "fciqmc_group_create")
        self.handle = h

    def step(self, n: int = 1):
        check(self._L.fciqmc_group_step(self.handle, int(n)), "fciqmc_group_step")

    def sync(self) -> int:
        return check(self._L.fciqmc_group_sync(self.handle), "fciqmc_group_sync")

    def history(self, max_rows: int = 1 << 16) -> list[dict]:
        rows = (Row * max_rows)()
        n = ctypes.c_int64()
        check(self._L.fciqmc_group_history(self.handle, rows, max_rows, ctypes.byref(n)), "fciqmc_group_history")
        return [{f: getattr(rows[k], f) for f in ROW_FIELDS} for k in range(n.value)]

    def walkers(self):
        """The run's list: the partitions' lists concatenated (dets, pops, H_ii - E0)."""
        parts = [p.walkers() for p in self.parts]
        return tuple(np.concatenate([x[k] for x in parts]) for k in range(3))

    def estimates(self) -> dict:
        """Estimators of the run's list: walkers, determinants, C_0 and numerator summed over the partitions
        (numerators in partition order); shift and status of partition 0 (the same in every partition)."""
        es = [p.estimates() for p in self.parts]
        out = dict(es[0])
        for k in ("n_walkers", "n_dets", "c0"):
            out[k] = sum(e[k] for e in es)
        num = 0.0
        for e in es:
            num += e["proj_num"]
        out["proj_num"] = num
        out["e_proj"] = out["e_ref"] + num / out["c0"] if out["c0"] else float("nan")
        out["status"] = next((e["status"] for e in es if e["status"]), 0)
        return out

    def set_walkers(self, dets, pops, hdiag=None, **state):
        """Loads a list, each determinant into its partition; state keywords as for Fciqmc.set_walkers."""
        W = self.parts[0].W
        dets = np.asarray(dets, dtype=np.uint64).reshape(-1, W)
        pops = np.asarray(pops, dtype=np.int32)
        own = owners(self.n_orb, dets, self.n)
        for r, p in enumerate(self.parts):
            m = own == r
            p.set_walkers(dets[m], pops[m], None if hdiag is None else np.asarray(hdiag)[m], **state)

    def close(self):
        if getattr(self, "handle", None):
            self._L.fciqmc_group_destroy(self.handle)
            self.handle = None
        for p in self.parts:
            p.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
