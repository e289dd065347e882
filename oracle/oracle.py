"""ctypes binding of the CPU oracle (fciqmc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the CPU
baseline of the benchmark; never by the product package. The oracle shares no
code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fciqmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ROW_FIELDS = ["iter", "shift", "nw_in", "nd_in", "c0_in", "num_in", "nw_out", "nd_out",
              "attempts", "nulls", "spawn_events", "spawned_walkers", "death_walkers",
              "clone_walkers", "merged_entries", "aborted_walkers", "inserted_dets"]


class Row(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double if f in ("shift", "num_in") else ctypes.c_int64) for f in ROW_FIELDS]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP over chunks of spawning attempts)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        # FCIQMC_ORACLE_LIB lets the mutation test load a deliberately broken copy of the oracle
        L = ctypes.CDLL(os.environ.get("FCIQMC_ORACLE_LIB") or build())
        P = ctypes.POINTER
        u64p, i32p, f64p, i64p = P(ctypes.c_uint64), P(ctypes.c_int32), P(ctypes.c_double), P(ctypes.c_int64)
        L.oq_create.restype = ctypes.c_void_p
        L.oq_create.argtypes = [f64p, f64p, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                i32p, ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64,
                                ctypes.c_double, u64p]
        L.oq_destroy.argtypes = [ctypes.c_void_p]
        L.oq_philox.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.oq_digits.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u64p, ctypes.c_int, u64p]
        L.oq_log.restype = ctypes.c_double
        L.oq_log.argtypes = [ctypes.c_double]
        L.oq_fingerprint.restype = ctypes.c_uint64
        L.oq_fingerprint.argtypes = [ctypes.c_void_p, u64p]
        L.oq_hdiag.restype = ctypes.c_double
        L.oq_hdiag.argtypes = [ctypes.c_void_p, u64p]
        L.oq_hij.restype = ctypes.c_double
        L.oq_hij.argtypes = [ctypes.c_void_p, u64p, u64p]
        L.oq_excite_ranks.restype = ctypes.c_int
        L.oq_excite_ranks.argtypes = [ctypes.c_void_p, u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_uint64, u64p, i64p]
        L.oq_iterate.restype = ctypes.c_int
        L.oq_iterate.argtypes = [ctypes.c_void_p, ctypes.c_int, P(Row)]
        L.oq_n_dets.restype = ctypes.c_int64
        L.oq_n_dets.argtypes = [ctypes.c_void_p]
        L.oq_words.restype = ctypes.c_int
        L.oq_words.argtypes = [ctypes.c_void_p]
        L.oq_get_walkers.argtypes = [ctypes.c_void_p, u64p, i32p, f64p]
        L.oq_set_walkers.restype = ctypes.c_int
        L.oq_set_walkers.argtypes = [ctypes.c_void_p, u64p, i32p, ctypes.c_int64, ctypes.c_uint32,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_int]
        L.oq_get_state.argtypes = [ctypes.c_void_p, i64p, f64p, i64p, i64p, i64p]
        L.oq_info.argtypes = [ctypes.c_void_p, f64p, f64p, i64p, i64p, u64p, u64p]
        L.oq_map1.argtypes = [ctypes.c_void_p, u64p]
        L.oq_hmatrix.argtypes = [ctypes.c_void_p, u64p, ctypes.c_int64, f64p]
        L.oq_estimate.argtypes = [ctypes.c_void_p, i64p, i64p, i64p, f64p]
        L.oq_rdm.restype = ctypes.c_int
        L.oq_rdm.argtypes = [ctypes.c_void_p, u64p, f64p, ctypes.c_int64, f64p, f64p, f64p]
        L.oq_attempt.restype = ctypes.c_int64
        L.oq_attempt.argtypes = [ctypes.c_void_p, u64p, ctypes.c_int32, ctypes.c_uint32, u64p,
                                 P(ctypes.c_int)]
        L.oq_set_space.restype = ctypes.c_int
        L.oq_set_space.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p, u64p]
        L.oq_in_space.restype = ctypes.c_int
        L.oq_in_space.argtypes = [ctypes.c_void_p, u64p]
        L.oq_set_hphf.restype = ctypes.c_int
        L.oq_set_hphf.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.oq_gen_prob.restype = ctypes.c_double
        L.oq_gen_prob.argtypes = [ctypes.c_void_p, u64p, u64p]
        L.oq_hphf_hij.restype = ctypes.c_double
        L.oq_hphf_hij.argtypes = [ctypes.c_void_p, u64p, u64p]
        L.oq_hphf_hdiag.restype = ctypes.c_double
        L.oq_hphf_hdiag.argtypes = [ctypes.c_void_p, u64p]
        L.oq_set_real.restype = ctypes.c_int
        L.oq_set_real.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
        L.oq_set_threads.argtypes = [ctypes.c_int]
        L.oq_set_threads.restype = None
        L.oq_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def philox(ctr, key) -> list[int]:
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().oq_philox(c, k, o)
    return list(o)


def digits(r0: int, r1: int, radices) -> list[int]:
    """Successive mixed-radix digits of the choice word of one attempt's Philox words (r0, r1)."""
    n = np.ascontiguousarray(radices, dtype=np.uint64)
    k = np.zeros(len(n), dtype=np.uint64)
    lib().oq_digits(r0, r1, _p(n, ctypes.c_uint64), len(n), _p(k, ctypes.c_uint64))
    return [int(x) for x in k]


def log(x: float) -> float:
    return lib().oq_log(x)


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (results do not depend on it); returns the count in effect."""
    lib().oq_set_threads(int(n))
    return int(lib().oq_max_threads())


class Oracle:
    """Plain CPU FCIQMC (see fciqmc_oracle.c for the method and the readings)."""

    def __init__(self, system, *, tau, initiator_threshold=-1, target_walkers=1 << 62,
                 shift_damping=0.05, shift_period=10, initial_shift=0.0, initial_population=10,
                 seed=1, p_double=0.0, ms2=0, reference=None, max_excitation=None, max_seniority=None,
                 frozen_occupied=None, frozen_empty=None, hphf=False, walker_fraction_bits=0,
                 occupation_threshold=1.0):
        L = lib()
        self.system = system
        self.n_orb, self.n_elec = system.n_orb, system.n_elec
        self.W = (2 * system.n_orb + 63) // 64
        self._h = np.ascontiguousarray(system.h, dtype=np.float64)
        self._eri = np.ascontiguousarray(system.eri_s8, dtype=np.float64)
        irr = None
        if system.irrep is not None:
            self._irr = np.ascontiguousarray(system.irrep, dtype=np.int32)
            irr = _p(self._irr, ctypes.c_int32)
        ref = None
        if reference is not None:
            self._ref = np.ascontiguousarray(reference, dtype=np.uint64)
            ref = _p(self._ref, ctypes.c_uint64)
        self.h = L.oq_create(_p(self._h, ctypes.c_double), _p(self._eri, ctypes.c_double), system.e_core,
                             system.n_elec, system.n_orb, ms2, irr, tau, initiator_threshold,
                             target_walkers, shift_damping, shift_period, initial_shift,
                             initial_population, seed, p_double, ref)
        if not self.h:
            raise ValueError("oracle: invalid system or options")
        if max_excitation is not None or max_seniority is not None or frozen_occupied is not None \
                or frozen_empty is not None:
            flags = (1 if max_excitation is not None else 0) | (2 if max_seniority is not None else 0)
            self._fo = self._det(frozen_occupied if frozen_occupied is not None else [0, 0])
            self._fe = self._det(frozen_empty if frozen_empty is not None else [0, 0])
            if L.oq_set_space(self.h, flags, int(max_excitation or 0), int(max_seniority or 0),
                              _p(self._fo, ctypes.c_uint64), _p(self._fe, ctypes.c_uint64)) != 0:
                raise ValueError("oracle: the reference lies outside the permitted space")
        if hphf and L.oq_set_hphf(self.h, 1) != 0:
            raise ValueError("oracle: spin-coupled functions need M_s = 0 and a closed-shell reference")
        self.frac_bits = int(walker_fraction_bits)
        if self.frac_bits and L.oq_set_real(self.h, self.frac_bits, float(occupation_threshold)) != 0:
            raise ValueError("oracle: invalid hybrid-walker resolution or occupation threshold")

    def __del__(self):
        if getattr(self, "h", None):
            lib().oq_destroy(self.h)
            self.h = None

    # -- facts
    def info(self) -> dict:
        e0, pd = ctypes.c_double(), ctypes.c_double()
        ns, nd = ctypes.c_int64(), ctypes.c_int64()
        d53 = ctypes.c_uint64()
        ref = np.zeros(2, dtype=np.uint64)
        lib().oq_info(self.h, ctypes.byref(e0), ctypes.byref(pd), ctypes.byref(ns), ctypes.byref(nd),
                      ctypes.byref(d53), _p(ref, ctypes.c_uint64))
        return dict(E0=e0.value, p_double=pd.value, n_single_ref=ns.value, n_double_ref=nd.value,
                    d53=d53.value, ref=ref[:self.W].copy())

    def map1(self) -> np.ndarray:
        out = np.zeros(2 * self.n_orb, dtype=np.uint64)
        lib().oq_map1(self.h, _p(out, ctypes.c_uint64))
        return out

    def _det(self, d) -> np.ndarray:
        a = np.zeros(2, dtype=np.uint64)
        a[:self.W] = np.asarray(d, dtype=np.uint64).reshape(-1)[:self.W]
        return a

    def fingerprint(self, d) -> int:
        return int(lib().oq_fingerprint(self.h, _p(self._det(d), ctypes.c_uint64)))

    def gen_prob(self, src, dst) -> float:
        """Probability that one attempt from src generates the determinant dst."""
        return lib().oq_gen_prob(self.h, _p(self._det(src), ctypes.c_uint64), _p(self._det(dst), ctypes.c_uint64))

    def hphf_hij(self, a, b) -> float:
        return lib().oq_hphf_hij(self.h, _p(self._det(a), ctypes.c_uint64), _p(self._det(b), ctypes.c_uint64))

    def hphf_hdiag(self, a) -> float:
        return lib().oq_hphf_hdiag(self.h, _p(self._det(a), ctypes.c_uint64))

    def in_space(self, d) -> bool:
        return bool(lib().oq_in_space(self.h, _p(self._det(d), ctypes.c_uint64)))

    def hdiag(self, d) -> float:
        return lib().oq_hdiag(self.h, _p(self._det(d), ctypes.c_uint64))

    def hij(self, src, dst) -> float:
        return lib().oq_hij(self.h, _p(self._det(src), ctypes.c_uint64), _p(self._det(dst), ctypes.c_uint64))

    def hmatrix(self, dets: np.ndarray) -> np.ndarray:
        dets = np.ascontiguousarray(np.asarray(dets, dtype=np.uint64).reshape(-1, self.W))
        n = dets.shape[0]
        out = np.zeros((n, n))
        lib().oq_hmatrix(self.h, _p(dets, ctypes.c_uint64), n, _p(out, ctypes.c_double))
        return out

    def excite_ranks(self, d, kind: int, k1: int, k2: int = 0, k3: int = 0):
        child = np.zeros(2, dtype=np.uint64)
        info = np.zeros(10, dtype=np.int64)
        r = lib().oq_excite_ranks(self.h, _p(self._det(d), ctypes.c_uint64), kind, k1, k2, k3,
                                  _p(child, ctypes.c_uint64), _p(info, ctypes.c_int64))
        return r, child[:self.W].copy(), info

    def attempt(self, d, c: int, a: int):
        child = np.zeros(2, dtype=np.uint64)
        is_null = ctypes.c_int()
        amt = lib().oq_attempt(self.h, _p(self._det(d), ctypes.c_uint64), c, a, _p(child, ctypes.c_uint64),
                               ctypes.byref(is_null))
        return int(amt), child[:self.W].copy(), bool(is_null.value)

    def rdm_energy(self, dets, c):
        """E = c^T H c / c^T c over the list and its gradients (grad_h (M, M), grad_eri packed)."""
        dets = np.ascontiguousarray(np.asarray(dets, dtype=np.uint64).reshape(-1, self.W))
        c = np.ascontiguousarray(c, dtype=np.float64)
        M = self.n_orb
        npair = M * (M + 1) // 2
        gh = np.zeros((M, M))
        ge = np.zeros(npair * (npair + 1) // 2)
        E = ctypes.c_double()
        lib().oq_rdm(self.h, _p(dets, ctypes.c_uint64), _p(c, ctypes.c_double), len(c), ctypes.byref(E),
                     _p(gh, ctypes.c_double), _p(ge, ctypes.c_double))
        return E.value, gh, ge

    # -- dynamics
    def iterate(self, n: int = 1) -> list[dict]:
        rows = (Row * n)()
        rc = lib().oq_iterate(self.h, n, rows)
        if rc != 0:
            raise RuntimeError("oracle: population overflow")
        return [{f: getattr(r, f) for f in ROW_FIELDS} for r in rows]

    def walkers(self):
        n = lib().oq_n_dets(self.h)
        dets = np.zeros((max(n, 1), self.W), dtype=np.uint64)
        pops = np.zeros(max(n, 1), dtype=np.int32)
        hd = np.zeros(max(n, 1))
        lib().oq_get_walkers(self.h, _p(dets, ctypes.c_uint64), _p(pops, ctypes.c_int32), _p(hd, ctypes.c_double))
        return dets[:n], pops[:n], hd[:n]

    def set_walkers(self, dets, pops, *, iteration=0, shift=0.0, vary=False, nw_prev=0, n_since=0):
        dets = np.ascontiguousarray(np.asarray(dets, dtype=np.uint64).reshape(-1, self.W))
        pops = np.ascontiguousarray(pops, dtype=np.int32)
        rc = lib().oq_set_walkers(self.h, _p(dets, ctypes.c_uint64), _p(pops, ctypes.c_int32), len(pops),
                                  iteration, shift, int(vary), nw_prev, n_since)
        if rc == -3:
            raise ValueError("oracle: a determinant outside the permitted space in set_walkers")
        if rc == -4:
            raise ValueError("oracle: a determinant that is not the stored one of its spin-coupled pair")
        if rc != 0:
            raise ValueError("oracle: duplicate determinants in set_walkers")

    def state(self) -> dict:
        it, vary, prev, since = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        s = ctypes.c_double()
        lib().oq_get_state(self.h, ctypes.byref(it), ctypes.byref(s), ctypes.byref(vary), ctypes.byref(prev),
                           ctypes.byref(since))
        return dict(iteration=it.value, shift=s.value, vary=bool(vary.value), nw_prev=prev.value,
                    n_since=since.value)

    def estimate(self) -> dict:
        nw, nd, c0 = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        num = ctypes.c_double()
        lib().oq_estimate(self.h, ctypes.byref(nw), ctypes.byref(nd), ctypes.byref(c0), ctypes.byref(num))
        return dict(nw=nw.value, nd=nd.value, c0=c0.value, num=num.value)
