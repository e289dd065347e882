"""Build and load the CUDA library (libfciqmc.so) and declare its C ABI for ctypes.

The library is compiled in-tree for sm_103a with nvcc. There is no fallback: if
the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
# FCIQMC_DEBUG_BUILD=1 selects the debug build (-DFCIQMC_DEBUG: device table indices checked, a violation
# reported as FCIQMC_ERR_BOUNDS), built and loaded as its own library beside the normal one.
DEBUG = os.environ.get("FCIQMC_DEBUG_BUILD", "") == "1"
LIB = os.path.join(BUILD, "libfciqmc_debug.so" if DEBUG else "libfciqmc.so")
SOURCES = ["fciqmc.cu", "fciqmc_spawn_w1.cu", "fciqmc_spawn_w2.cu", "fciqmc_static.cu", "fciqmc_rdm.cu"]
DEPS = SOURCES + ["fciqmc_kernels.cuh", "fciqmc_cycle.cuh", "fciqmc_device.cuh", "fciqmc_spawn.h", "fciqmc_spawn_impl.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-ffp-contract=off", "-fmad=false"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, d) for d in DEPS] + [os.path.join(INCLUDE, "fciqmc.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libfciqmc.so for sm_103a (only when sources changed)."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tag = f".tmp{os.getpid()}" + ("d" if DEBUG else "")
    extra = os.environ.get("FCIQMC_NVCC_FLAGS", "").split()  # tuning defines, e.g. -DFQ_SWEEP_MIN_BLOCKS=3
    if DEBUG:
        extra.append("-DFCIQMC_DEBUG")
    compile_flags = [f for f in NVCC_FLAGS if f != "-shared"]
    objs, procs = [], []
    for src in SOURCES:  # one nvcc per translation unit, in parallel
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + tag + ".o")
        cmd = [nvcc(), ARCH, *compile_flags, *extra, "-I" + INCLUDE, "-c", "-o", obj, os.path.join(CSRC, src)]
        if verbose:
            print(" ".join(cmd))
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd)))
    failed = [cmd for cmd, p in procs if p.wait() != 0]
    try:
        if failed:
            raise subprocess.CalledProcessError(1, failed[0])
        tmp = LIB + tag
        subprocess.check_call([nvcc(), ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    finally:
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    return LIB


class Options(ctypes.Structure):
    _fields_ = [("shift_damping", ctypes.c_double), ("shift_period", ctypes.c_int32),
                ("initial_population", ctypes.c_int32), ("initial_shift", ctypes.c_double),
                ("target_walkers", ctypes.c_int64), ("seed", ctypes.c_uint64), ("p_double", ctypes.c_double),
                ("main_capacity", ctypes.c_int64), ("spawn_capacity", ctypes.c_int64),
                ("history_capacity", ctypes.c_int64), ("reference", ctypes.POINTER(ctypes.c_uint64)),
                ("grid_blocks", ctypes.c_int32), ("index_load", ctypes.c_double),
                ("space_flags", ctypes.c_uint32), ("max_excitation", ctypes.c_int32),
                ("max_seniority", ctypes.c_int32), ("frozen_occupied", ctypes.POINTER(ctypes.c_uint64)),
                ("frozen_empty", ctypes.POINTER(ctypes.c_uint64)), ("hphf", ctypes.c_int32),
                ("n_partitions", ctypes.c_int32), ("partition_index", ctypes.c_int32),
                ("outbox_capacity", ctypes.c_int64), ("walker_fraction_bits", ctypes.c_int32),
                ("occupation_threshold", ctypes.c_double)]


ROW_FIELDS = ["iteration", "shift", "nw_in", "nd_in", "c0_in", "num_in", "nw_out", "nd_out", "attempts", "nulls",
              "spawn_events", "spawned_walkers", "death_walkers", "clone_walkers", "merged_entries",
              "aborted_walkers", "inserted_dets", "heavy_attempts"]


class Row(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double if f in ("shift", "num_in") else ctypes.c_int64) for f in ROW_FIELDS]


class Estimates(ctypes.Structure):
    _fields_ = [("iteration", ctypes.c_int64), ("shift", ctypes.c_double), ("e_ref", ctypes.c_double),
                ("e_shift", ctypes.c_double), ("e_proj", ctypes.c_double), ("proj_num", ctypes.c_double),
                ("c0", ctypes.c_int64), ("n_walkers", ctypes.c_int64), ("n_dets", ctypes.c_int64),
                ("vary_shift", ctypes.c_int32), ("status", ctypes.c_int32), ("list_slots", ctypes.c_int64),
                ("compactions", ctypes.c_int64), ("exact_spawns", ctypes.c_int64), ("exact_deaths", ctypes.c_int64)]


class State(ctypes.Structure):
    _fields_ = [("iteration", ctypes.c_int64), ("shift", ctypes.c_double), ("vary_shift", ctypes.c_int32),
                ("shift_counter", ctypes.c_int32), ("nw_last_update", ctypes.c_int64)]


class Info(ctypes.Structure):
    _fields_ = [("n_elec", ctypes.c_int32), ("n_orb", ctypes.c_int32), ("words", ctypes.c_int32),
                ("e0", ctypes.c_double), ("e_core", ctypes.c_double), ("p_double", ctypes.c_double),
                ("d53", ctypes.c_uint64), ("n_single_ref", ctypes.c_int64), ("n_double_ref", ctypes.c_int64),
                ("reference", ctypes.c_uint64 * 2), ("main_capacity", ctypes.c_int64),
                ("index_capacity", ctypes.c_int64), ("spawn_capacity", ctypes.c_int64),
                ("history_capacity", ctypes.c_int64), ("workspace_bytes", ctypes.c_size_t),
                ("grid_blocks", ctypes.c_int32), ("num_sms", ctypes.c_int32),
                ("reference_excitations", ctypes.c_int64)]


# every symbol declared in include/fciqmc.h
SYMBOLS = ["fciqmc_default_options", "fciqmc_workspace_bytes", "fciqmc_create", "fciqmc_step", "fciqmc_sync",
           "fciqmc_estimators", "fciqmc_history", "fciqmc_n_dets", "fciqmc_get_walkers", "fciqmc_set_walkers",
           "fciqmc_get_state", "fciqmc_get_info", "fciqmc_profile", "fciqmc_estimate_list_static", "fciqmc_destroy",
           "fciqmc_strerror", "fciqmc_rdm_workspace_bytes", "fciqmc_rdm_create", "fciqmc_rdm_energy",
           "fciqmc_rdm_gradient", "fciqmc_rdm_info", "fciqmc_rdm_destroy", "fciqmc_batch_create",
           "fciqmc_batch_step", "fciqmc_batch_destroy", "fciqmc_rng_throughput", "fciqmc_group_workspace_bytes",
           "fciqmc_group_create", "fciqmc_group_step", "fciqmc_group_sync", "fciqmc_group_history",
           "fciqmc_group_destroy", "fciqmc_owner"]
STATIC_MAX_DETS = 1 << 23
STATIC_SPIN_COUPLED = 1
N_KERNELS = 8
KERNEL_NAMES = ["compact_copy", "index_clear", "index_fill", "compact_finish", "sweep", "heavy", "annihilate",
                "finish"]

_lock = threading.Lock()
_lib = None


def _declare(L):
    P = ctypes.POINTER
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    u64p, i32p, f64p = P(ctypes.c_uint64), P(ctypes.c_int32), P(ctypes.c_double)
    L.fciqmc_default_options.argtypes = [P(Options)]
    L.fciqmc_default_options.restype = None
    L.fciqmc_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, P(Options)]
    L.fciqmc_workspace_bytes.restype = ctypes.c_size_t
    L.fciqmc_create.argtypes = [f64p, f64p, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p,
                                ctypes.c_double, i32, P(Options), vp, ctypes.c_size_t, vp, P(vp)]
    L.fciqmc_step.argtypes = [vp, i32]
    L.fciqmc_sync.argtypes = [vp]
    L.fciqmc_estimators.argtypes = [vp, P(Estimates)]
    L.fciqmc_history.argtypes = [vp, P(Row), i64, P(i64)]
    L.fciqmc_n_dets.argtypes = [vp, P(i64)]
    L.fciqmc_get_walkers.argtypes = [vp, u64p, i32p, f64p, i64, P(i64)]
    L.fciqmc_set_walkers.argtypes = [vp, u64p, i32p, f64p, i64, P(State)]
    L.fciqmc_get_state.argtypes = [vp, P(State)]
    L.fciqmc_get_info.argtypes = [vp, P(Info)]
    L.fciqmc_profile.argtypes = [vp, i32, f64p]
    L.fciqmc_estimate_list_static.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, u64p, vp, vp, i64, i32, vp, vp]
    L.fciqmc_estimate_list_static.restype = ctypes.c_int
    L.fciqmc_rdm_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, i64]
    L.fciqmc_rdm_workspace_bytes.restype = ctypes.c_size_t
    L.fciqmc_rdm_create.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, i64, vp, ctypes.c_size_t, vp, P(vp)]
    L.fciqmc_rdm_energy.argtypes = [vp, vp, vp, vp]
    L.fciqmc_rdm_gradient.argtypes = [vp, vp, vp, vp]
    L.fciqmc_rdm_info.argtypes = [vp, P(i64)]
    L.fciqmc_rdm_destroy.argtypes = [vp]
    L.fciqmc_rdm_destroy.restype = None
    for name in ("fciqmc_rdm_create", "fciqmc_rdm_energy", "fciqmc_rdm_gradient", "fciqmc_rdm_info"):
        getattr(L, name).restype = ctypes.c_int
    L.fciqmc_batch_create.argtypes = [P(vp), ctypes.c_int, i32, P(vp)]
    L.fciqmc_batch_create.restype = ctypes.c_int
    L.fciqmc_batch_step.argtypes = [vp, i32, vp]
    L.fciqmc_batch_step.restype = ctypes.c_int
    L.fciqmc_batch_destroy.argtypes = [vp]
    L.fciqmc_batch_destroy.restype = None
    L.fciqmc_group_workspace_bytes.argtypes = [i32, i64]
    L.fciqmc_group_workspace_bytes.restype = ctypes.c_size_t
    L.fciqmc_group_create.argtypes = [P(vp), i32, i64, vp, ctypes.c_size_t, vp, P(vp)]
    L.fciqmc_group_step.argtypes = [vp, i32]
    L.fciqmc_group_sync.argtypes = [vp]
    L.fciqmc_group_history.argtypes = [vp, P(Row), i64, P(i64)]
    L.fciqmc_group_destroy.argtypes = [vp]
    L.fciqmc_group_destroy.restype = None
    L.fciqmc_owner.argtypes = [ctypes.c_int, u64p, i64, i32, i32p]
    for name in ("fciqmc_group_create", "fciqmc_group_step", "fciqmc_group_sync", "fciqmc_group_history",
                 "fciqmc_owner"):
        getattr(L, name).restype = ctypes.c_int
    L.fciqmc_rng_throughput.argtypes = [i64, vp, P(ctypes.c_double)]
    L.fciqmc_rng_throughput.restype = ctypes.c_int
    L.fciqmc_destroy.argtypes = [vp]
    L.fciqmc_destroy.restype = None
    L.fciqmc_strerror.argtypes = [ctypes.c_int]
    L.fciqmc_strerror.restype = ctypes.c_char_p
    for name in ("fciqmc_create", "fciqmc_step", "fciqmc_sync", "fciqmc_estimators", "fciqmc_history",
                 "fciqmc_n_dets", "fciqmc_get_walkers", "fciqmc_set_walkers", "fciqmc_get_state", "fciqmc_get_info",
                 "fciqmc_profile"):
        getattr(L, name).restype = ctypes.c_int


def load(build_if_needed: bool = True):
    """The loaded library; raises if it cannot be built or loaded."""
    global _lib
    with _lock:
        if _lib is None:
            path = build() if build_if_needed else LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libfciqmc.so not built ({path}); run __graft_entry__.build()")
            L = ctypes.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


class FciqmcError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        msg = load(False).fciqmc_strerror(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


def check(status: int, where: str = "") -> int:
    if status != 0:
        raise FciqmcError(status, where)
    return status
