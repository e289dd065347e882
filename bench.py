#!/usr/bin/env python
"""Benchmark of the FCIQMC walker cycle: spawn attempts/s and iterations/s at 1e8 walkers.

Workload (default "24e60o"): 24 electrons in 60 spatial orbitals (two uint64 words per
determinant), 8 irreps, synthetic decaying-Cholesky integrals with a near-degenerate frontier,
initiator threshold 3, tau = 0.001, 1e8 target walkers, main list of 2e8 slots. The walker
population is grown on the GPU from the reference at a moderate initial shift (untimed), the shift
starts varying at the target, the run settles for 4000 more iterations (the shift, N_w and N_d are
then flat to a few per mille per 500 iterations), and after warm-up iterations K iterations are
timed with CUDA events on the run's stream.
One "step" is one full iteration: spawning, death, annihilation with the initiator filter,
estimators and shift. The main list (GBs) is far larger than L2, so no L2 flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

N > 1 runs under torchrun: each rank advances an independent replica (its own seed), the
timed region is bracketed by barriers, the time is the maximum over ranks and the value is the
total number of attempts of all ranks divided by that time (weak scaling).
"""
from __future__ import annotations

import argparse
import csv
import ctypes
import io
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1305_6981_gb300 import synth  # noqa: E402

METRIC = "spawn attempts/s at 1e8 walkers (24e/60o, initiator, tau 0.001)"

# Instruction-issue roofline of the spawning kernels (they are bound by their instruction stream, not
# by HBM). Per-unit figures are warp instructions per attempt from ncu: smsp__inst_executed.sum of a launch
# divided by the attempts of that launch. Metrics collected at full size must be a one-pass set, checked on
# the medium case first (--ncu-case --target 5000000); multi-pass sets (--set full) stay on that medium case,
# one kernel and one launch. The commands are in the profile summary named in WARP_INST_SOURCE. The figures
# must be re-measured whenever those kernels change.
WARP_INST_PER_ATTEMPT = {"heavy": 12.53, "sweep": 27.10}
WARP_INST_SOURCE = "profiles/counters_24e60o_steady.txt (full size, steady state, one-pass capture)"
# DRAM bytes (read + write) per launch at the full workload, from the same capture.
DRAM_BYTES_PER_LAUNCH = {"heavy": 35_700_000, "sweep": 562_900_000, "annihilate": 87_700_000}
ISSUE_PER_CLK_PER_SM = 4  # warp instructions: 4 schedulers per SM, one issue each per clock
N_SMS = 152

WORKLOADS = {
    "24e60o": dict(system=synth.large_24e60o, tau=0.001, thr=3, target=100_000_000, main_capacity=200_000_000,
                   spawn_capacity=1 << 27, initial_population=20_000, initial_shift=0.5, max_growth=40_000,
                   equilibrate=4000,
                   desc="24e/60o (W=2), 8 irreps, initiator 3, tau 0.001, 1e8 target walkers, 2e8-slot main list, "
                        "timed at steady state (grown at shift 0.5, 4000 iterations after the shift starts varying)"),
    "24e60o-cas": dict(system=synth.large_24e60o, tau=0.001, thr=3, target=100_000_000, main_capacity=200_000_000,
                       spawn_capacity=1 << 27, initial_population=20_000, initial_shift=0.5, max_growth=40_000,
                       equilibrate=4000,
                       space=dict(frozen_occupied=[(1 << 8) - 1, 0], frozen_empty=[0, ((1 << 32) - 1) << 24]),
                       desc="24e/60o active space CAS(16e,40o): spatial orbitals 0..3 frozen doubly occupied, "
                            "44..59 deleted (Sec. VI null excitations), initiator 3, tau 0.001, 1e8 target walkers"),
    "24e60o-hphf": dict(system=synth.large_24e60o, tau=0.002, thr=3, target=50_000_000, main_capacity=100_000_000,
                        spawn_capacity=1 << 26, initial_population=20_000, initial_shift=0.5, max_growth=40_000,
                        equilibrate=2000, space=dict(hphf=True),
                        desc="24e/60o on spin-coupled functions (Sec. VI C: half the space, so half the walkers "
                             "and twice the time step of the determinant run), initiator 3, tau 0.002, "
                             "5e7 target walkers"),
    "24e60o-real": dict(system=synth.large_24e60o, tau=0.001, thr=3, target=100_000_000, main_capacity=200_000_000,
                        spawn_capacity=1 << 27, initial_population=20_000, initial_shift=0.5, max_growth=40_000,
                        equilibrate=4000, space=dict(walker_fraction_bits=4, occupation_threshold=1.0),
                        desc="24e/60o with real/integer hybrid walkers (populations in units of 1/16 walker, "
                             "occupation threshold 1 walker), initiator 3, tau 0.001, 1e8 target walkers, steady state"),
    "24e60o-part4": dict(system=synth.large_24e60o, tau=0.001, thr=3, target=100_000_000, main_capacity=75_000_000,
                         spawn_capacity=1 << 25, initial_population=20_000, initial_shift=0.5, max_growth=40_000,
                         equilibrate=4000, partitions=4, outbox_capacity=1 << 20,
                         desc="24e/60o divided among 4 hash partitions on one GPU (Sec. V A: owner = Algorithm 1 "
                              "fingerprint mod 4, spawns routed through per-destination outboxes), initiator 3, "
                              "tau 0.001, 1e8 target walkers, steady state; beside it the unpartitioned run from "
                              "the same list"),
    "12e24o": dict(system=synth.init_12e24o, tau=0.005, thr=3, target=1_000_000, main_capacity=4_000_000,
                   spawn_capacity=1 << 22, initial_population=2_000, initial_shift=1.0, max_growth=20_000,
                   equilibrate=50, desc="12e/24o (W=1), 8 irreps, initiator 3, tau 0.005, 1e6 target walkers"),
    "batch64": dict(system=None, tau=0.005, thr=3, target=0, main_capacity=0, spawn_capacity=0, initial_population=0,
                    initial_shift=1.0, max_growth=6000, equilibrate=20,
                    desc="64 independent runs, 8e/16o..16e/40o (seeded), targets log-uniform 1e4..2e6, tau 0.005, "
                         "initiator 3, one CUDA graph per launch vs the same runs advanced one at a time"),
    "energy16e40o": dict(system=synth.rdm_16e40o, tau=0.0, thr=-1, target=0, main_capacity=0, spawn_capacity=0,
                         initial_population=0, initial_shift=0.0, max_growth=0, equilibrate=0,
                         desc="energy functional and density matrices over 1e6 sampled determinants of 16e/40o "
                              "(--target overrides the number of determinants)"),
    "8e8o": dict(system=synth.tiny_8e8o, tau=0.01, thr=-1, target=1 << 14, main_capacity=1 << 14,
                 spawn_capacity=1 << 14, initial_population=1_000, initial_shift=0.5, max_growth=5_000,
                 equilibrate=50, desc="8e/8o (W=1), no symmetry, plain FCIQMC, tau 0.01, 2^14 target walkers"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="24e60o", choices=sorted(WORKLOADS))
    ap.add_argument("--target", type=int, default=0, help="override target walkers (smaller runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--growth-log", default="")
    ap.add_argument("--save-state", default="",
                    help="after growth and settling, save the walker list and run state to this .npz file")
    ap.add_argument("--load-state", default="",
                    help="start from a list saved by --save-state instead of growing (few launches before the "
                         "timed region, for profiler captures)")
    ap.add_argument("--settle", type=int, default=-1,
                    help="iterations after the shift starts varying before warm-up (default: the workload's)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-runs and energy-functional measurements appended to the default line")
    ap.add_argument("--ncu-case", action="store_true",
                    help="grow to --target walkers, run one iteration inside the NVTX range 'prof' and exit "
                         "(the case the ncu summaries are taken on)")
    return ap.parse_args()


# ---------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi samples during the timed region (clocks, power, throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for r in csv.reader(f):
                if len(r) >= 9:
                    rows.append([x.strip() for x in r])
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# ---------------------------------------------------------------------------- oracle baseline
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample(wl, system):
    """The bounded sample that both the CPU baseline of the GPU arm and the reference arm time: a synthetic
    snapshot of the workload (2e5 walkers for the 24e/60o workloads, 5e4 otherwise; the reference holds 5%,
    the rest sit on random 1..4-fold excitations), restricted to the permitted space."""
    from oracle.oracle import Oracle, lib
    lib()
    n = 200_000 if wl["desc"].startswith("24e/60o") else 50_000
    dets, pops = synth.walker_snapshot(system, n, seed=7)
    q = Oracle(system, tau=wl["tau"], initiator_threshold=wl["thr"], seed=1, **wl.get("space", {}))
    if wl.get("space", {}).get("hphf"):
        dets, pops = synth.stored_pairs(dets, pops)
    keep = np.array([q.in_space(d) for d in dets])
    bits = wl.get("space", {}).get("walker_fraction_bits", 0)
    return q, dets[keep], (pops[keep].astype(np.int64) << bits).astype(np.int32)  # hybrid walkers: units


def oracle_baseline(wl, system, steps: int, warmup: int, one_thread_steps: int = 2):
    """The CPU oracle as it stands, timed on this host on the bounded sample of oracle_sample: whole
    iterations (spawning, death, merge, annihilation, estimators) restarted from the sample each time, on
    all cores and on one thread. Returns a dict with both rates, the cores used and the CPU model."""
    from oracle import oracle as O
    q, dets, pops = oracle_sample(wl, system)
    cores = O.set_threads(os.cpu_count() or 1)

    def timed(n_steps, first_iter):
        att, tsum = 0, 0.0
        for k in range(n_steps):
            q.set_walkers(dets, pops, iteration=first_iter + k, shift=0.0)
            t0 = time.perf_counter()
            rows = q.iterate(1)
            tsum += time.perf_counter() - t0
            att += rows[0]["attempts"]
        return att, tsum

    timed(warmup, 0)
    att, tsum = timed(steps, warmup)
    O.set_threads(1)
    att1, tsum1 = timed(one_thread_steps, warmup + steps)
    O.set_threads(cores)
    return {"value": att / tsum, "unit": "attempts/s", "cores": cores, "kind": "oracle",
            "one_thread": att1 / tsum1, "cpu_model": cpu_model(), "ms_per_step": 1e3 * tsum / max(steps, 1),
            "sample": f"{steps} oracle iterations on all {cores} cores (and {one_thread_steps} on one thread) of a "
                      f"synthetic snapshot of the workload: {len(pops)} determinants / {int(np.abs(pops).sum())} "
                      f"walkers (reference 5%, random 1..4-fold excitations); the same sample as the reference arm"}


# ---------------------------------------------------------------------------- reference arm
def _reference_line(args, metric, value, unit, higher, config, sample):
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"impl": "reference", "metric": metric, "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": higher, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference_batch(args, wl):
    """The oracle over the 64 uneven runs, one after another, each on a synthetic snapshot of its target
    population capped at 2e4 walkers: aggregate attempts/s."""
    from oracle.oracle import Oracle, lib
    lib()
    specs = synth.batch_systems(64, seed=3)
    runs = []
    for k, sp in enumerate(specs):
        system = synth.make_system(sp["n_orb"], sp["n_elec"], seed=sp["sys_seed"] % 100000, n_chol=sp["n_orb"] // 2,
                                   name=f"run{k}")
        dets, pops = synth.walker_snapshot(system, min(int(sp["target"]), 20_000), seed=7)
        runs.append((Oracle(system, tau=wl["tau"], initiator_threshold=wl["thr"], seed=sp["seed"]), dets, pops))
    att, tsum = 0, 0.0
    for k in range(args.warmup + args.steps):
        for q, dets, pops in runs:
            q.set_walkers(dets, pops, iteration=k, shift=0.0)
            t0 = time.perf_counter()
            rows = q.iterate(1)
            if k >= args.warmup:
                tsum += time.perf_counter() - t0
                att += rows[0]["attempts"]
    value = att / tsum
    walkers = sum(int(np.abs(p).sum()) for _, _, p in runs)
    out = _reference_line(args, "aggregate spawn attempts/s, 64 uneven independent runs (one graph per launch)",
                          value, "attempts/s", True, {"workload": "batch64", "system": wl["desc"]},
                          f"{args.steps} iterations of each of the 64 runs on snapshots of at most 2e4 walkers "
                          f"({walkers} walkers in total)")
    out["ms_per_step"] = 1e3 * tsum / max(args.steps, 1)
    return out


ENERGY_METRIC = ("energy functional forward + first backward: connected determinant pairs per second "
                 "(16e/40o sampled vector)")


def connected_pairs(dets) -> int:
    """Unordered pairs of distinct determinants that differ by a single or a double excitation (the pairs
    whose matrix elements and density-matrix terms the energy functional evaluates)."""
    def popcount(x):  # 64-bit population count, lane-parallel on uint64 arrays
        x = x - ((x >> np.uint64(1)) & np.uint64(0x5555555555555555))
        x = (x & np.uint64(0x3333333333333333)) + ((x >> np.uint64(2)) & np.uint64(0x3333333333333333))
        x = (x + (x >> np.uint64(4))) & np.uint64(0x0F0F0F0F0F0F0F0F)
        return ((x * np.uint64(0x0101010101010101)) >> np.uint64(56)).astype(np.int64)

    d = np.ascontiguousarray(dets, dtype=np.uint64).reshape(len(dets), -1)
    n = 0
    for i in range(len(d) - 1):
        x = d[i + 1:] ^ d[i]
        c = sum(popcount(x[:, w]) for w in range(d.shape[1]))
        n += int(((c == 2) | (c == 4)).sum())
    return n


def run_reference_energy(args, wl):
    """The oracle's energy functional and density matrices (one call gives both) on a 5000-determinant
    sample of the 16e/40o vector, in connected determinant pairs per second like the GPU arm (at most three
    timed calls: the oracle's pair search is quadratic in the determinants)."""
    from oracle.oracle import Oracle, lib
    lib()
    n = 5_000
    s = wl["system"]()
    dets, c = synth.sampled_vector(s, n, seed=5)
    q = Oracle(s, tau=0.01)
    for _ in range(min(args.warmup, 1)):
        q.rdm_energy(dets, c)
    calls = min(max(args.steps, 1), 3)
    t0 = time.perf_counter()
    for _ in range(calls):
        q.rdm_energy(dets, c)
    sec = (time.perf_counter() - t0) / calls
    pairs = connected_pairs(dets)
    out = _reference_line(args, ENERGY_METRIC, pairs / sec, "pairs/s", True,
                          {"workload": "energy16e40o", "n_dets": n, "connected_pairs": pairs},
                          f"{n} of the sampled determinants (the GPU arm uses 1e6); {pairs} connected pairs")
    out["ms_per_step"] = 1e3 * sec
    return out


def run_reference(args, wl, rank, world):
    if rank != 0:
        return
    if args.workload == "batch64":
        print(json.dumps(run_reference_batch(args, wl)), flush=True)
        return
    if args.workload == "energy16e40o":
        print(json.dumps(run_reference_energy(args, wl)), flush=True)
        return
    system = wl["system"]()
    b = oracle_baseline(wl, system, max(args.steps, 1), args.warmup)
    out = _reference_line(args, METRIC, b["value"], "attempts/s", True,
                          {"workload": args.workload, "system": wl["desc"], "sample": b["sample"]}, b["sample"])
    out["ms_per_step"] = b["ms_per_step"]
    out["cpu_baseline"].update({"cores": b["cores"], "one_thread": b["one_thread"], "cpu_model": b["cpu_model"]})
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------- GPU arm
def algorithmic_bytes(W, nd, slots, merged, inserted):
    """HBM bytes one iteration must move: per occupied determinant its words, population
    and float diagonal read plus the new population written; per vacated slot its population read and
    written; per distinct spawned determinant the merge entry written and read back with its position,
    one index entry and one population read-modify-write; per insertion the new slot and index entry."""
    entry = 8 * W + 8
    sweep = nd * (8 * W + 4 + 4 + 4) + (slots - nd) * 8 + merged * (entry + 4)
    annih = merged * (entry + 4) + merged * (entry + 8) + inserted * (8 * W + 8 + 4 + 4 + entry)
    return sweep, annih


def replica_seed(rank: int) -> int:
    """Random-number seed of the replica on a rank (independent replicas, one per GPU)."""
    return 1 + rank


def reduce_over_ranks(ms: float, attempts: float, world: int, device) -> tuple[float, float]:
    """The timed region's length (the maximum over ranks) and the attempts of all ranks (their sum)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    a = torch.tensor([attempts], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(a, op=dist.ReduceOp.SUM)
    return float(t.item()), float(a.item())


def grow(args, wl, rank):
    """Create the run and grow the population on the GPU until the shift starts varying (untimed)."""
    from paper_1305_6981_gb300 import Fciqmc

    system = wl["system"]()
    target = args.target or wl["target"]
    cap = wl["main_capacity"] if not args.target else max(2 * args.target, 1 << 16)
    scap = wl["spawn_capacity"] if not args.target else max(1 << 14, 1 << int(np.ceil(np.log2(args.target))))
    g = Fciqmc(system, wl["tau"], wl["thr"], target_walkers=target, initial_population=wl["initial_population"],
               initial_shift=wl["initial_shift"], seed=replica_seed(rank), main_capacity=cap, spawn_capacity=scap,
               **wl.get("space", {}))
    t_grow = time.perf_counter()
    grown, chunk = 0, 50
    log = []
    if getattr(args, "load_state", ""):
        z = np.load(args.load_state)
        st = {k: z["state"][i] for i, k in enumerate(("iteration", "shift", "vary_shift", "shift_counter",
                                                       "nw_last_update"))}
        g.set_walkers(z["dets"], z["pops"], z["hdiag"], iteration=int(st["iteration"]), shift=float(st["shift"]),
                      vary=int(st["vary_shift"]), shift_counter=int(st["shift_counter"]),
                      nw_last_update=int(st["nw_last_update"]))
        return g, int(st["iteration"]), time.perf_counter() - t_grow, log
    while True:
        g.step(chunk)
        grown += chunk
        e = g.estimates()
        log.append((grown, e["n_walkers"], e["n_dets"], e["shift"], e["list_slots"]))
        if e["status"] != 0:
            raise RuntimeError(f"device status {e['status']} during growth at {grown}: {log[-1]}")
        if e["vary_shift"] or grown >= wl["max_growth"]:
            break
    settle = wl["equilibrate"] if getattr(args, "settle", -1) < 0 else args.settle
    while settle > 0:  # settle towards the steady state of the varying shift
        k = min(settle, 500)
        g.step(k)
        settle -= k
        grown += k
        e = g.estimates()
        log.append((grown, e["n_walkers"], e["n_dets"], e["shift"], e["list_slots"]))
        if e["status"] != 0:
            raise RuntimeError(f"device status {e['status']} while settling at {grown}: {log[-1]}")
    if getattr(args, "save_state", ""):
        d, p, hd = g.walkers()
        st = g.state()
        np.savez(args.save_state, dets=d, pops=p, hdiag=hd,
                 state=np.array([st["iteration"], st["shift"], st["vary_shift"], st["shift_counter"],
                                 st["nw_last_update"]], dtype=np.float64))
    return g, grown, time.perf_counter() - t_grow, log


def run_ncu_case(args, wl):
    import torch
    torch.cuda.set_device(0)
    g, grown, _, _ = grow(args, wl, 0)
    g.sync()
    torch.cuda.nvtx.range_push("prof")
    g.step(1)
    torch.cuda.nvtx.range_pop()
    st = g.sync()
    row = g.history(1)[0]
    info = g.info()
    print(json.dumps({"ncu_case": args.workload, "target": args.target or wl["target"], "grown": grown, "status": st,
                      "workspace_gb": info["workspace_bytes"] / 1e9, "row": row}), flush=True)
    g.close()


def run_gpu(args, wl, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    g, grown, t_grow, log = grow(args, wl, rank)
    info = g.info()
    if args.growth_log and rank == 0:
        with open(args.growth_log, "w") as f:
            json.dump(log, f)
    # warm-up
    g.step(args.warmup)
    g.sync()
    stream = g.stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local_rank)
    e_before = g.estimates()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    g.step(args.steps)
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    st = g.sync()
    rows = g.history(args.steps)
    # the rate no attempt stream can exceed: one Philox4x32-10 block per attempt (measured after the window)
    from paper_1305_6981_gb300 import rng_throughput
    rng_rate = rng_throughput(1 << 31, g.stream)
    attempts = sum(r["attempts"] for r in rows)
    nd_mean = float(np.mean([r["nd_in"] for r in rows]))
    nw_mean = float(np.mean([r["nw_in"] for r in rows]))
    merged_mean = float(np.mean([r["merged_entries"] for r in rows]))
    inserted_mean = float(np.mean([r["inserted_dets"] for r in rows]))
    ms_max, att_all = reduce_over_ranks(ms, float(attempts), world, "cuda")
    # per-kernel times (same iterations, kernels launched one by one between events)
    est = g.estimates()
    exact = {"spawn_per_iter": (est["exact_spawns"] - e_before["exact_spawns"]) / args.steps,
             "death_per_iter": (est["exact_deaths"] - e_before["exact_deaths"]) / args.steps}
    prof = g.profile(5)
    prow = g.history(5)
    slots = est["list_slots"]
    sweep_b, annih_b = algorithmic_bytes(info["words"], nd_mean, slots, merged_mean, inserted_mean)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    # dominant kernel and its instruction-issue roofline
    heavy_att = float(np.mean([r["heavy_attempts"] for r in prow]))
    light_att = float(np.mean([r["attempts"] - r["heavy_attempts"] for r in prow]))
    units = {"heavy": heavy_att, "sweep": light_att}
    dom = max(("sweep", "heavy"), key=lambda k: prof[k])
    dom_ms = prof[dom] / 5.0
    sm_mhz = clk.get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    issue_peak = ISSUE_PER_CLK_PER_SM * N_SMS * sm_mhz * 1e6 / 1e9  # Gwarp-inst/s
    achieved = WARP_INST_PER_ATTEMPT[dom] * units[dom] / (dom_ms * 1e-3) / 1e9
    cycle_gbs = (sweep_b + annih_b) / (ms_max / args.steps * 1e-3) / 1e9
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": att_all / (ms_max * 1e-3), "unit": "attempts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "iterations_per_s": args.steps / (ms_max * 1e-3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "system": wl["desc"], "walkers_mean": nw_mean,
                       "dets_mean": nd_mean, "list_slots": slots, "merged_per_iter": merged_mean,
                       "inserted_per_iter": inserted_mean, "growth_iterations": grown,
                       "growth_seconds": round(t_grow, 1), "l2": "inputs larger than L2 (main list ~GBs)",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "steady_state": {"shift_at_timing": rows[0]["shift"] if rows else None,
                                        "shift_at_end": rows[-1]["shift"] if rows else None,
                                        "nw_first": rows[0]["nw_in"] if rows else None,
                                        "nw_last": rows[-1]["nw_out"] if rows else None,
                                        "nw_drift": (rows[-1]["nw_out"] / rows[0]["nw_in"] - 1.0) if rows else None,
                                        "dets_first": rows[0]["nd_in"] if rows else None,
                                        "heavy_share": (sum(r["heavy_attempts"] for r in rows)
                                                        / max(1, sum(r["attempts"] for r in rows))),
                                        "c0_first": rows[0]["c0_in"] if rows else None}},
            # the per-unit instruction counts were measured on the default workload's kernels
            "roofline": ({"bound": "alu", "kernel": f"k_{dom}", "achieved": achieved, "peak": issue_peak,
                          "unit": "Gwarp-inst/s", "frac": achieved / issue_peak,
                          "traffic": DRAM_BYTES_PER_LAUNCH.get(dom),
                          "per_unit": f"{WARP_INST_PER_ATTEMPT[dom]} warp instructions per attempt (ncu, "
                                      f"{WARP_INST_SOURCE})",
                          "units_per_launch": units[dom], "launch_ms": dom_ms,
                          "peak_derivation": f"{ISSUE_PER_CLK_PER_SM} warp-inst/clk/SM x {N_SMS} SMs x "
                                             f"{sm_mhz:.0f} MHz"}
                         if args.workload == "24e60o" and not args.target else None),
            "hbm": {"cycle_algorithmic_gbs": cycle_gbs, "peak": hbm_peak, "frac": cycle_gbs / hbm_peak,
                    "peak_source": peak_src, "bytes_per_iter": sweep_b + annih_b},
            # attempts/s against the Philox4x32-10 rate measured live on this GPU (one block per attempt)
            "alu_floor": {"philox_blocks_per_s": rng_rate, "attempts_per_s": att_all / (ms_max * 1e-3),
                          "frac": att_all / (ms_max * 1e-3) / rng_rate / world},
            "kernel_ms_per_iter": {k: v / 5.0 for k, v in prof.items()},
            "clocks": clk,
            "status": st,
            "exact_path": exact,
            # per iteration: 6 compaction kernels, sweep, tile sums, heavy, annihilate, new-slot diagonal
            # elements, finish (and the occupation threshold with hybrid walkers)
            "gpu_launches": (12 + (1 if wl.get("space", {}).get("walker_fraction_bits") else 0)) * args.steps,
        }
    return g, out, info


def run_partitioned(args, wl):
    """The workload divided among hash partitions on one GPU (fciqmc_group_*): grown and settled as the
    default workload, then K timed iterations of the group; beside it, an unpartitioned run loaded with the
    same list and state and timed over the same number of iterations (the cost of the decomposition)."""
    import torch

    from paper_1305_6981_gb300 import Fciqmc, Partitioned

    torch.cuda.set_device(0)
    system = wl["system"]()
    n_parts = wl["partitions"]
    target = args.target or wl["target"]
    g = Partitioned(system, wl["tau"], wl["thr"], n_partitions=n_parts, target_walkers=target,
                    initial_population=wl["initial_population"], initial_shift=wl["initial_shift"], seed=1,
                    main_capacity=wl["main_capacity"], spawn_capacity=wl["spawn_capacity"],
                    outbox_capacity=wl["outbox_capacity"])
    t_grow = time.perf_counter()
    grown = 0
    while grown < wl["max_growth"]:
        g.step(50)
        grown += 50
        e = g.estimates()
        if e["status"] != 0:
            raise RuntimeError(f"device status {e['status']} during growth at {grown}")
        if e["vary_shift"]:
            break
    settle = wl["equilibrate"] if args.settle < 0 else args.settle
    g.step(settle)
    grown += settle
    g.step(args.warmup)
    g.sync()
    t_grow = time.perf_counter() - t_grow

    def timed(run, stream):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        run.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1)

    d, p, hd = g.walkers()
    st = g.parts[0].state()
    clocks = Clocks(0)
    clocks.start()
    time.sleep(0.3)
    ms = timed(g, g.stream)
    clk = clocks.stop()
    status = g.sync()
    rows = g.history(args.steps)
    att = sum(r["attempts"] for r in rows)
    per_part = [len(x.walkers()[1]) for x in g.parts]
    g.close()
    # the same list, unpartitioned
    u = Fciqmc(system, wl["tau"], wl["thr"], target_walkers=target, seed=1, main_capacity=2 * len(p) + (1 << 20),
               spawn_capacity=wl["spawn_capacity"] * n_parts)
    u.set_walkers(d, p, hd, iteration=st["iteration"], shift=st["shift"], vary=st["vary_shift"],
                  shift_counter=st["shift_counter"], nw_last_update=st["nw_last_update"])
    u.step(args.warmup)
    ms_u = timed(u, u.stream)
    rows_u = u.history(args.steps)
    att_u = sum(r["attempts"] for r in rows_u)
    u.close()
    return {"metric": METRIC, "value": att / (ms * 1e-3), "unit": "attempts/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "system": wl["desc"], "partitions": n_parts,
                       "walkers_mean": float(np.mean([r["nw_in"] for r in rows])), "dets": int(len(p)),
                       "dets_per_partition": per_part, "growth_iterations": grown,
                       "growth_seconds": round(t_grow, 1), "parallelism": f"{n_parts} partitions on 1 GPU"},
            "unpartitioned_same_state": {"value": att_u / (ms_u * 1e-3), "unit": "attempts/s",
                                         "ms_per_step": ms_u / args.steps},
            "partition_cost": (ms / args.steps) / (ms_u / args.steps),
            "clocks": clk, "status": status, "gpu_launches": (12 * n_parts + 1) * args.steps}


def run_batch(args, wl):
    """Aggregate spawn attempts/s of 64 uneven runs advanced by one graph per launch, against the same
    runs advanced one at a time (each with its own graph launches on its own stream, in sequence)."""
    import torch

    from paper_1305_6981_gb300 import Batch, Fciqmc
    from paper_1305_6981_gb300.autotune import bucket_of, tune_buckets

    torch.cuda.set_device(0)
    specs = synth.batch_systems(64, seed=3)
    systems = [synth.make_system(sp["n_orb"], sp["n_elec"], seed=sp["sys_seed"] % 100000, n_chol=sp["n_orb"] // 2,
                                 name=f"run{k}") for k, sp in enumerate(specs)]
    targets = np.array([sp["target"] for sp in specs])
    # autotune one representative per size bucket (one octave of target walkers): block count, index load factor
    # and spawn-table size; every run takes its bucket's choice, scaled to its own target
    t_tune = time.perf_counter()
    per_run, tuned = tune_buckets(systems, [int(t) for t in targets], wl["tau"], wl["thr"], trial_iterations=10)
    t_tune = time.perf_counter() - t_tune

    def make(k):
        rep_target = int(targets[tuned[bucket_of(int(targets[k]))]["representative"]])
        o = dict(per_run[k])
        o["main_capacity"] = max(4 * int(targets[k]), 1 << 14)
        o["spawn_capacity"] = max(1 << 12, int(o["spawn_capacity"] * targets[k] / rep_target))
        return Fciqmc(systems[k], wl["tau"], wl["thr"], target_walkers=int(targets[k]),
                      initial_population=max(100, int(targets[k]) // 100), initial_shift=wl["initial_shift"],
                      seed=specs[k]["seed"], **o)

    runs = [make(k) for k in range(64)]
    L = 10
    batch = Batch(runs, iterations_per_launch=L)
    t_grow = time.perf_counter()
    grown = 0
    while grown < wl["max_growth"]:
        batch.step(5)
        grown += 5 * L
        if all(r.estimates()["vary_shift"] for r in runs):
            break
    batch.step(max(1, wl["equilibrate"] // L))
    t_grow = time.perf_counter() - t_grow
    torch.cuda.synchronize()
    K = max(1, args.steps)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    batch.step(max(1, args.warmup))
    torch.cuda.synchronize()
    ev0.record(stream)
    batch.step(K)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_batch = ev0.elapsed_time(ev1)
    att_batch = sum(sum(r2["attempts"] for r2 in r.history(K * L)) for r in runs)
    # the same runs, one at a time
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in runs:
        r.step(K * L)
        r.sync()
    ms_seq = (time.perf_counter() - t0) * 1e3
    att_seq = sum(sum(r2["attempts"] for r2 in r.history(K * L)) for r in runs)
    status = max(abs(r.sync()) for r in runs)
    out = {
        "metric": "aggregate spawn attempts/s, 64 uneven independent runs (one graph per launch)",
        "value": att_batch / (ms_batch * 1e-3), "unit": "attempts/s", "n_gpus": 1, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_batch / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batch64", "system": wl["desc"], "iterations_per_launch": L,
                   "walkers_total": int(sum(r.estimates()["n_walkers"] for r in runs)),
                   "growth_iterations": grown, "growth_seconds": round(t_grow, 1), "tune_seconds": round(t_tune, 1),
                   "tuned": {f"2^{b}..2^{b + 1} walkers ({r['members']} runs)":
                             dict(r["best"], ms_per_iteration=r["ms_per_iteration"]) for b, r in tuned.items()}},
        "sequential": {"value": att_seq / (ms_seq * 1e-3), "unit": "attempts/s", "ms_total": ms_seq},
        "speedup_vs_sequential": (att_batch / ms_batch) / (att_seq / ms_seq),
        "status": status,
    }
    batch.close()
    for r in runs:
        r.close()
    return out


def energy_functional_timing(n_dets: int = 1_000_000):
    """Forward and backward of E(h, V; c) on the 16e/40o sampled vector: pair construction, one forward,
    the first backward (density matrices), one more forward."""
    import torch

    from paper_1305_6981_gb300 import EnergyFunctional

    s = synth.rdm_16e40o()
    dets, c = synth.sampled_vector(s, n_dets, seed=5)
    h = torch.as_tensor(s.h).cuda()
    v = torch.as_tensor(s.eri_s8).cuda()
    one = torch.ones((), dtype=torch.float64, device="cuda")
    # warm-up on a small vector (module loading, allocator), outside the timed calls
    wd, wc = synth.sampled_vector(s, 2000, seed=6)
    w = EnergyFunctional(s.n_elec, s.n_orb, wd, wc)
    w.energy(h, v)
    w.gradient(one)
    w.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f = EnergyFunctional(s.n_elec, s.n_orb, dets, c)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.nvtx.range_push("timed")
    ev[0].record()
    E = f.energy(h, v)
    ev[1].record()
    gh, ge = f.gradient(one)
    ev[2].record()
    f.energy(h, v)
    ev[3].record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    info = f.info()
    out = {"n_dets": n_dets, "system": "16e/40o (W=2), amplitudes exp(-level), levels 1..6",
           "energy": float(E), "create_ms": 1e3 * t_create, "forward_ms": ev[0].elapsed_time(ev[1]),
           "backward_first_ms": ev[1].elapsed_time(ev[2]), "forward_again_ms": ev[2].elapsed_time(ev[3]),
           **info}
    f.close()
    return out


def e2e_rate(g, args, info, world):
    """Same metric through the C ABI with host buffers: per step the walker list (determinants,
    populations, diagonal elements) goes host->device from pinned memory, one iteration runs, and the
    resulting list comes back device->host into pinned memory."""
    import torch
    n0 = g.estimates()["n_dets"]
    cap = int(n0 * 1.5) + 1024
    W = info["words"]
    dets = torch.empty((cap, W), dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    pops = torch.empty(cap, dtype=torch.int32, pin_memory=True).numpy()
    hd = torch.empty(cap, dtype=torch.float64, pin_memory=True).numpy()
    n = g.walkers_into(dets, pops, hd)
    st = g.state()
    K = max(1, min(args.steps, 10))
    h2d = d2h = 0
    att = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(K):
        g.set_walkers(dets[:n], pops[:n], hd[:n], iteration=st["iteration"] + k, shift=st["shift"],
                      vary=st["vary_shift"], shift_counter=st["shift_counter"], nw_last_update=st["nw_last_update"])
        h2d += n * (8 * W + 4 + 8)
        g.step(1)
        att += g.history(1)[0]["attempts"]
        n = g.walkers_into(dets, pops, hd)
        d2h += n * (8 * W + 4 + 8)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": att / dt, "unit": "attempts/s", "h2d_bytes_per_step": h2d // K, "d2h_bytes_per_step": d2h // K,
            "steps": K}, dets[:n].copy(), pops[:n].copy()


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return
    if args.ncu_case:
        run_ncu_case(args, wl)
        return
    if args.workload == "energy16e40o":
        import torch
        torch.cuda.set_device(0)
        r = energy_functional_timing(args.target or 1_000_000)
        pairs = r["single_pairs"] + r["double_pairs"]
        ms = r["forward_ms"] + r["backward_first_ms"]
        print(json.dumps({"metric": ENERGY_METRIC, "value": pairs / (ms * 1e-3), "unit": "pairs/s", "n_gpus": 1,
                          "steps": 1, "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "energy16e40o", "n_dets": r["n_dets"], "connected_pairs": pairs},
                          "detail": r}), flush=True)
        return
    if args.workload == "batch64":
        print(json.dumps(run_batch(args, wl)), flush=True)
        return
    if wl.get("partitions"):
        print(json.dumps(run_partitioned(args, wl)), flush=True)
        return
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    g, out, info = run_gpu(args, wl, rank, world, local_rank)
    if rank == 0:
        if not args.no_e2e and world == 1:
            e2e, dets, pops = e2e_rate(g, args, info, world)
            out["e2e"] = e2e
        else:
            dets, pops, _ = g.walkers()
            out["e2e"] = None
        if not args.no_cpu_baseline and world == 1:
            b = oracle_baseline(wl, wl["system"](), 20, 3)
            b.pop("ms_per_step")
            out["cpu_baseline"] = b
        if not args.no_extras and world == 1 and args.workload == "24e60o":
            g.close()
            bargs = argparse.Namespace(**vars(args))
            bargs.steps, bargs.warmup = 5, 1
            b = run_batch(bargs, WORKLOADS["batch64"])
            out["batched_64_runs"] = {k: b[k] for k in ("value", "unit", "sequential", "speedup_vs_sequential",
                                                         "ms_per_step", "status")}
            out["batched_64_runs"]["walkers_total"] = b["config"]["walkers_total"]
            out["batched_64_runs"]["tuned"] = b["config"]["tuned"]
            out["batched_64_runs"]["tune_seconds"] = b["config"]["tune_seconds"]
            out["energy_functional"] = energy_functional_timing()
        print(json.dumps(out), flush=True)
    if getattr(g, "handle", None):
        g.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
