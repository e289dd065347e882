"""Autotuner for the launch shape of a run: the number of blocks of the spawning and annihilation
kernels, the load factor of the determinant hash index and the size of the spawn merge table.

None of these changes a run's results (the random numbers are keyed by determinant, attempt and
iteration), so the tuner simply times short trials: it grows one run to its target walker number,
takes a snapshot, and for every candidate restarts from the snapshot and times a fixed number of
iterations with CUDA events. The fastest candidate is kept, and cached in a JSON file keyed by the
problem shape so that later runs of the same shape skip the trials."""
from __future__ import annotations

import itertools
import json
import os
import time

import numpy as np

from .fciqmc import Fciqmc

DEFAULT_CANDIDATES = {
    "grid_blocks": [0, 38, 152],
    "index_load": [0.25, 0.5, 0.75],
    "spawn_factor": [0.25, 0.5, 1.0],
}


def _key(system, tau, thr, target) -> str:
    return f"{system.n_elec}e{system.n_orb}o_t{tau}_i{thr}_w{int(round(np.log2(max(target, 2))))}"


def tune(system, tau: float, thr: int, target: int, *, trial_iterations: int = 20, grow_limit: int = 20000,
         candidates: dict | None = None, cache_path: str | None = None, seed: int = 1) -> dict:
    """Returns the fastest options (grid_blocks, index_load, spawn_capacity, main_capacity) and the timings."""
    import torch

    key = _key(system, tau, thr, target)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    cands = candidates or DEFAULT_CANDIDATES
    cap = max(4 * target, 1 << 14)
    base = Fciqmc(system, tau, thr, target_walkers=target, initial_population=max(100, target // 100),
                  initial_shift=1.0, seed=seed, main_capacity=cap, spawn_capacity=max(1 << 12, target // 2))
    grown = 0
    while grown < grow_limit:
        base.step(50)
        grown += 50
        if base.estimates()["vary_shift"]:
            break
    base.step(20)
    dets, pops, hd = base.walkers()
    st = base.state()
    base.close()
    trials = []
    for gb, load, sf in itertools.product(cands["grid_blocks"], cands["index_load"], cands["spawn_factor"]):
        opts = dict(grid_blocks=int(gb), index_load=float(load), main_capacity=cap,
                    spawn_capacity=int(max(1 << 12, sf * target)))
        run = Fciqmc(system, tau, thr, target_walkers=target, seed=seed, **opts)
        run.set_walkers(dets, pops, hd, iteration=st["iteration"], shift=st["shift"], vary=st["vary_shift"],
                        shift_counter=st["shift_counter"], nw_last_update=st["nw_last_update"])
        run.step(3)
        run.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(run.stream)
        run.step(trial_iterations)
        ev1.record(run.stream)
        status = run.sync()
        ms = ev0.elapsed_time(ev1) / trial_iterations
        trials.append(dict(options=opts, ms_per_iteration=ms, status=status))
        run.close()
    ok = [t for t in trials if t["status"] == 0]
    best = min(ok, key=lambda t: t["ms_per_iteration"])
    result = dict(key=key, best=best["options"], ms_per_iteration=best["ms_per_iteration"], trials=trials,
                  when=time.strftime("%Y-%m-%dT%H:%M:%S"))
    if cache_path:
        cache[key] = result
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return result


def bucket_of(target: int, width: float = 1.0) -> int:
    """Size bucket of a run: its target walker number on a log2 scale, `width` octaves per bucket."""
    return int(np.floor(np.log2(max(int(target), 2)) / width))


def tune_buckets(systems, targets, tau: float, thr: int, *, width: float = 1.0, **kw) -> tuple[list, dict]:
    """Tunes one representative run per size bucket (the run with the median target of the bucket) and gives
    every run its bucket's options. Returns (options per run, {bucket: tune() result with the representative's
    index})."""
    buckets: dict = {}
    for k, t in enumerate(targets):
        buckets.setdefault(bucket_of(t, width), []).append(k)
    results = {}
    for b, members in sorted(buckets.items()):
        order = sorted(members, key=lambda k: targets[k])
        rep = order[len(order) // 2]
        r = tune(systems[rep], tau, thr, int(targets[rep]), **kw)
        r = dict(r, representative=rep, members=len(members))
        results[b] = r
    per_run = [dict(results[bucket_of(t, width)]["best"]) for t in targets]
    return per_run, results
