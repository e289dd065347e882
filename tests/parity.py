"""Helpers for comparing the CUDA path with the oracle (tests only)."""
from __future__ import annotations

import numpy as np


def canonical(dets: np.ndarray, pops: np.ndarray, hd: np.ndarray | None = None):
    """Walker list sorted by determinant (words as an unsigned big number)."""
    dets = np.asarray(dets, dtype=np.uint64)
    if len(pops) == 0:  # an empty list
        out = (dets.reshape(0, 0), np.asarray(pops)[:0])
        return out + (np.asarray(hd)[:0],) if hd is not None else out
    dets = dets.reshape(len(pops), -1)
    keys = [dets[:, w] for w in range(dets.shape[1])]
    order = np.lexsort(keys)
    out = (dets[order], np.asarray(pops)[order])
    if hd is not None:
        out = out + (np.asarray(hd)[order],)
    return out


def same_lists(a, b) -> bool:
    da, pa = canonical(a[0], a[1])
    db, pb = canonical(b[0], b[1])
    return da.shape == db.shape and np.array_equal(da, db) and np.array_equal(pa, pb)


INT_FIELDS = ["iteration", "nw_in", "nd_in", "c0_in", "nw_out", "nd_out", "attempts", "nulls", "spawn_events",
              "spawned_walkers", "death_walkers", "clone_walkers", "merged_entries", "aborted_walkers",
              "inserted_dets"]


def compare_rows(rows_gpu, rows_oracle, rel=1e-11):
    """Integer fields bit-exact, shift bit-exact, projected-energy numerator within rel."""
    assert len(rows_gpu) == len(rows_oracle)
    for g, o in zip(rows_gpu, rows_oracle):
        for f in INT_FIELDS:
            of = "iter" if f == "iteration" else f
            assert g[f] == o[of], (f, g[f], o[of], g["iteration"])
        assert g["shift"] == o["shift"], (g["shift"], o["shift"], g["iteration"])
        scale = max(abs(o["num_in"]), 1e-300)
        assert abs(g["num_in"] - o["num_in"]) <= rel * scale, (g["num_in"], o["num_in"], g["iteration"])
