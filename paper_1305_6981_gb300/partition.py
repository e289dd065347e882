"""Host side of the exchange step of a hash-partitioned run spread over processes (Sec. V A, Fig. 2).

A partition's determinants are those whose Algorithm 1 fingerprint is congruent to the partition's index
modulo the partition count (owners(), computed by the library's fciqmc_owner). Each iteration every
partition sends the spawned entries bound for the others in one collective: first the per-destination
counts, then the entries (the paper's single MPI_AlltoAllv, here torch.distributed.all_to_all_single, which
runs over NCCL on device tensors or gloo on host tensors); then the partitions' counters are summed for the
run's row, the numerator added in partition order so that every rank gets the same value.

Within one process, fciqmc_group_* does the same exchange on the device (Partitioned); these functions are
the per-process form of that step, argument marshalling around collectives with no arithmetic of the method.
"""
from __future__ import annotations

import numpy as np

from .fciqmc import owners  # noqa: F401  (re-exported: the partition of each determinant)

INT_FIELDS = ("nw_in", "nd_in", "c0_in", "nw_out", "nd_out", "attempts", "nulls", "spawn_events", "spawned_walkers",
              "death_walkers", "clone_walkers", "merged_entries", "aborted_walkers", "inserted_dets",
              "heavy_attempts")


def route(keys: np.ndarray, vals: np.ndarray, dest: np.ndarray, n_parts: int):
    """Orders spawned entries by destination partition (the spawned array of Fig. 2): returns the entries
    sorted by destination (stable, so each destination's entries keep their order) and the count per
    destination."""
    order = np.argsort(dest, kind="stable")
    counts = np.bincount(dest, minlength=n_parts).astype(np.int64)
    return keys[order], vals[order], counts


def exchange(keys: np.ndarray, vals: np.ndarray, counts: np.ndarray, group=None):
    """One all-to-all of routed entries (keys (n, W) uint64, vals (n,) int64 payloads, counts per destination):
    returns the entries every partition sent to this one, ordered by source partition."""
    import torch
    import torch.distributed as dist

    W = keys.shape[1] if keys.ndim == 2 else 1
    send_counts = torch.as_tensor(np.asarray(counts, dtype=np.int64))
    recv_counts = torch.empty_like(send_counts)
    dist.all_to_all_single(recv_counts, send_counts, group=group)
    rows = np.concatenate([np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, W).view(np.int64),
                           np.asarray(vals, dtype=np.int64).reshape(-1, 1)], axis=1)
    send = torch.from_numpy(np.ascontiguousarray(rows)).reshape(-1)
    recv = torch.empty(int(recv_counts.sum()) * (W + 1), dtype=torch.int64)
    dist.all_to_all_single(recv, send, [int(c) * (W + 1) for c in recv_counts.tolist()],
                           [int(c) * (W + 1) for c in send_counts.tolist()], group=group)
    r = recv.numpy().reshape(-1, W + 1)
    return np.ascontiguousarray(r[:, :W]).view(np.uint64), np.ascontiguousarray(r[:, W])


def reduce_row(row: dict, group=None) -> dict:
    """The run's row from this partition's row: integer counters summed over partitions, numerators gathered
    and added in partition order (the same value on every rank), shift and iteration unchanged."""
    import torch
    import torch.distributed as dist

    ints = torch.tensor([int(row[f]) for f in INT_FIELDS], dtype=torch.int64)
    dist.all_reduce(ints, op=dist.ReduceOp.SUM, group=group)
    nums = [torch.zeros(1, dtype=torch.float64) for _ in range(dist.get_world_size(group))]
    dist.all_gather(nums, torch.tensor([float(row["num_in"])], dtype=torch.float64), group=group)
    total = 0.0
    for x in nums:
        total += float(x.item())
    out = dict(row)
    out.update({f: int(v) for f, v in zip(INT_FIELDS, ints.tolist())})
    out["num_in"] = total
    return out
