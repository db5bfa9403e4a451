"""Work distribution over the processes of a multi-GPU run (one process per GPU).

A single field does not shard without a halo exchange per half-sweep, but the
units of a batch (independent fields, or patches of one refinement level whose
boundary values are already fixed) do: each rank solves its share with no
data-path collective, and only timings and statistics are gathered.

* ``rank_info()``: (rank, world size, local rank) from the launcher's
  environment (torchrun's RANK / WORLD_SIZE / LOCAL_RANK), (0, 1, 0) otherwise.
* ``greedy_partition(weights, nparts)``: the longest-processing-time rule:
  units in decreasing weight order, each to the currently lightest part
  (ties to the lower part index), so the heaviest part exceeds the mean by at
  most the largest unit.  Deterministic: every rank computes the same split.
* ``max_over_ranks(x)``: the maximum of a float over all ranks (the job's time
  is the slowest rank's), through torch.distributed when it is initialised.
"""
from __future__ import annotations

import os


def rank_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    if world < 1 or not (0 <= rank < world):
        raise ValueError(f"inconsistent RANK={rank} WORLD_SIZE={world}")
    return rank, world, local


def greedy_partition(weights, nparts):
    """Index lists (one per part, each in increasing index order)."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    load = [0] * nparts
    parts = [[] for _ in range(nparts)]
    for i in order:
        p = min(range(nparts), key=lambda q: (load[q], q))
        parts[p].append(i)
        load[p] += weights[i]
    return [sorted(p) for p in parts]


def max_over_ranks(x, device=None):
    """max of the float x over the ranks of the default process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
