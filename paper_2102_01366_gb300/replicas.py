"""Host logic for running independent replicas / cases on several GPUs.

A single tetrahedral mesh needs halo exchanges per stage to be split across
devices; independent cases do not: each rank advances its own cases with no
data-path collective.  What remains on the host is

* ``assign_cases``: longest-processing-time-first partition of cases (by cell
  count) over ranks, deterministic;
* ``rank_batch``: this rank's share of a batch of independent cases (its
  cases' meshes and the matching columns of the state);
* ``max_over_ranks``: the barrier and max-reduction of a per-rank time, on
  whatever torch.distributed backend the process group uses (NCCL on GPUs,
  gloo in the CPU tests);
* ``aggregate``: whole-job throughput = units processed by all ranks divided
  by the slowest rank's time (weak scaling when every rank has the same work).
"""
from __future__ import annotations

import heapq
import os


def world():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def assign_cases(cells, world_size):
    """Partition case indices over ranks, largest case first onto the least
    loaded rank (ties to the lower rank).  Returns a list of index lists."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(cells)), key=lambda i: (-int(cells[i]), i))
    heap = [(0, r) for r in range(world_size)]
    heapq.heapify(heap)
    out = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(cells[i]), r))
    return [sorted(x) for x in out]


def rank_batch(meshes, W, dW, world_size, rank):
    """This rank's cases of a batch: (case ids, their meshes, W[:, cells],
    dW[:, cells]).  W and dW hold the cases' cells one case after another,
    in case order (as the batch generator returns them)."""
    import numpy as np
    cells = [int(m["tet"].shape[0]) for m in meshes]
    first = np.concatenate([[0], np.cumsum(cells)]).astype(np.int64)
    mine = assign_cases(cells, world_size)[rank]
    cols = np.concatenate([np.arange(first[k], first[k + 1]) for k in mine]) if mine else np.zeros(0, np.int64)
    return mine, [meshes[k] for k in mine], np.ascontiguousarray(W[:, cols]), np.ascontiguousarray(dW[:, cols])


def max_over_ranks(value, device=None):
    """Barrier, then the maximum of ``value`` over all ranks (identity when
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    if device is None:
        device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device=None):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    if device is None:
        device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate(units_this_rank, seconds_this_rank, device=None):
    """Whole-job throughput (units per second) over all ranks."""
    total = sum_over_ranks(units_this_rank, device)
    slowest = max_over_ranks(seconds_this_rank, device)
    return total / slowest
