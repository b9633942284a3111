"""Splitting the hot path over several GPUs (one process per GPU).

Vectors are independent under W, W^T and S (§II-A, §III-A), so a batch shards
by rows and a set of transforms by whole transforms, with no exchange of data
between ranks.  The only collective steps are the ones the method has:

* the gradients with respect to the reflector vectors and the spectrum are
  sums over the batch (§IV, the fit of W diag(d) W^T), so data-parallel
  fitting adds the per-rank sums: :func:`allreduce_sum`;
* a timed step takes the slowest rank: :func:`reduce_max`.

The helpers work on any torch.distributed backend (NCCL on GPUs, gloo on the
host); the partitioning functions are plain host arithmetic.
"""

from __future__ import annotations

import heapq


def shard_rows(batch: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [r0, r1) of a batch of `batch` rows that rank `rank` of `world` takes:
    contiguous, sizes differing by at most one, covering the batch once."""
    if world < 1 or not 0 <= rank < world or batch < 0:
        raise ValueError(f"batch={batch}, world={world}, rank={rank}")
    base, extra = divmod(batch, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def transform_cost(n: int, h: int, batch: int) -> float:
    """Predicted time of one transform, in units of FP32 FMA work plus its row
    traffic at the FP32 ridge: batch * (4 n h + 96 n)."""
    return float(batch) * (4.0 * n * h + 96.0 * n)


def shard_transforms(specs, world: int) -> list[list[int]]:
    """Assign transforms (n, h, batch, ...) to `world` ranks by predicted cost:
    largest first, each to the least loaded rank (LPT).  Returns, per rank, the
    indices of its transforms in their original order."""
    if world < 1:
        raise ValueError(f"world={world}")
    order = sorted(range(len(specs)), key=lambda i: -transform_cost(*specs[i][:3]))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + transform_cost(*specs[i][:3]), r))
    return [sorted(ix) for ix in out]


def reduce_max(value: float, dist, device=None) -> float:
    """The largest `value` over all ranks (the slowest rank's time)."""
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(tensors, dist) -> None:
    """Add the tensors in place over all ranks (per-rank gradient sums)."""
    for t in tensors:
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
