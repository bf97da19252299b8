"""Host-side logic for running independent SP2 problems on several GPUs (one rank each).

A single density-matrix solve does not shard without a per-layer exchange of X,
so several GPUs serve independent problems: replicas of one problem (the
benchmark's weak scaling) or the instances of a batch.  Nothing here touches the
data path; ranks only exchange scalars and small per-instance records through
``torch.distributed`` (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

import heapq
from typing import List, Sequence

import torch
import torch.distributed as dist


def lpt_assign(costs: Sequence[float], world: int) -> List[List[int]]:
    """Longest-processing-time-first assignment of work items to ``world`` ranks.

    Items are taken in decreasing cost (ties by index) and each goes to the rank
    with the least total so far (ties to the lower rank).  Returns, per rank, the
    item indices in increasing order.  The result is deterministic, so every rank
    computes the same assignment without communication.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0.0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-float(costs[k]), k)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(x) for x in out]


def solve_cost(n: int) -> float:
    """Relative cost of one solve of size n (dense squares: n^3 per layer)."""
    return float(n) ** 3


def shard_instances(sizes: Sequence[int], rank: int, world: int) -> List[int]:
    """Indices of the batch instances this rank solves."""
    return lpt_assign([solve_cost(n) for n in sizes], world)[rank]


def aggregate_step_time(ms: float, work: float, device=None):
    """Max step time over ranks and the sum of the work (e.g. flops) all ranks did.

    The whole-job rate is then sum(work) / max(ms): the units all ranks processed
    over the slowest rank's time."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, work
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    v = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return float(t.item()), float(v.item())


def gather_records(records: dict, world: int):
    """All ranks' {instance index: record} maps merged on every rank (small host objects)."""
    if world == 1 or not dist.is_initialized():
        return dict(records)
    parts = [None] * world
    dist.all_gather_object(parts, records)
    merged = {}
    for p in parts:
        merged.update(p)
    return merged


def run_sharded_batch(sizes: Sequence[int], solve, rank: int, world: int, device=None):
    """One batch over ``world`` ranks: this rank solves its LPT share and every rank
    ends with all instances' records.

    ``solve(indices)`` solves the given instances on this rank (one grouped launch
    on its GPU) and returns ({index: record}, ms, work), ``work`` in whatever unit
    the rate is quoted in (flops).  Returns (records of every instance, this rank's
    indices, the slowest rank's ms, the work of all ranks): the whole-job rate is
    work / ms.  The data path has no collective; only these scalars and records
    cross ranks."""
    mine = shard_instances(sizes, rank, world)
    records, ms, work = solve(mine)
    if set(records) != set(mine):
        raise ValueError("solve() must return one record per assigned instance")
    ms_all, work_all = aggregate_step_time(ms, work, device=device)
    merged = gather_records(records, world)
    return merged, mine, ms_all, work_all
