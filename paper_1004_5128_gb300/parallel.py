"""Multi-GPU layout: the memory-sum path shards by instance with no data-path collective.

Independent problem instances are split over ranks (one process per GPU) so that every rank
gets about the same history traffic; each rank then runs its shard as one persistent batch
launch.  The only collectives are outside the data path: a barrier around timing and a max
over ranks of the elapsed time.  Within one instance the path would shard by spatial slabs with
a one-cell halo of u^k per step; on the single-GPU machines this build targets that layout is not
used, and a single instance is run as replicas.
"""
from __future__ import annotations

import heapq


def schedule_terms(p: dict, samples: int = 64) -> float:
    """Estimated history rows read over p's run: sum_k n(k), from the library's own schedule
    sampled at `samples` evenly spaced steps (exact for full and short memory)."""
    K = p["K"]
    if p["mem_mode"] == 0:
        return K * (K - 1) / 2.0
    if p["mem_mode"] == 1:
        L = p["mem_L"]
        return sum(min(L, k) for k in range(K))
    from . import _lib
    from .frd import make_problem
    fp = make_problem(p, max_steps=max(1, K))
    ks = sorted(set(int(i * (K - 1) / max(1, samples - 1)) for i in range(samples)))
    n = [len(_lib.fd_schedule(fp, k)[0]) - 1 for k in ks]
    total = 0.0
    for (k0, n0), (k1, n1) in zip(zip(ks, n), zip(ks[1:], n[1:])):
        total += 0.5 * (n0 + n1) * (k1 - k0)
    return total


def instance_cost(p: dict) -> float:
    """History elements streamed by one instance (rows read x points)."""
    return schedule_terms(p) * p["nx"] * p["ny"] * p.get("nz", 1)


def shard(problems: list, world_size: int) -> list:
    """Greedy longest-processing-time split: list of index lists, one per rank, covering every
    instance exactly once, with rank loads within the largest single instance of each other."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(problems)), key=lambda i: -instance_cost(problems[i]))
    heap = [(0.0, r) for r in range(world_size)]
    out = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + instance_cost(problems[i]), r))
    return [sorted(x) for x in out]


def max_over_ranks(value: float) -> float:
    """Max of a scalar over the default process group (the value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float) -> float:
    """Sum of a scalar over the default process group (the value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
