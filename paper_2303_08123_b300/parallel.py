"""Multi-GPU evaluation of a protocol population: replicas, no collective on
the data path.

Protocols are independent (the paper runs its evaluations on 2-4 GPUs with no
exchange between them, "GPU implementation: acceleration, fidelity &
normality").  A population is split across ranks by estimated cost
(lattice sites x horizon, longest-processing-time greedy), every rank
simulates its share on its own GPU, and one host-side gather returns all
results to every rank.  Launch one process per GPU (torchrun); any
torch.distributed backend works for the gather (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import heapq

import numpy as np


def protocol_cost(L, protocols, regrowth_h: float = 120.0) -> np.ndarray:
    """Estimated work of each protocol: L^3 sites x horizon in hours."""
    L = np.asarray(L, dtype=np.float64)
    horizon = np.array([sum(w) + regrowth_h for _, w in protocols], dtype=np.float64)
    return L ** 3 * horizon


def shard(costs, world: int):
    """Indices per rank, greedy on decreasing cost (each protocol goes to the
    currently least-loaded rank); returns (shards, load per rank)."""
    order = np.argsort(-np.asarray(costs, dtype=np.float64), kind="stable")
    heap = [(0.0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(int(i))
        heapq.heappush(heap, (load + float(costs[i]), r))
    loads = np.zeros(world)
    for r in range(world):
        loads[r] = float(np.sum(np.asarray(costs)[shards[r]])) if shards[r] else 0.0
        shards[r].sort()
    return shards, loads


def evaluate(protocols, L, R, simulate_fn, rank: int, world: int, group=None):
    """Every rank simulates its shard with `simulate_fn(protocols, L, R) -> counts`
    and all ranks receive the full result array (in the population's order)."""
    import torch.distributed as dist

    shards, _ = shard(protocol_cost(L, protocols), world)
    mine = shards[rank]
    local = simulate_fn([protocols[i] for i in mine], np.asarray(L)[mine], np.asarray(R)[mine]) if mine else []
    parts = [None] * world
    dist.all_gather_object(parts, (mine, [float(x) for x in local]), group=group)
    out = np.full(len(protocols), np.nan)
    for idx, vals in parts:
        out[idx] = vals
    return out
