"""Env sharding across GPUs (one process per GPU).

Envs are independent, so a multi-GPU run splits the env list into one
contiguous range per rank, balanced by an estimated per-env cost, and every
rank steps its own batch with no exchange inside the step.  Nothing here
computes any part of the step.
"""
from __future__ import annotations

import numpy as np


def env_cost(body_off, joint_off) -> np.ndarray:
    """Per-env cost estimate: rows x sweeps dominate (8 rows per joint), then
    the all-pairs broadphase and per-body work."""
    nb = np.diff(np.asarray(body_off, np.int64))
    nj = np.diff(np.asarray(joint_off, np.int64))
    return 32 * nj + nb * nb + 12 * nb


def shard_ranges(costs, world: int):
    """Contiguous [start, end) env ranges, one per rank, whose cost sums are
    as even as a prefix split allows (every rank gets at least one env when
    there are enough envs)."""
    costs = np.asarray(costs, np.float64)
    E = len(costs)
    if world < 1:
        raise ValueError("world must be >= 1")
    cum = np.concatenate([[0.0], np.cumsum(costs)])
    total = cum[-1]
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        k = int(np.searchsorted(cum, target, side="left"))
        # nearest prefix boundary to the target, kept strictly increasing
        if k > 0 and abs(cum[k - 1] - target) <= abs(cum[min(k, E)] - target):
            k -= 1
        lo = bounds[-1] + (1 if E - bounds[-1] > world - r else 0)
        hi = E - (world - r) if E >= world else E
        bounds.append(int(min(max(k, lo), max(hi, lo))))
    bounds.append(E)
    return [(bounds[i], bounds[i + 1]) for i in range(world)]


def local_envs(scene, rank: int, world: int):
    """The env indices rank `rank` owns."""
    ranges = shard_ranges(env_cost(scene.body_off, scene.joint_off), world)
    s, e = ranges[rank]
    return list(range(s, e))
