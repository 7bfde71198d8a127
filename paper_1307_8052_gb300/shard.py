"""Sharding of independent q-points over processes, one GPU each.

The q-points of Eq. 2 are independent problems: every rank evaluates the
frequency terms e_q(w) of its share with its own context, and E_c is the
weighted sum over all q-points.  No device collective touches the data path;
the partial energies (one scalar per rank) and the step time are reduced over
the process group on the host side of the step.
"""
from __future__ import annotations

from typing import Sequence


def shard_qpoints(costs: Sequence[float], world: int) -> list[list[int]]:
    """Split q-point indices over ``world`` ranks, balancing the estimated cost
    (e.g. NG^2 * pairs per q-point): longest first, each to the least-loaded
    rank (ties to the lower rank).  Deterministic; every q-point is assigned once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for iq in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(iq)
        load[r] += float(costs[iq])
    return [sorted(s) for s in out]


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def sum_over_ranks(x: float, device=None) -> float:
    """Sum of a host scalar over the process group (identity without one)."""
    dist = _dist()
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a host scalar over the process group (identity without one)."""
    dist = _dist()
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sharded_energy(evaluate, costs: Sequence[float], wq: Sequence[float], rank: int, world: int,
                   device=None) -> float:
    """E_c over all q-points with this rank's share evaluated locally.

    ``evaluate(iqs, wq_of_iqs)`` returns the weighted partial energy of the given
    q-points (e.g. a wrapper of ``rpa_energy``); it is called once, possibly
    with an empty list."""
    mine = shard_qpoints(costs, world)[rank]
    part = evaluate(mine, [wq[i] for i in mine]) if mine else 0.0
    return sum_over_ranks(part, device)


def partition(iqs: Sequence[int], costs: Sequence[float], world: int, replicas: bool = False) -> list[list[int]]:
    """q-point indices of every rank: a balanced share of ``iqs`` (``costs[i]``
    belongs to ``iqs[i]``), or all of them on every rank with ``replicas``."""
    if replicas:
        return [list(iqs) for _ in range(world)]
    return [[iqs[i] for i in part] for part in shard_qpoints(costs, world)]


def sharded_step(evaluate_q, iqs: Sequence[int], costs: Sequence[float], wq: Sequence[float], rank: int,
                 world: int, device=None, replicas: bool = False) -> float:
    """One E_c step over the q-points ``iqs`` (weights ``wq``, costs ``costs``,
    aligned with ``iqs``) on ``world`` ranks.

    ``evaluate_q(q_indices, weights)`` returns the weighted energy of the given
    q-points on this rank (a wrapper of ``rpa_energy``).  Sharded: this rank's
    balanced share is evaluated and the scalar partial energies are summed over
    the ranks, so every rank returns the E_c of all of ``iqs``.  Replicas:
    every rank evaluates all of ``iqs`` on its own and returns that E_c."""
    if replicas:
        return float(evaluate_q(list(iqs), list(wq)))

    def by_position(pos, wqs):
        return evaluate_q([iqs[i] for i in pos], wqs)
    return sharded_energy(by_position, costs, wq, rank, world, device)
