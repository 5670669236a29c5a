"""Sample sharding across ranks and the cross-rank ensemble moments.

The samples of the qMC / quadrature ensemble are independent (the paper's
first level of parallelism, Section 4): each rank steps its own samples with
no data-path collective.  Two host-side pieces complete that picture:

* ``shard_even`` / ``lpt_assign``: which samples a rank owns.  Uniform
  samples split into contiguous equal blocks; samples of unequal cost (e.g.
  two grid sizes in one ensemble) are assigned longest-processing-time first.
* ``combine_moments``: the ensemble statistics over all ranks from each
  rank's local ``elder_moments`` output (eqs. pdestat and numer_var, the
  exceedance estimate of Section 3.3).  With local weights 1/S_r and rank
  weights W_r = S_r / S, the global moments are exactly
      mean = sum_r W_r mean_r,
      var  = sum_r W_r (var_r + (mean_r - mean)^2),
      P    = sum_r W_r P_r,
  three all-reduces of [N] arrays at output times only.
"""
from __future__ import annotations

import heapq

import torch
import torch.distributed as dist


def shard_even(total: int, world: int, rank: int) -> range:
    """Contiguous block of sample indices owned by ``rank`` (sizes differ by
    at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def lpt_assign(costs, world: int) -> list[list[int]]:
    """Longest-processing-time-first assignment of samples to ``world``
    ranks; returns the sample indices of every rank (each list sorted).
    Its makespan is at most 4/3 of the optimum."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(x) for x in out]


def combine_moments(mean: torch.Tensor, var: torch.Tensor, pexc: torch.Tensor,
                    n_local: int, group=None):
    """Global (mean, var, P(c > c*)) from every rank's local moments over its
    ``n_local`` samples (local weights 1/n_local).  Collective over
    ``group``; every rank returns the same tensors."""
    if not (dist.is_available() and dist.is_initialized()):
        return mean, var, pexc
    n = torch.tensor([float(n_local)], dtype=torch.float64, device=mean.device)
    dist.all_reduce(n, group=group)
    w = float(n_local) / float(n.item())
    m = mean * w
    dist.all_reduce(m, group=group)
    v = (var + (mean - m) ** 2) * w
    dist.all_reduce(v, group=group)
    p = pexc * w
    dist.all_reduce(p, group=group)
    return m, v, p
