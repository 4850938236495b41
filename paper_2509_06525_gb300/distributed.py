"""Multi-rank helpers for the KPM trace estimate (Sec. 2.4).

The R random vectors of the stochastic trace are independent: rank k of W
takes a contiguous block of vector indices (kpm_moments' first_vector), so
the ranks together hold exactly the ensemble one call over all R_total
vectors would draw, with no exchange during the recursion.  The only
collective is the gather of the R x M moments at the end (a few KB), and the
max-over-ranks step time of a weak-scaling run.  The functions take any
torch.distributed process group (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

from typing import Optional, Tuple

import torch
import torch.distributed as dist


def vector_shard(r_total: int, rank: int, world: int) -> Tuple[int, int]:
    """(first, count) of rank's block of r_total vectors; the first
    r_total % world ranks hold one vector more."""
    if not (0 <= rank < world) or r_total < world:
        raise ValueError(f"need 0 <= rank < world <= r_total (rank={rank}, world={world}, r_total={r_total})")
    base, extra = divmod(r_total, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def gather_moments(mu_local: torch.Tensor, r_total: int, group: Optional[dist.ProcessGroup] = None) -> torch.Tensor:
    """All ranks' per-vector moments [count_k, M] -> [r_total, M] in vector
    order, on every rank."""
    world = dist.get_world_size(group)
    M = mu_local.shape[1]
    width = -(-r_total // world)
    padded = torch.zeros((width, M), dtype=mu_local.dtype, device=mu_local.device)
    padded[:mu_local.shape[0]] = mu_local
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    out = []
    for k in range(world):
        _, count = vector_shard(r_total, k, world)
        out.append(parts[k][:count])
    return torch.cat(out, 0)


def max_over_ranks(value: float, device, group: Optional[dist.ProcessGroup] = None) -> float:
    """The largest of the ranks' values (step times of a weak-scaling run)."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
