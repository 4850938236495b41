"""Multi-rank helpers: the KPM trace estimate (Sec. 2.4) and the
band-energy training (Sec. 3, Eq. 3).

The R random vectors of the stochastic trace are independent: rank k of W
takes a contiguous block of vector indices (kpm_moments' first_vector), so
the ranks together hold exactly the ensemble one call over all R_total
vectors would draw, with no exchange during the recursion.  The only
collective is the gather of the R x M moments at the end (a few KB), and the
max-over-ranks step time of a weak-scaling run.

The band-energy training shards its periodic cells the same way.  Its loss
couples the whole batch through S = sum w |E_pre - E_ref| (dL/dE = 2 S w
sign + 2 w D), so a step has two exchanges: an all-gather of the ranks'
band energies (every rank then evaluates the loss of the whole batch) and an
all-reduce of the parameter gradients.

The functions take any torch.distributed process group (NCCL on GPUs, gloo
on CPU).
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple

import torch
import torch.distributed as dist


def block_shard(total: int, rank: int, world: int) -> Tuple[int, int]:
    """(first, count) of rank's contiguous block of `total` items; the first
    total % world ranks hold one item more."""
    if not (0 <= rank < world) or total < world:
        raise ValueError(f"need 0 <= rank < world <= total (rank={rank}, world={world}, total={total})")
    base, extra = divmod(total, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def vector_shard(r_total: int, rank: int, world: int) -> Tuple[int, int]:
    """(first, count) of rank's block of r_total random vectors."""
    return block_shard(r_total, rank, world)


def _staged(t: torch.Tensor, group) -> bool:
    """Device tensors go through host memory on the gloo backend (which does
    not gather device tensors); NCCL takes them as they are."""
    return t.is_cuda and dist.get_backend(group) == "gloo"


def gather_blocks(local: torch.Tensor, total: int, group: Optional[dist.ProcessGroup] = None) -> torch.Tensor:
    """All ranks' blocks [count_k, ...] (block_shard order) -> [total, ...]
    on every rank."""
    world = dist.get_world_size(group)
    width = -(-total // world)
    dev = local.device
    src = local.cpu() if _staged(local, group) else local
    padded = torch.zeros((width,) + tuple(src.shape[1:]), dtype=src.dtype, device=src.device)
    padded[:src.shape[0]] = src
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    out = torch.cat([parts[k][:block_shard(total, k, world)[1]] for k in range(world)], 0)
    return out.to(dev)


def all_reduce_sum(t: torch.Tensor, group: Optional[dist.ProcessGroup] = None) -> torch.Tensor:
    """In-place sum over ranks (through host memory on gloo)."""
    if _staged(t, group):
        h = t.cpu()
        dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
        t.copy_(h)
    else:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def gather_moments(mu_local: torch.Tensor, r_total: int, group: Optional[dist.ProcessGroup] = None) -> torch.Tensor:
    """All ranks' per-vector moments [count_k, M] -> [r_total, M] in vector
    order, on every rank."""
    return gather_blocks(mu_local, r_total, group)


def band_step(forward_local: Callable, loss_all: Callable, backward_local: Callable, e_ref_all: torch.Tensor,
              n_cells: int, group: Optional[dist.ProcessGroup] = None):
    """One data-parallel step of the band-energy training over cells
    sharded with block_shard:

        E_local, ctx = forward_local()               this rank's model H and bands
        E_all = all-gather of E_local                [n_cells, n_k, n_bands]
        dLdE_all, stats = loss_all(E_all, e_ref_all) Eq. 3 of the whole batch, on every rank
        grad = backward_local(ctx, dLdE_all[first:first + count])
        grad = all-reduce (sum) of grad

    Returns (stats, grad)."""
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    first, count = block_shard(n_cells, rank, world)
    e_local, ctx = forward_local()
    if e_local.shape[0] != count:
        raise ValueError(f"rank {rank} holds {e_local.shape[0]} cells, its shard has {count}")
    e_all = gather_blocks(e_local, n_cells, group)
    dLdE_all, stats = loss_all(e_all, e_ref_all)
    grad = backward_local(ctx, dLdE_all[first:first + count].contiguous())
    all_reduce_sum(grad, group)
    return stats, grad


def max_over_ranks(value: float, device, group: Optional[dist.ProcessGroup] = None) -> float:
    """The largest of the ranks' values (step times of a weak-scaling run)."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
