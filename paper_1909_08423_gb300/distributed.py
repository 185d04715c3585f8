"""Walker sharding across ranks (one process per GPU).

Walkers are independent Markov chains, so the local-energy and sampling
path shards by contiguous walker ranges with no exchange.  A VMC loss
gradient over all ranks has three exchange steps: the clipping window needs
the median and mean deviation of every walker's E_loc (an all-gather of the
W local energies), the loss is their mean, and the parameter gradient is a
sum over walkers (an all-reduce).  ``clip_fn`` is the library's clipping call
(or any function with its contract); these helpers only move data.
"""

from __future__ import annotations

import torch
import torch.distributed as dist


def world_size(group=None):
    """Ranks in `group` (1 when torch.distributed is not initialised)."""
    if not (dist.is_available() and dist.is_initialized()):
        return 1
    return dist.get_world_size(group)


def rank_of(group=None):
    if not (dist.is_available() and dist.is_initialized()):
        return 0
    return dist.get_rank(group)


def shard(W_total, rank, world):
    """Contiguous walker range [lo, hi) of one rank."""
    base, rem = divmod(W_total, world)
    lo = rank * base + min(rank, rem)
    return lo, lo + base + (1 if rank < rem else 0)


def global_clip(E_local, clip_fn, group=None):
    """Clipped energies and loss weights for this rank's walkers, computed
    over the walkers of all ranks.  Returns (E_clipped_local, cot_local,
    loss)."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    n = torch.tensor([E_local.numel()], device=E_local.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    m = max(sizes)
    pad = torch.zeros(m, dtype=E_local.dtype, device=E_local.device)
    pad[:E_local.numel()] = E_local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    E_all = torch.cat([p[:s] for p, s in zip(parts, sizes)]).contiguous()
    Ec = torch.empty_like(E_all)
    cot = torch.empty_like(E_all)
    clip_fn(E_all, Ec, cot)
    lo = sum(sizes[:rank])
    hi = lo + sizes[rank]
    return Ec[lo:hi].clone(), cot[lo:hi].clone(), Ec.mean()


def allreduce_grad(g, group=None):
    dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return g
