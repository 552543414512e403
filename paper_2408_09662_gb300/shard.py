"""Data-parallel sharding across ranks (one process per GPU).

Instances are independent (CusADi §I: the parallelism is across environments,
not within one), so a batch of N instances is split into contiguous ranges,
one per rank, with no exchange on the evaluation path.  The only collective is
the gradient of a parameter shared by every instance (a broadcast input such as
a rollout's feedback gain): each rank reduces its own instances in-kernel and
the ranks then sum their partial gradients.
"""
from __future__ import annotations

import torch


def instance_range(N: int, rank: int, world: int) -> tuple:
    """[start, stop) of this rank's instances: contiguous, sizes differ by <= 1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(N, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def allreduce_shared_grad(grad: torch.Tensor, group=None) -> torch.Tensor:
    """Sums a shared parameter's gradient over ranks in place (no-op on one rank)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad
