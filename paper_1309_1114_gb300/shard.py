"""Sharding a frame over ranks: the paper's MPI scheme (Sec. 2).

Each rank renders the particles of its own chunk into a partial image; the
partial additive images are summed (E_p = A_p makes the result independent of
the order, so the sum over ranks equals the whole frame), and the E=A map
1 - exp(-S) is applied once, after the sum.  The benchmark's multi-GPU mode
instead runs independent replicas (weak scaling, no collective); these helpers
are the composition step for a frame split across ranks.
"""
from __future__ import annotations


def partition(n: int, world: int) -> list:
    """Contiguous particle ranges [lo, hi) of equal size (+-1), one per rank."""
    if world < 1 or n < 0:
        raise ValueError("partition: world >= 1 and n >= 0")
    return [(n * r // world, n * (r + 1) // world) for r in range(world)]


def allreduce_image(img, group=None):
    """Sum the ranks' partial additive images in place (torch.distributed)."""
    import torch.distributed as dist
    dist.all_reduce(img, op=dist.ReduceOp.SUM, group=group)
    return img


def ea_map(img):
    """E_p = A_p solution of Eq. 1 applied to a summed image: 1 - exp(-S)."""
    import torch
    return -torch.expm1(-img)


def max_over_ranks(value: float, group=None) -> float:
    """Largest value over ranks (the benchmark's time per step)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
