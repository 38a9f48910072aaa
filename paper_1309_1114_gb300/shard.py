"""Frames split over ranks: the paper's MPI scheme (Sec. 2), on the library.

Each rank renders the particles of its own contiguous chunk with the library
into a partial additive image; the partial images are summed over the ranks
(E_p = A_p makes the sum independent of the order in which particles are
added, so the sum over ranks is the whole frame), and the E = A map
1 - exp(-S), when the frame asks for it, is applied once, after the sum, by the
library (``spl_apply_ea``: the map is not linear, so it cannot be applied to
the partial images).  The general absorption mode is not additive over chunks
and is refused.  The benchmark's multi-GPU mode runs independent replicas
instead (weak scaling, no collective); these helpers are the composition of a
frame split across ranks.
"""
from __future__ import annotations

from . import splotch as S


def partition(n: int, world: int) -> list:
    """Contiguous particle ranges [lo, hi) of equal size (+-1), one per rank."""
    if world < 1 or n < 0:
        raise ValueError("partition: world >= 1 and n >= 0")
    return [(n * r // world, n * (r + 1) // world) for r in range(world)]


def render_partial(renderer, parts: dict, rank: int, world: int, image, stream=None) -> bool:
    """Render rank's chunk of parts (host or device arrays) into image (a CUDA
    float32 tensor) as an additive partial image with the renderer's camera,
    colour map and parameters.  Returns whether the frame asks for the E = A
    map, which compose() applies after the sum."""
    n = int(parts["x"].shape[0])
    lo, hi = partition(n, world)[rank]
    renderer.load({k: v[lo:hi] for k, v in parts.items()})
    q = renderer.get_params()
    if q["mode"] == S.SPL_MODE_ABSORB:
        raise ValueError("the general absorption form is not additive over particle chunks")
    ea = q["mode"] == S.SPL_MODE_EA
    if ea:
        renderer.set_params(**dict(q, mode=S.SPL_MODE_ADDITIVE))
    try:
        renderer.render(image, stream)
    finally:
        if ea:
            renderer.set_params(**q)
    return ea


def allreduce_image(img, group=None):
    """Sum the ranks' partial additive images in place (torch.distributed; a
    CUDA image goes through host memory when the backend is gloo)."""
    import torch.distributed as dist
    if getattr(img, "is_cuda", False) and dist.get_backend(group) == "gloo":
        host = img.cpu()
        dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
        img.copy_(host)
        return img
    dist.all_reduce(img, op=dist.ReduceOp.SUM, group=group)
    return img


def compose(renderer, image, ea: bool, group=None):
    """Sum of the partial images over the ranks, then the E = A map (library)."""
    allreduce_image(image, group)
    if ea:
        renderer.apply_ea(image)
    return image


def render_frame(renderer, parts: dict, image, group=None, stream=None):
    """The whole frame on every rank: this rank's partial image, the sum over
    the ranks, and the E = A map when the renderer's mode asks for it."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    ea = render_partial(renderer, parts, rank, world, image, stream)
    return compose(renderer, image, ea, group)


def max_over_ranks(value: float, group=None) -> float:
    """Largest value over ranks (the benchmark's time per step)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
