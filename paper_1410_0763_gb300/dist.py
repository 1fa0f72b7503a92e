"""Direction-sharded sweeps over several ranks (one process per GPU).

The sweep's directions are independent until the angle average (Sec. 2.2,
Eq. mean_intensity), so rank r of W sweeps the contiguous block of RING
indices [r N_d / W, (r + 1) N_d / W) and produces its additive share of
J^in; the shares are gathered to every rank in rank order and summed in that
order by ``art_sum_partials`` (Kahan), so the result is the same for a given
W whatever order the collective uses internally.  The gather is the only
exchange on the path.
"""
from __future__ import annotations

import numpy as np


def direction_block(nside: int, rank: int, world: int) -> tuple[int, int]:
    """RING-index range [begin, end) of rank `rank` out of `world` (contiguous, sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    nd = 12 * nside * nside
    return nd * rank // world, nd * (rank + 1) // world


def gather_in_rank_order(part, group=None):
    """All-gather one tensor per rank; returns a [world, ...] tensor whose row r is rank r's part."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    out = [torch.empty_like(part) for _ in range(world)]
    dist.all_gather(out, part.contiguous(), group=group)
    return torch.stack(out)


def sweep_jin_sharded(kappa, src, nside: int, group=None, field_form: int = 0, **ctx_kw):
    """J^in of a grid whose sweep is split over the ranks of `group` by direction.

    kappa, src: this rank's CUDA float32 tensors [nz][ny][nx] (the same fields on
    every rank).  Returns J^in [nz][ny][nx] on every rank.
    """
    import torch
    import torch.distributed as dist
    from . import art
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    b, e = direction_block(nside, rank, world)
    part = torch.zeros_like(kappa)
    if e > b:
        sw = art.ArtSweep(tuple(kappa.shape), nside, 1, field_form=field_form, dir_range=(b, e), **ctx_kw)
        sw.set_fields(kappa.reshape(-1), src.reshape(-1))
        sw.sweep(J_in=part.reshape(-1))
        sw.close()
    parts = gather_in_rank_order(part, group)
    out = torch.empty_like(kappa)
    art.art_sum_partials(parts.reshape(world, -1), out.reshape(-1))
    return out


def combine_in_rank_order(parts: np.ndarray) -> np.ndarray:
    """Host form of the combination (rank-order Kahan sum in float64), for CPU ranks."""
    s = np.zeros(parts.shape[1:], dtype=np.float64)
    c = np.zeros_like(s)
    for p in parts:
        y = p - c
        t = s + y
        c = (t - s) - y
        s = t
    return s
