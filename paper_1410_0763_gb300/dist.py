"""Direction-sharded sweeps over several ranks (one process per GPU).

The sweep's directions are independent until the angle average (Sec. 2.2,
Eq. mean_intensity; the paper's Sec. 3.2 spreads directions over its GPUs
the same way), so rank r of W sweeps the contiguous block of RING indices
[r N_d / W, (r + 1) N_d / W) and produces its additive share of J^in.  The
shares are combined by a rank-ordered reduce-scatter:

* the cells are split into W contiguous blocks; rank q receives block q of
  every rank's share (point-to-point, so the data movement is (W - 1)/W of a
  share per rank in each direction);
* rank q sums the W pieces of its block in rank order with Kahan
  compensation on the GPU (``art_sum_partials``), so the result does not
  depend on how a collective would order a sum;
* the summed blocks are all-gathered, so every rank holds J^in.

For a fixed W the result is bit-identical on every rank and from run to run.
"""
from __future__ import annotations


def direction_block(nside: int, rank: int, world: int) -> tuple[int, int]:
    """RING-index range [begin, end) of rank `rank` out of `world` (contiguous, sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    nd = 12 * nside * nside
    return nd * rank // world, nd * (rank + 1) // world


def cell_block(n: int, rank: int, world: int) -> tuple[int, int]:
    """Element range [begin, end) of the reduce-scatter block that rank `rank` sums."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return n * rank // world, n * (rank + 1) // world


def exchange_blocks(share, group=None):
    """Rank-ordered scatter: returns a [world, len] tensor whose row r is block `rank` of rank r's
    share (a flat tensor of the same length on every rank).  Point-to-point sends and receives,
    so it works on the gloo and the NCCL backend alike."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    n = share.numel()
    flat = share.reshape(-1).contiguous()
    b, e = cell_block(n, rank, world)
    out = torch.empty((world, e - b), dtype=share.dtype, device=share.device)
    out[rank].copy_(flat[b:e])
    ops = []
    for q in range(world):
        if q == rank:
            continue
        qb, qe = cell_block(n, q, world)
        peer = dist.get_global_rank(group, q) if group is not None else q
        ops.append(dist.P2POp(dist.isend, flat[qb:qe].contiguous(), peer, group))
        ops.append(dist.P2POp(dist.irecv, out[q], peer, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return out


def gather_blocks(block, n: int, group=None):
    """All-gather the ranks' summed blocks (rank q holds elements cell_block(n, q, W)) into a flat
    tensor of n elements on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    size = max(cell_block(n, q, world)[1] - cell_block(n, q, world)[0] for q in range(world))
    pad = torch.zeros(size, dtype=block.dtype, device=block.device)
    pad[:block.numel()].copy_(block.reshape(-1))
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    out = torch.empty(n, dtype=block.dtype, device=block.device)
    for q in range(world):
        b, e = cell_block(n, q, world)
        out[b:e].copy_(parts[q][:e - b])
    return out


class ShardedSweep:
    """This rank's share of a direction-sharded sweep, and the combination of all shares.

    shape: (nz, ny, nx); the same fields on every rank.  The context for this rank's RING-index
    block stays allocated across calls.  FP32, CUDA tensors, one process per GPU."""

    def __init__(self, shape, nside: int, nbins: int = 1, group=None, **ctx_kw):
        import torch.distributed as dist
        from . import art
        self.group = group
        self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        self.block = direction_block(nside, self.rank, self.world)
        self.shape, self.nbins = tuple(shape), int(nbins)
        self.sw = None
        if self.block[1] > self.block[0]:
            self.sw = art.ArtSweep(self.shape, nside, self.nbins, dir_range=self.block, **ctx_kw)

    def set_fields(self, kappa, src):
        if self.sw is not None:
            self.sw.set_fields(kappa.reshape(-1), src.reshape(-1))

    def share(self, out):
        """This rank's additive share of J^in ([bins][nz][ny][nx], still divided by the full N_d)."""
        if self.sw is None:
            out.zero_()
        else:
            self.sw.sweep(J_in=out.reshape(-1))
        return out

    def jin(self, share):
        """J^in from this rank's share: rank-ordered reduce-scatter and all-gather."""
        import torch
        from . import art
        n = share.numel()
        pieces = exchange_blocks(share, self.group)
        mine = torch.empty(pieces.shape[1], dtype=share.dtype, device=share.device)
        if mine.numel():
            art.art_sum_partials(pieces, mine)
        return gather_blocks(mine, n, self.group).reshape(share.shape)

    def check(self) -> int:
        from . import art
        return self.sw.check() if self.sw is not None else art.ART_OK

    def close(self):
        if self.sw is not None:
            self.sw.close()
            self.sw = None


def sweep_jin_sharded(kappa, src, nside: int, group=None, **ctx_kw):
    """J^in of a grid whose sweep is split over the ranks of `group` by direction (one call:
    creates and releases the context; ShardedSweep keeps it)."""
    import torch
    s = ShardedSweep(tuple(kappa.shape[-3:]), nside, 1 if kappa.dim() == 3 else kappa.shape[0], group, **ctx_kw)
    try:
        s.set_fields(kappa, src)
        part = s.share(torch.empty_like(kappa))
        return s.jin(part)
    finally:
        s.close()
