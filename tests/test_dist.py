"""Direction-sharded sweep over ranks: the partition of the RING indices and
of the cells, the rank-ordered reduce-scatter (point-to-point exchange of cell
blocks, rank-order Kahan sum of each block, all-gather of the summed blocks),
run as world-size-2 and -3 gloo process groups on CPU (each rank's share
computed by the oracle, since this host has no GPU; the block sum, which the
library does on the GPU, is written here in numpy), against the unsharded
oracle sweep."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1410_0763_gb300 import dist as adist


def test_direction_blocks_partition_the_sphere():
    for nside in (1, 2, 3, 8):
        nd = 12 * nside * nside
        for world in (1, 2, 3, 5, 8):
            blocks = [adist.direction_block(nside, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == nd
            assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        adist.direction_block(1, 2, 2)


def test_cell_blocks_partition_the_cells():
    for n in (1, 7, 1000, 4096 * 3 + 1):
        for world in (1, 2, 3, 8):
            blocks = [adist.cell_block(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))


def kahan_rows(parts: np.ndarray) -> np.ndarray:
    """Rank-order Kahan sum of the rows (what art_sum_partials computes on the GPU)."""
    s = np.zeros(parts.shape[1:], dtype=parts.dtype)
    c = np.zeros_like(s)
    for p in parts:
        y = p - c
        t = s + y
        c = (t - s) - y
        s = t
    return s


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1410_0763_gb300 import workloads as wl
    case = wl.lognormal_iid(10, 2, seed=3)
    nside = 2
    b, e = adist.direction_block(nside, rank, world)
    acc, _ = oracle.sweep_range(case.kappa, case.src, nside, b, e, nthreads=1)
    share = torch.as_tensor(acc / (12 * nside * nside))
    pieces = adist.exchange_blocks(share.reshape(-1))
    n = share.numel()
    b, e = adist.cell_block(n, rank, world)
    assert pieces.shape == (world, e - b)
    mine = torch.as_tensor(kahan_rows(pieces.numpy()))
    jin = adist.gather_blocks(mine, n).reshape(share.shape).numpy()
    np.save(os.path.join(out_dir, f"jin_{rank}.npy"), jin)
    np.save(os.path.join(out_dir, f"share_{rank}.npy"), share.numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reproduce_the_full_sweep(tmp_path, world):
    import socket
    with socket.socket() as s_:
        s_.bind(("127.0.0.1", 0))
        port = s_.getsockname()[1]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    import oracle
    from paper_1410_0763_gb300 import workloads as wl
    case = wl.lognormal_iid(10, 2, seed=3)
    want, _, _ = oracle.sweep(case.kappa, case.src, 2)
    results = [np.load(tmp_path / f"jin_{r}.npy") for r in range(world)]
    for r in range(1, world):
        assert np.array_equal(results[r], results[0])      # every rank holds the same combination
    assert np.allclose(results[0], want, rtol=1e-13, atol=0)
    # the combination is the rank-order Kahan sum of the shares, cell by cell
    shares = np.stack([np.load(tmp_path / f"share_{r}.npy") for r in range(world)])
    assert np.array_equal(results[0], kahan_rows(shares))
