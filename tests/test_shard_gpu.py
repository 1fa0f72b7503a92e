"""Direction shards on the GPU: contexts restricted to RING-index blocks give
additive J^in shares whose fixed-order sum (art_sum_partials) matches the
unsharded sweep; FP64 shares match the oracle's per-range sums."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1410_0763_gb300 import art, build
from paper_1410_0763_gb300 import dist as adist
from paper_1410_0763_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    art.load()


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def share(kap, S, nside, rng_, precision="fp32"):
    dt = torch.float64 if precision == "fp64" else torch.float32
    k = torch.as_tensor(kap, dtype=dt, device="cuda").reshape(-1)
    s = torch.as_tensor(S, dtype=dt, device="cuda").reshape(-1)
    sw = art.ArtSweep(kap.shape, nside, 1, precision=precision, dir_range=rng_)
    out = torch.empty_like(k)
    sw.set_fields(k, s)
    sw.sweep(J_in=out)
    torch.cuda.synchronize()
    st = sw.stats
    sw.close()
    return out, st


@pytest.mark.parametrize("world", [2, 3, 7])
def test_fp32_shards_sum_to_the_full_sweep(world):
    c = wl.grf(32, 4, seed=9)
    full, st_full = share(c.kappa, c.src, 4, None)
    parts, segs = [], 0
    for r in range(world):
        p, st = share(c.kappa, c.src, 4, adist.direction_block(4, r, world))
        parts.append(p)
        segs += st.segments
    assert segs == st_full.segments
    out = torch.empty_like(full)
    art.art_sum_partials(torch.stack(parts), out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), full.cpu().numpy()) < 2e-6


def test_fp64_shares_match_the_oracle_ranges(orc):
    c = wl.lognormal_iid(12, 2, seed=4)
    nd = 48
    for b, e in [(0, 17), (17, 48), (5, 6)]:
        got, _ = share(c.kappa, c.src, 2, (b, e), "fp64")
        acc, _ = orc.sweep_range(c.kappa, c.src, 2, b, e)
        assert rel(got.cpu().numpy().reshape(c.kappa.shape), acc / nd) < 1e-12


def test_shard_rejects_J_output():
    c = wl.grf(16, 1, seed=2)
    k = torch.as_tensor(c.kappa, dtype=torch.float32, device="cuda").reshape(-1)
    s = torch.as_tensor(c.src, dtype=torch.float32, device="cuda").reshape(-1)
    sw = art.ArtSweep(c.kappa.shape, 1, 1, dir_range=(0, 6))
    sw.set_fields(k, s)
    with pytest.raises(art.ArtError) as e:
        sw.sweep(J=torch.empty_like(k), J_in=torch.empty_like(k))
    assert e.value.status == art.ART_E_INVALID
    sw.close()


def _one_rank_sharded(q):
    import os
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    import socket
    with socket.socket() as s_:
        s_.bind(("127.0.0.1", 0))
        os.environ["MASTER_PORT"] = str(s_.getsockname()[1])
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        build.build()
        art.load()
        c = wl.grf(24, 3, seed=11)
        k = torch.as_tensor(c.kappa, dtype=torch.float32, device="cuda")
        s = torch.as_tensor(c.src, dtype=torch.float32, device="cuda")
        sh = adist.ShardedSweep(c.kappa.shape, 3, 1)
        sh.set_fields(k, s)
        jin = sh.jin(sh.share(torch.empty_like(k))).cpu().numpy()
        jin2 = sh.jin(sh.share(torch.empty_like(k))).cpu().numpy()
        sh.close()
        full, _ = share(c.kappa, c.src, 3, None)
        q.put((bool(np.array_equal(jin, full.cpu().numpy().reshape(jin.shape))), bool(np.array_equal(jin, jin2))))
    finally:
        dist.destroy_process_group()


def test_sharded_sweep_on_one_rank_equals_the_full_sweep():
    """ShardedSweep (the multi-GPU path of bench.py --shard) on a one-rank NCCL group: the
    context kept across calls, the exchange and the rank-order sum reduce to the full sweep,
    bit for bit, call after call."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_one_rank_sharded, args=(q,))
    p.start()
    p.join(300)
    assert p.exitcode == 0
    assert q.get(timeout=5) == (True, True)
