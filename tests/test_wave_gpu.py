"""GPU parity of the wavefront sweep (the default FP32 sweep with the paper's
cell average) against the FP64 oracle, through the C ABI.

Bar: 1e-5 relative per cell on J and J^in (the FP32 target), as for the
slab-block kernels.  Every compiled wavefront shape (art_options.variant 16-27:
8 x 8- or 8 x 16-column warp tiles (two or four rows per lane), 2 x 1, 2 x 2,
2 x 4 or 4 x 2 warps per CTA, 20 / 19 / 17 / 16 / 12 / 4
direction slots) runs on ragged grids that span several CTA tiles along both
transverse axes, with classes split into direction groups where they exceed
the slots.  The bounded waits are checked by stalling one tile on purpose: the
tiles downstream of it give up after the bound and the sweep reports
ART_E_TIMEOUT, after which the context sweeps correctly again.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1410_0763_gb300 import art, build
from paper_1410_0763_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

WAVE0 = 16   # art_options.variant of the first wavefront shape


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    art.load()


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def run(kap, src, nside, form=0, nbins=1, i_bc=None, check=True, **kw):
    shape = kap.shape[-3:]
    k = torch.as_tensor(np.ascontiguousarray(kap), dtype=torch.float32, device="cuda")
    s = torch.as_tensor(np.ascontiguousarray(src), dtype=torch.float32, device="cuda")
    sw = art.ArtSweep(shape, nside, nbins, field_form=form, **kw)
    if i_bc is not None:
        sw.set_boundary_intensity(i_bc)
    shard = kw.get("dir_range") is not None
    J = None if shard else torch.empty_like(k)   # a direction shard has J^in only
    Jin = torch.empty_like(k)
    sw.set_fields(k, s)
    sw.sweep(J, Jin)
    torch.cuda.synchronize()
    st = sw.check()
    stats = sw.stats
    sw.close()
    if check:
        assert st == art.ART_OK
    Jh = None if shard else J.cpu().numpy().astype(np.float64)
    return Jh, Jin.cpu().numpy().astype(np.float64), stats


def lognormal(shape, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return f32(scale * np.exp(rng.standard_normal(shape))), f32(rng.random(shape))


def test_default_fp32_context_uses_the_wavefront_sweep():
    kap, S = lognormal((12, 14, 16), 1)
    _, _, st = run(kap, S, 2)
    assert st.variant >= WAVE0 and st.launches == 2 and st.ctas_per_launch > 0


@pytest.mark.parametrize("variant,nside", [(WAVE0, 8), (WAVE0 + 1, 4), (WAVE0 + 1, 3), (WAVE0 + 2, 2),
                                           (WAVE0 + 2, 1), (WAVE0 + 3, 8), (WAVE0 + 4, 8), (WAVE0 + 2, 4),
                                           (WAVE0 + 1, 8), (WAVE0 + 3, 2), (WAVE0 + 4, 3),
                                           (WAVE0 + 5, 8), (WAVE0 + 5, 4), (WAVE0 + 6, 8), (WAVE0 + 6, 2),
                                           (WAVE0 + 7, 8), (WAVE0 + 7, 3), (WAVE0 + 8, 8), (WAVE0 + 8, 1),
                                           (WAVE0 + 9, 4), (WAVE0 + 9, 8), (WAVE0 + 10, 8), (WAVE0 + 10, 2), (WAVE0 + 10, 4),
                                           (WAVE0 + 11, 8), (WAVE0 + 11, 3)])
def test_ragged_grids_every_shape(orc, variant, nside):
    """Ragged against every tile (16 x 16 and 32 x 16 columns); shapes with fewer slots than a
    class's directions split it into groups."""
    shape = (21, 26, 37) if nside < 8 else (19, 23, 34)
    kap, S = lognormal(shape, 7 + nside)
    jin_o, j_o, _ = orc.sweep(kap, S, nside)
    J, Jin, st = run(kap, S, nside, variant=variant)
    assert st.variant == variant
    assert rel(Jin, jin_o) < 1e-5
    assert rel(J, j_o) < 1e-5


@pytest.mark.parametrize("scale", [0.02, 0.3, 3.0])
@pytest.mark.parametrize("variant", [0, WAVE0 + 1, WAVE0 + 10])
def test_thin_mixed_and_thick_media(orc, scale, variant):
    """Media whose warps take the series path, both paths, or the exponential path."""
    kap, S = lognormal((20, 24, 28), 11, scale)
    jin_o, j_o, _ = orc.sweep(kap, S, 4)
    J, Jin, _ = run(kap, S, 4, variant=variant)
    assert rel(Jin, jin_o) < 1e-5
    assert rel(J, j_o) < 1e-5


@pytest.mark.parametrize("variant", [0, WAVE0 + 6, WAVE0 + 10])
@pytest.mark.parametrize("hi", [0.0099, 0.0189, 0.094, 0.249, 0.499])
def test_second_thin_path(orc, variant, hi):
    """kappa uniform in [0, hi): a warp whose kappa stay below 0.019, 0.095 or 0.5 takes the
    economized series of degree 2, 3 or 5 (degrees 2 and 5 in shapes with the registers for
    them; the degree-3 and mixed paths in the others), each up to the top of its range,
    x = sqrt(3) hi."""
    rng = np.random.default_rng(19)
    shape = (22, 27, 35)
    kap, S = f32(hi * rng.random(shape)), f32(rng.random(shape))
    jin_o, j_o, _ = orc.sweep(kap, S, 4)
    J, Jin, _ = run(kap, S, 4, variant=variant)
    assert rel(Jin, jin_o) < 1e-5
    assert rel(J, j_o) < 1e-5


def test_grf_64_nside4(orc):
    c = wl.grf(64, 4)
    kap, S = f32(c.kappa), f32(c.src)
    jin_o, j_o, _ = orc.sweep(kap, S, 4)
    J, Jin, _ = run(kap, S, 4)
    assert rel(Jin, jin_o) < 1e-5
    assert rel(J, j_o) < 1e-5


def test_emissivity_form_with_transparent_cells(orc):
    rng = np.random.default_rng(9)
    shape = (18, 22, 17)
    kap = 0.3 * np.exp(rng.standard_normal(shape))
    kap[rng.random(shape) < 0.3] = 0.0
    kap = f32(kap)
    eps = f32(rng.random(shape))
    jin_o, j_o, _ = orc.sweep(kap, eps, 3, field_form=1)
    J, Jin, _ = run(kap, eps, 3, form=1)
    assert rel(Jin, jin_o) < 1e-5
    assert rel(J, j_o) < 1e-5


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 2, 2), (1, 5, 7), (9, 1, 1), (1, 1, 13), (3, 40, 1), (1, 37, 41),
                                   (257, 6, 5), (5, 9, 257)])
@pytest.mark.parametrize("variant,nside,i_bc", [(0, 1, None), (0, 2, 0.8), (0, 4, None), (WAVE0 + 11, 4, 0.5)])
def test_degenerate_grids(orc, shape, variant, nside, i_bc):
    """A single cell, a 2^3 cube, planes, lines, thin slabs and long bars (every transverse tile
    ragged or of one column; sweeps of one to 257 slabs), with and without a boundary intensity;
    the default shape and the four-row shape.  With vacuum boundaries a single cell receives no
    intensity (J^in = 0 exactly)."""
    kap, S = lognormal(shape, 21)
    jin_o, j_o, _ = orc.sweep(kap, S, nside, i_bc=0.0 if i_bc is None else i_bc)
    J, Jin, st = run(kap, S, nside, i_bc=None if i_bc is None else [i_bc], variant=variant)
    assert st.variant >= WAVE0
    assert rel(Jin, jin_o) < 1e-5
    assert rel(J, j_o) < 1e-5
    if shape == (1, 1, 1) and i_bc is None:
        assert Jin[0, 0, 0] == 0.0


def test_boundary_intensity(orc):
    kap, S = lognormal((17, 20, 23), 12)
    jin_o, j_o, _ = orc.sweep(kap, S, 2, i_bc=0.8)
    J, Jin, _ = run(kap, S, 2, i_bc=[0.8])
    assert rel(Jin, jin_o) < 1e-5
    assert rel(J, j_o) < 1e-5


@pytest.mark.parametrize("nbins,boundary", [(3, 0.0), (3, 0.7), (9, 0.0)])
def test_multiple_bins(orc, nbins, boundary):
    """Up to 8 bins go through one launch (their units in bin order under one ticket counter,
    each bin with its fields, boundary intensity, edge buffers, flags and J partials); more
    bins through one launch each.  Every bin against the oracle."""
    shape = (12, 14, 16)
    rng = np.random.default_rng(5 + nbins)
    kap = f32((0.1 + 0.1 * np.arange(nbins))[:, None, None, None] * np.exp(rng.standard_normal((nbins,) + shape)))
    S = f32(rng.random((nbins,) + shape))
    sw = art.ArtSweep(shape, 3, nbins)
    if boundary:
        sw.set_boundary_intensity([boundary * (b + 1) for b in range(nbins)])
    k = torch.as_tensor(np.ascontiguousarray(kap), dtype=torch.float32, device="cuda")
    s = torch.as_tensor(np.ascontiguousarray(S), dtype=torch.float32, device="cuda")
    J, Jin = torch.empty_like(k), torch.empty_like(k)
    sw.set_fields(k, s)
    sw.sweep(J, Jin)
    assert sw.check() == art.ART_OK
    st = sw.stats
    sw.close()
    assert st.variant >= WAVE0 and st.bins_per_launch == (nbins if nbins <= 8 else 1)
    J, Jin = J.cpu().numpy().astype(np.float64), Jin.cpu().numpy().astype(np.float64)
    for b in range(nbins):
        jin_o, j_o, _ = orc.sweep(kap[b], S[b], 3, i_bc=boundary * (b + 1))
        assert rel(Jin[b], jin_o) < 1e-5
        assert rel(J[b], j_o) < 1e-5


def test_wave_counters():
    """art_wave_counters: zeros unless the library was built with ART_WAVE_STATS=1; there, the
    warp cycles at the step barriers are a part of the cycles in the units, and a second read
    (after the clear) is zero."""
    import os
    shape = (20, 22, 24)
    kap, S = lognormal(shape, 3)
    sw = art.ArtSweep(shape, 4)
    k = torch.as_tensor(np.ascontiguousarray(kap), dtype=torch.float32, device="cuda")
    s = torch.as_tensor(np.ascontiguousarray(S), dtype=torch.float32, device="cuda")
    sw.set_fields(k, s)
    sw.sweep(None, torch.empty_like(k))
    assert sw.check() == art.ART_OK
    c1, c2 = sw.wave_counters(), sw.wave_counters()
    sw.close()
    assert all(v == 0 for v in c2.values())
    if os.environ.get("ART_WAVE_STATS") == "1":
        assert 0 < c1["barrier_cycles"] < c1["unit_cycles"]
    else:
        assert all(v == 0 for v in c1.values())


def test_direction_shards_add_up(orc):
    kap, S = lognormal((14, 15, 16), 13)
    nd = 12 * 3 * 3
    full = np.zeros(kap.shape)
    cuts = [0, 31, 70, nd]
    for a, b in zip(cuts[:-1], cuts[1:]):
        _, jin, st = run(kap, S, 3, dir_range=(a, b))
        assert st.variant >= WAVE0
        full += jin
    jin_o, _, _ = orc.sweep(kap, S, 3)
    assert rel(full, jin_o) < 1e-5


def test_deterministic_bitwise():
    kap, S = lognormal((24, 20, 28), 14)
    a = run(kap, S, 4)[1]
    b = run(kap, S, 4)[1]
    assert np.array_equal(a, b)


def test_batch_of_uneven_grids_matches_single_contexts(orc):
    shapes = [(9, 11, 13), (20, 16, 18), (12, 12, 12)]
    nsides = [2, 4, 3]
    rng = np.random.default_rng(15)
    ks = [f32(0.5 * np.exp(rng.standard_normal(s))) for s in shapes]
    ss = [f32(rng.random(s)) for s in shapes]
    kap = np.concatenate([k.ravel() for k in ks])
    src = np.concatenate([s.ravel() for s in ss])
    sw = art.ArtSweep(shapes, nsides, 1)
    variant = sw.stats.variant
    assert variant >= WAVE0
    k = torch.as_tensor(kap, dtype=torch.float32, device="cuda")
    s = torch.as_tensor(src, dtype=torch.float32, device="cuda")
    Jin = torch.empty_like(k)
    sw.set_fields(k, s)
    sw.sweep(None, Jin)
    assert sw.check() == art.ART_OK
    sw.close()
    got = Jin.cpu().numpy().astype(np.float64)
    off = 0
    for kk, s_, ns in zip(ks, ss, nsides):
        n = kk.size
        jin_o, _, _ = orc.sweep(kk, s_, ns)
        assert rel(got[off:off + n].reshape(kk.shape), jin_o) < 1e-5
        single = run(kk, s_, ns, variant=variant)[1]   # the same kernel shape: the same arithmetic
        assert np.array_equal(got[off:off + n].reshape(kk.shape), single)
        off += n


def test_graph_replay_matches_plain_launches():
    kap, S = lognormal((16, 18, 20), 16)
    a = run(kap, S, 4)[1]
    b = run(kap, S, 4, graph=True)[1]
    assert np.array_equal(a, b)


def test_a_stalled_tile_times_out_and_the_context_recovers(orc):
    """A unit that never publishes its progress: the tiles downstream of it wait until the
    bound (0.2 s), the sweep reports ART_E_TIMEOUT, and the next sweep is correct."""
    kap, S = lognormal((40, 36, 44), 17)
    k = torch.as_tensor(kap, dtype=torch.float32, device="cuda")
    s = torch.as_tensor(S, dtype=torch.float32, device="cuda")
    sw = art.ArtSweep(kap.shape, 2, 1)
    sw.set_fields(k, s)
    Jin = torch.empty_like(k)
    sw.set_wait(0.2, 0)   # unit 0 starts a tile diagonal: every class has tiles downstream of it
    sw.sweep(None, Jin)
    assert sw.check() == art.ART_E_TIMEOUT
    sw.set_wait(2.0, -1)
    sw.sweep(None, Jin)
    assert sw.check() == art.ART_OK
    sw.close()
    jin_o, _, _ = orc.sweep(kap, S, 2)
    assert rel(Jin.cpu().numpy().astype(np.float64), jin_o) < 1e-5


def test_a_stalled_tile_of_a_later_bin_times_out_and_the_context_recovers(orc):
    """The same with 3 bins in one launch: the stalled unit is the first of the last bin (its
    ticket follows all units of the earlier bins); the context recovers and every bin is
    correct afterwards."""
    rng = np.random.default_rng(23)
    shape = (40, 36, 44)
    kap = f32(0.3 * np.exp(rng.standard_normal((3,) + shape)))
    S = f32(rng.random((3,) + shape))
    k = torch.as_tensor(kap, dtype=torch.float32, device="cuda")
    s = torch.as_tensor(S, dtype=torch.float32, device="cuda")
    sw = art.ArtSweep(shape, 2, 3)
    st = sw.stats
    assert st.bins_per_launch == 3
    sw.set_fields(k, s)
    Jin = torch.empty_like(k)
    sw.set_wait(0.2, 2 * st.ctas_per_launch)   # ticket of unit 0 of bin 2
    sw.sweep(None, Jin)
    assert sw.check() == art.ART_E_TIMEOUT
    sw.set_wait(2.0, -1)
    sw.sweep(None, Jin)
    assert sw.check() == art.ART_OK
    sw.close()
    got = Jin.cpu().numpy().astype(np.float64)
    for b in range(3):
        jin_o, _, _ = orc.sweep(kap[b], S[b], 2)
        assert rel(got[b], jin_o) < 1e-5


def clump_boundary_cells(rho, rng, count):
    """Cells of the clumpy medium whose density differs from a face neighbour's by more than
    10x (the surfaces of the overdense spheres), `count` of them at random."""
    jump = np.zeros(rho.shape, dtype=bool)
    for ax in range(3):
        hi = np.maximum(rho, np.roll(rho, 1, ax)) > 10.0 * np.minimum(rho, np.roll(rho, 1, ax))
        edge = [slice(None)] * 3
        edge[ax] = 0
        hi[tuple(edge)] = False            # no wrap-around across the box faces
        jump |= hi
    idx = np.flatnonzero(jump)
    return rng.choice(idx, min(count, idx.size), replace=False)


def test_clumpy_256_four_bins_sampled_cells(orc):
    """The headline workload at full size (256^3 clumpy medium, N_side 8, 4 bins), in the launch
    configuration the benchmark times (all bins in one context, autotuned variant): J^in of
    1000 cells per bin against the oracle, computed cell by cell -- 400 on the clumps'
    surfaces, the 8 corners, cells on every face and the rest uniform.  FP32 bar at 256^3:
    1e-4 relative per cell."""
    c = wl.clumpy_sweep()
    kap, S = f32(c.kappa), f32(c.src)
    nb, n = kap.shape[0], kap.shape[-1]
    k = torch.as_tensor(np.ascontiguousarray(kap), dtype=torch.float32, device="cuda")
    s = torch.as_tensor(np.ascontiguousarray(S), dtype=torch.float32, device="cuda")
    sw = art.ArtSweep((n, n, n), 8, nb)
    sw.set_fields(k, s)
    sw.autotune(1)
    Jin = torch.empty_like(k)
    sw.sweep(None, Jin)
    torch.cuda.synchronize()
    assert sw.check() == art.ART_OK
    variant = sw.stats.variant
    sw.close()
    Jin = Jin.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(12)
    rho = S[0]
    corners = [z * n * n + y * n + x for z in (0, n - 1) for y in (0, n - 1) for x in (0, n - 1)]
    faces = []
    for ax in range(3):
        for side in (0, n - 1):
            p = rng.integers(0, n, size=(10, 3))
            p[:, ax] = side
            faces += list(p[:, 0] * n * n + p[:, 1] * n + p[:, 2])
    edge = clump_boundary_cells(rho, rng, 400)
    rest = rng.choice(n ** 3, 1000 - len(corners) - len(faces) - edge.size, replace=False)
    cells = np.unique(np.concatenate([corners, faces, edge, rest]).astype(np.int64))
    assert cells.size >= 990 and edge.size == 400
    for b in range(nb):
        ref = orc.jin_cells(kap[b], S[b], 8, cells, nthreads=orc.default_threads())
        got = Jin[b].ravel()[cells]
        assert np.all(ref > 0)
        err = np.abs(got - ref) / ref
        assert err.max() < 1e-4, (b, variant, float(err.max()), int(cells[np.argmax(err)]))
