"""GPU parity of the incident-radiation boundaries (Sec. 4.3, Test 3) against
the FP64 oracle: the sweep with a boundary intensity on every entering ray,
the plane-parallel incident flux, and the RT / balance iteration lit by that
flux (with and without the diffuse field).

Bounds: the sweep as in test_sweep_gpu (FP64 1e-12, FP32 1e-5 relative);
the beam 4e-5 relative (FP32 optical depth summed over up to 28 cells, the
point sources' bound); the iteration 1e-4 relative in y and 1 - y, and an
iteration count within what a factor 2 in the residual near tol moves it by
at the oracle's contraction rate (one iteration when it converges fast).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1410_0763_gb300 import art, build
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


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def sweep_jin(kap, S, nside, i_bc, precision="fp32", **kw):
    dt = torch.float64 if precision == "fp64" else torch.float32
    k = torch.as_tensor(np.ascontiguousarray(kap), dtype=dt, device="cuda")
    s = torch.as_tensor(np.ascontiguousarray(S), dtype=dt, device="cuda")
    sw = art.ArtSweep(kap.shape, nside, 1, precision=precision, **kw)
    sw.set_boundary_intensity([i_bc])
    out = torch.empty_like(k)
    sw.set_fields(k, s)
    sw.sweep(J_in=out)
    torch.cuda.synchronize()
    sw.close()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("precision,tiles", [("fp64", (0, 0, 0)), ("fp32", (32, 16, 4)), ("fp32", (32, 8, 4)),
                                             ("fp32", (64, 8, 2)), ("fp32", (32, 16, 8))])
def test_sweep_with_boundary_intensity_matches_oracle(orc, precision, tiles):
    rng = np.random.default_rng(31)
    shape = (21, 26, 37)
    kap = f32(0.5 * np.exp(rng.standard_normal(shape)))
    S = f32(rng.random(shape))
    want, _, _ = orc.sweep(kap, S, 2, i_bc=0.7)
    tb, tc, blk = tiles
    got = sweep_jin(kap, S, 2, 0.7, precision, tile_b=tb, tile_c=tc, slab=blk)
    assert rel(got, want) < (1e-12 if precision == "fp64" else 1e-5)


def test_empty_box_keeps_the_boundary_intensity():
    z = np.zeros((19, 23, 29))
    got = sweep_jin(z, z, 4, 2.5)
    assert np.allclose(got, 2.5, rtol=1e-6, atol=0)


def test_graph_replay_follows_a_new_boundary_intensity(orc):
    rng = np.random.default_rng(32)
    shape = (16, 20, 24)
    kap = f32(0.5 * np.exp(rng.standard_normal(shape)))
    S = f32(rng.random(shape))
    k = torch.as_tensor(kap, dtype=torch.float32, device="cuda")
    s = torch.as_tensor(S, dtype=torch.float32, device="cuda")
    sw = art.ArtSweep(shape, 2, 1, graph=True)
    sw.set_fields(k, s)
    out = torch.empty_like(k)
    sw.sweep(J_in=out)
    vac = out.cpu().numpy().astype(np.float64)
    sw.set_boundary_intensity([1.5])
    sw.sweep(J_in=out)
    lit = out.cpu().numpy().astype(np.float64)
    sw.set_boundary_intensity(None)
    sw.sweep(J_in=out)
    back = out.cpu().numpy().astype(np.float64)
    sw.close()
    assert np.array_equal(back, vac)
    assert rel(vac, orc.sweep(kap, S, 2)[0]) < 1e-5
    assert rel(lit, orc.sweep(kap, S, 2, i_bc=1.5)[0]) < 1e-5


def test_batch_with_boundary_intensity(orc):
    rng = np.random.default_rng(33)
    shapes = [(12, 14, 16), (9, 11, 13)]
    cases = [(f32(0.5 * np.exp(rng.standard_normal(s))), f32(rng.random(s))) for s in shapes]
    sw = art.ArtSweep(shapes, [2, 1], 1)
    sw.set_boundary_intensity([0.4])
    k = torch.cat([torch.as_tensor(c[0].ravel(), dtype=torch.float32) for c in cases]).cuda()
    s = torch.cat([torch.as_tensor(c[1].ravel(), dtype=torch.float32) for c in cases]).cuda()
    out = torch.empty_like(k)
    sw.set_fields(k, s)
    sw.sweep(J_in=out)
    got = out.cpu().numpy().astype(np.float64)
    for (kap, S), off, ns in zip(cases, sw.offsets, [2, 1]):
        want, _, _ = orc.sweep(kap, S, ns, i_bc=0.4)
        assert rel(got[off:off + kap.size].reshape(kap.shape), want) < 1e-5
    sw.close()


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("direction", [1, -1])
@pytest.mark.parametrize("nbins", [1, 3])
def test_plane_source_matches_oracle(orc, axis, direction, nbins):
    rng = np.random.default_rng(40 + 3 * axis + nbins)
    shape = (20, 24, 28)
    kap = (0.3 * np.exp(rng.standard_normal((nbins,) + shape))).astype(np.float32)
    sigma = [6.3e-18, 3.1e-18, 1.2e-18][:nbins]
    flux = [1e6, 4e5, 1e5][:nbins]
    sw = art.ArtSweep(shape, 1, nbins, dx_cm=1e20)
    g = torch.empty(shape, dtype=torch.float32, device="cuda")
    sw.plane_source(torch.as_tensor(kap, device="cuda"), sigma, axis, direction, flux, g)
    torch.cuda.synchronize()
    sw.close()
    want = orc.plane_source(kap.astype(np.float64), sigma, axis, direction, flux)
    assert rel(g.cpu().numpy().astype(np.float64), want) < 4e-5


def _iterate_gpu(case, chem, tol=1e-6, max_iter=400, bins=None):
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    if bins is not None:
        sw.set_source_spectrum(bins[1], bins[0])
    sw.set_plane_source(*case.plane)
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device="cuda")
    y = torch.as_tensor(case.y0, dtype=torch.float64, device="cuda").clone()
    rep, hist = sw.iterate(nH, chem, [], y, tol=tol, max_iter=max_iter)
    sw.close()
    return y.cpu().numpy(), rep


@pytest.mark.parametrize("otsa", [False, True])
def test_iteration_lit_by_a_plane_flux_matches_oracle(orc, otsa):
    case = wl.shadow_clump(n=16, nside=2)
    chem = dict(case.chem, alphaA=case.chem["alphaB"]) if otsa else case.chem
    y, rep = _iterate_gpu(case, chem)
    y_o, it_o, hist_o, conv = orc.iterate(case.nH, case.nside, chem, case.pos, case.Q, case.y0, 1e-6, 400,
                                          plane=case.plane)
    assert conv and rep.converged
    assert abs(rep.iterations - it_o) <= _iteration_slack(hist_o)
    assert rel(y, y_o) < 1e-4
    assert rel(1 - y, 1 - y_o) < 1e-4


def _iteration_slack(hist):
    """Iterations by which the stopping point may move when the residual near
    tol differs by up to a factor 2 (FP32 rates against FP64): 1 + ln 2 /
    ln(1/q), q the oracle's contraction ratio over its last iterations."""
    q = float(np.exp(np.mean(np.log(hist[-6:] / hist[-7:-1]))))
    return 1 + (math.ceil(math.log(2.0) / -math.log(q)) if q < 1.0 else len(hist))


def test_iteration_lit_by_a_plane_flux_with_bins_matches_oracle(orc):
    case = wl.shadow_clump(n=16, nside=2)
    frac, sig, _ = wl.blackbody_bins()
    y, rep = _iterate_gpu(case, case.chem, bins=(frac, sig))
    y_o, it_o, hist_o, conv = orc.iterate(case.nH, case.nside, case.chem, case.pos, case.Q, case.y0, 1e-6, 400,
                                          sigma_bins=sig, frac_bins=frac, plane=case.plane)
    assert conv and rep.converged and abs(rep.iterations - it_o) <= _iteration_slack(hist_o)
    assert rel(y, y_o) < 1e-4
    assert rel(1 - y, 1 - y_o) < 1e-4


def test_invalid_arguments_are_rejected():
    shape = (8, 9, 10)
    sw = art.ArtSweep(shape, 1, 1, dx_cm=1e20)
    k = torch.zeros(shape, dtype=torch.float32, device="cuda")
    g = torch.empty_like(k)
    for axis, direction, flux in ((3, 1, [1e6]), (0, 0, [1e6]), (0, 1, [-1.0]), (1, -1, [float("nan")])):
        with pytest.raises(art.ArtError) as ex:
            sw.plane_source(k, [6.3e-18], axis, direction, flux, g)
        assert ex.value.status == art.ART_E_INVALID
    for bad in ([-1.0], [float("inf")]):
        with pytest.raises(art.ArtError):
            sw.set_boundary_intensity(bad)
    with pytest.raises(art.ArtError):
        sw.set_plane_source(0, 2, 1e6)
    with pytest.raises(art.ArtError):
        sw.ablation_sweep(0, g)            # no fields yet
    sw.close()
    sw = art.ArtSweep(shape, 1, 1, precision="fp64")
    sw.set_fields(torch.zeros(shape, dtype=torch.float64, device="cuda"),
                  torch.zeros(shape, dtype=torch.float64, device="cuda"))
    with pytest.raises(art.ArtError) as ex:
        sw.ablation_sweep(1, g)            # FP32 contexts only
    assert ex.value.status == art.ART_E_INVALID
    sw.close()
