"""GPU parity of the point sources (App. A), the FP64 balance (App. B) and the
RT/balance iteration (App. D) against the FP64 oracle.

Point sources: all FP32 (source position split into its integer cell and
an FP32 fraction, rate constant folded on the host in FP64); within 4e-5
relative of the oracle on the FP32-rounded opacities.  Iteration: the converged neutral fraction within
1e-4 relative of the oracle's (the FP32 sweep and march errors of ~1e-6 are
amplified by the fixed point), same iteration count within one.  At the full
128^3 / N_side 8 configuration the GPU's converged state is checked as a
fixed point of the paper's equations evaluated by the oracle at sampled cells.
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


@pytest.mark.parametrize("nbins", [1, 3])
def test_point_sources_match_oracle(orc, nbins):
    rng = np.random.default_rng(21 + nbins)
    shape = (20, 24, 28)
    kap = (0.3 * np.exp(rng.standard_normal((nbins,) + shape))).astype(np.float32)
    nz, ny, nx = shape
    sources = [(nx / 2, ny / 2, nz / 2, 3e48),                 # on a vertex: tie-break
               (3.37, 17.81, 5.12, 1e48),
               (25.5, 0.25, 19.5, 2e48)]                       # on a cell-centre line
    sigma = [6.3e-18, 3.1e-18, 1.2e-18][:nbins]
    Qb = rng.uniform(0.5, 1.5, (3, nbins)) * np.array([s[3] for s in sources])[:, None]
    dx = 1.6e20
    sw = art.ArtSweep(shape, 2, nbins, dx_cm=dx)
    k = torch.as_tensor(kap, device="cuda")
    g = torch.empty(shape, dtype=torch.float32, device="cuda")
    sw.point_sources(k, sigma, sources, g, Qb=Qb)
    torch.cuda.synchronize()
    sw.close()
    ref = orc.point_sources(kap.astype(np.float64), sigma, np.array([s[:3] for s in sources]), Qb, dx)
    # FP32 geometry: each plane-crossing parameter T along a ray is rounded to
    # a few ulp of T, so a cell's optical depth is off by about
    # u * sum_c T_c |kappa_c - kappa_c+1| over the ray's crossings, and
    # e^-tau by the same amount relative.  On this medium (tau <= 33 along
    # rays of at most 43 cells) the worst of the 40k rays is ~1.5e-5.
    err = rel(g.cpu().numpy().astype(np.float64), ref)
    print(f"\nPRECISION point sources, {nbins} bin(s): max relative error {err:.2e}")
    assert err < 4e-5


def test_point_sources_thin_limit():
    # kappa -> 0: Gamma -> Q sigma / (4 pi r^2) far from the source (inverse square)
    shape = (32, 32, 32)
    sw = art.ArtSweep(shape, 1, 1, dx_cm=1e20)
    k = torch.zeros(shape, dtype=torch.float32, device="cuda")
    g = torch.empty_like(k)
    src = (1.3, 2.2, 0.7, 1e50)
    sw.point_sources(k, [6.3e-18], [src], g)
    torch.cuda.synchronize()
    sw.close()
    gh = g.cpu().numpy()
    for (x, y, z) in [(30, 5, 2), (20, 28, 31), (31, 31, 31)]:
        r = math.dist((x + 0.5, y + 0.5, z + 0.5), src[:3]) * 1e20
        assert gh[z, y, x] == pytest.approx(1e50 * 6.3e-18 / (4 * math.pi * r * r), rel=2e-3)


def _run_gpu_iteration(case, tol=1e-6, max_iter=300):
    shape = case.nH.shape
    sw = art.ArtSweep(shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device="cuda")
    y = torch.as_tensor(case.y0, dtype=torch.float64, device="cuda").clone()
    srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
    rep, hist = sw.iterate(nH, case.chem, srcs, y, tol=tol, max_iter=max_iter)
    torch.cuda.synchronize()
    sw.close()
    return y.cpu().numpy(), rep, hist


@pytest.mark.parametrize("n,nside,box", [(16, 2, 1.6), (20, 2, 3.0)])
def test_iteration_matches_oracle(orc, n, nside, box):
    case = wl.hii_region(n=n, nside=nside, box_kpc=box)
    y_gpu, rep, hist = _run_gpu_iteration(case)
    y_orc, it_orc, hist_orc, conv = orc.iterate(case.nH, case.nside, case.chem, case.pos, case.Q, case.y0,
                                                1e-6, 300)
    assert conv and rep.converged
    assert abs(rep.iterations - it_orc) <= 1
    assert rel(y_gpu, y_orc) < 1e-4
    assert rel(1 - y_gpu, 1 - y_orc) < 1e-4
    # the residual history follows the oracle's until the last few iterations
    k = min(len(hist), len(hist_orc)) - 3
    assert np.allclose(hist[:k], hist_orc[:k], rtol=1e-3, atol=1e-9)


def test_full_size_hii_region_is_a_fixed_point(orc):
    case = wl.hii_region()          # 128^3, N_side 8, Q = 5e48 at the centre
    y, rep, hist = _run_gpu_iteration(case, max_iter=200)
    assert rep.converged and hist[-1] < 1e-6
    assert np.all((y > 0) & (y < 1))
    # R_S = 5.4 kpc exceeds the half box: the whole box is ionized
    assert np.max(y) < 0.1
    ch = case.chem
    nH = case.nH
    ne = (1 - y) * nH
    kap = (y * nH * ch["sigma0"] * ch["dx"]).astype(np.float32).astype(np.float64)
    dalpha = ch["alphaA"] - ch["alphaB"]
    eps = (ch["h"] * ch["nu0"] * dalpha * ne * ne * ch["dx"] / (4 * math.pi * ch["dnu"]))
    eps = eps.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(3)
    cells = rng.choice(y.size, 24, replace=False)
    cells[:3] = [0, y.size - 1, (64 * 128 + 64) * 128 + 64]
    jin = orc.jin_cells(kap, eps, case.nside, cells, field_form=1)
    G = orc.band_integral(ch["sigma0"], ch["h"], ch["nu0"], ch["nu0"] + ch["dnu"])
    gpt = orc.point_sources(kap, [ch["sigma0"]], case.pos, case.Q.reshape(-1, 1), ch["dx"]).ravel()[cells]
    g = 4 * math.pi * G * jin + gpt
    y_check = orc.balance_eq(nH.ravel()[cells], ch["alphaB"], ch["gcoll"], g)
    assert rel(y.ravel()[cells], y_check) < 1e-4


def test_full_size_clumpy_medium_with_bins_is_a_fixed_point(orc):
    """The clumpy 256^3 medium, N_side 8, 8 sources over 4 blackbody bins, as
    the benchmark solves it: the GPU's converged state satisfies the balance
    at sampled cells with the oracle's J^in and point-source rates there."""
    case = wl.clumpy()
    frac, sig, _ = wl.blackbody_bins()
    ch = case.chem
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=ch["dx"])
    sw.set_source_spectrum(sig, frac)
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device="cuda")
    y = torch.as_tensor(case.y0, dtype=torch.float64, device="cuda").clone()
    srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
    rep, hist = sw.iterate(nH, ch, srcs, y, tol=1e-6, max_iter=400)
    sw.close()
    assert rep.converged
    y = y.cpu().numpy()
    ne = (1 - y) * case.nH
    kap = (y * case.nH * ch["sigma0"] * ch["dx"]).astype(np.float32).astype(np.float64)
    eps = (ch["h"] * ch["nu0"] * (ch["alphaA"] - ch["alphaB"]) * ne * ne * ch["dx"] / (4 * math.pi * ch["dnu"]))
    eps = eps.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(5)
    # cells across the range of ionization: half drawn from the neutral gas, half from the ionized
    flat = y.ravel()
    order = np.argsort(flat)
    cells = np.concatenate([rng.choice(order[: flat.size // 2], 8, replace=False),
                            rng.choice(order[flat.size // 2:], 8, replace=False)])
    jin = orc.jin_cells(kap, eps, case.nside, cells, field_form=1)
    G = orc.band_integral(ch["sigma0"], ch["h"], ch["nu0"], ch["nu0"] + ch["dnu"])
    kapb = np.stack([kap * (s / ch["sigma0"]) for s in sig])
    Qb = np.outer(case.Q, frac)
    gpt = orc.point_sources_cells(kapb, sig, case.pos, Qb, ch["dx"], cells)
    g = 4 * math.pi * G * jin + gpt
    y_check = orc.balance_eq(case.nH.ravel()[cells], ch["alphaB"], ch["gcoll"], g)
    assert rel(flat[cells], y_check) < 1e-4
    assert rel(1 - flat[cells], 1 - y_check) < 1e-4


def test_iteration_with_source_bins_matches_oracle(orc):
    """Point sources over three frequency bins (blackbody fractions, photon-weighted
    cross sections) inside the RT / balance iteration."""
    case = wl.hii_region(n=16, nside=2, box_kpc=1.6)
    frac, sig, _ = wl.blackbody_bins(edges_ev=(13.6, 24.6, 54.4, 200.0))
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    sw.set_source_spectrum(sig, frac)
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device="cuda")
    y = torch.as_tensor(case.y0, dtype=torch.float64, device="cuda").clone()
    srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
    rep, hist = sw.iterate(nH, case.chem, srcs, y, tol=1e-6, max_iter=300)
    sw.close()
    y_o, it_o, _, conv = orc.iterate(case.nH, case.nside, case.chem, case.pos, case.Q, case.y0, 1e-6, 300,
                                     sigma_bins=sig, frac_bins=frac)
    assert conv and rep.converged and abs(rep.iterations - it_o) <= 1
    yg = y.cpu().numpy()
    assert rel(yg, y_o) < 1e-4
    assert rel(1 - yg, 1 - y_o) < 1e-4


# --- on-the-spot approximation (Sec. 2.1, Eq. on_the_spot): alpha_A = alpha_B ---

def _stromgren_case(n, nside=2, nH=1e-1, Q=5e48, size_rs=2.5):
    rs = (3 * Q / (4 * math.pi * nH * nH * wl.ALPHA_B_1E4)) ** (1 / 3)
    dx = size_rs * rs / n
    case = wl.hii_region(n=n, nside=nside, box_kpc=n * dx / wl.KPC, nH=nH, Q=Q)
    return case, rs, dx


def _otsa(chem):
    return dict(chem, alphaA=chem["alphaB"])


def test_otsa_iteration_matches_oracle(orc):
    case, _, _ = _stromgren_case(20)
    case.chem = _otsa(case.chem)
    y_gpu, rep, hist = _run_gpu_iteration(case)
    y_o, it_o, hist_o, conv = orc.iterate(case.nH, case.nside, case.chem, case.pos, case.Q, case.y0, 1e-6, 300)
    assert conv and rep.converged and abs(rep.iterations - it_o) <= 1
    assert rel(y_gpu, y_o) < 1e-4
    assert rel(1 - y_gpu, 1 - y_o) < 1e-4


def test_otsa_stromgren_sphere_and_case_b_photon_balance(orc):
    """64^3, uniform n_H = 0.1 cm^-3, Q = 5e48 s^-1 at the centre, box 2.5 R_S.
    The converged on-the-spot state holds a case-B Stromgren sphere, and summed
    over the box, case-B recombinations equal photo- plus collisional
    ionizations with the oracle's point-source rates at that state."""
    case, rs, dx = _stromgren_case(64)
    case.chem = _otsa(case.chem)
    y, rep, hist = _run_gpu_iteration(case, max_iter=300)
    assert rep.converged
    ch = case.chem
    vol = np.sum(1 - y) * dx ** 3
    assert vol == pytest.approx(4 * math.pi / 3 * rs ** 3, rel=0.05)
    nH = case.nH
    ne, nHI = (1 - y) * nH, y * nH
    kap = (nHI * ch["sigma0"] * dx).astype(np.float32).astype(np.float64)
    gpt = orc.point_sources(kap, [ch["sigma0"]], case.pos, case.Q.reshape(-1, 1), dx)
    recomb = np.sum(ch["alphaB"] * ne * ne)
    ioniz = np.sum(nHI * (ch["gcoll"] * ne + gpt))
    assert recomb == pytest.approx(ioniz, rel=1e-4)


def test_diffuse_field_enlarges_ionized_region_gpu():
    """Sec. 4.1: with the recombination radiation transferred (alpha_A > alpha_B)
    the ionized region is larger than on the spot."""
    case, _, _ = _stromgren_case(32)
    y_diff, rep_d, _ = _run_gpu_iteration(case)
    case.chem = _otsa(case.chem)
    y_otsa, rep_o, _ = _run_gpu_iteration(case)
    assert rep_d.converged and rep_o.converged
    assert np.all(y_diff <= y_otsa * (1 + 1e-4))
    assert np.sum(1 - y_diff) > 1.02 * np.sum(1 - y_otsa)


@pytest.mark.parametrize("omega", [0.8, 1.3])
def test_relaxed_iteration_reaches_the_oracle_fixed_point(orc, omega):
    """Over-relaxation changes the path, not the fixed point: the relaxed GPU
    iteration, run to 1e-8, ends within 1e-4 of the oracle's plain iteration
    run to 1e-10."""
    case = wl.hii_region(n=16, nside=2, box_kpc=1.6)
    srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    sw.set_relaxation(omega)
    y = torch.as_tensor(case.y0, dtype=torch.float64, device="cuda").clone()
    rep, _ = sw.iterate(torch.as_tensor(case.nH, dtype=torch.float64, device="cuda"), case.chem, srcs, y, tol=1e-8,
                        max_iter=400)
    for bad in (0.0, 2.0, float("nan")):
        with pytest.raises(art.ArtError) as ex:
            sw.set_relaxation(bad)
        assert ex.value.status == art.ART_E_INVALID
    sw.close()
    y_orc, it_orc, _, conv = orc.iterate(case.nH, case.nside, case.chem, case.pos, case.Q, case.y0, 1e-10, 400)
    assert conv and rep.converged
    yg = y.cpu().numpy()
    assert rel(yg, y_orc) < 1e-4 and rel(1 - yg, 1 - y_orc) < 1e-4
