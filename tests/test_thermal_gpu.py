"""GPU time-dependent mode with the energy equation (App. C) against the FP64
oracle and the invariants its pins use.

* Cooling only (no sources, hot ionized gas): the device fits and the
  implicit energy solve match the oracle to 1e-9 (FP64 on both sides, no
  FP32 rates involved).
* Fixed step sequences with a source, on the spot and with the diffuse field
  transferred, with a plane flux over 4 blackbody bins, and in Test 2's
  geometry (a source beside a dense cold clump): y, 1 - y and T follow the
  oracle within 1e-4 (the FP32 rates' error, amplified by the chemistry as
  in the fixed-temperature mode).
* Neither heating nor cooling: the specific energy (2 - y) T of every cell is
  conserved to rounding.
* A heated Stromgren region (32^3, on the spot): its volume is the Stromgren
  volume taken with alpha_B at the ionized gas's mean temperature.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1410_0763_gb300 import art, build
from paper_1410_0763_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

KB = 1.380649e-16
EV = 1.602176634e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    art.load()


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda").clone()


def _srcs(case):
    return [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]


def _th(**kw):
    d = dict(kB=KB, e_bin=[3.72 * EV], e_diff=0.41 * EV, z=0.0, T_min=10.0, T_max=1e9, cool_mask=31,
             on_the_spot=0)
    d.update(kw)
    return d


def _ctx(case, bins=None):
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    if bins is not None:
        sw.set_source_spectrum(bins[1], bins[0])
    if case.plane is not None:
        sw.set_plane_source(*case.plane)
    return sw


def test_cooling_only_matches_oracle_in_fp64(orc):
    case = wl.hii_region(n=8, nside=1, box_kpc=1.6, nH=1e-2)
    rng = np.random.default_rng(4)
    y0 = rng.uniform(0.0, 0.3, case.nH.shape)
    T0 = 10 ** rng.uniform(4.0, 6.5, case.nH.shape)
    th = _th(on_the_spot=1, z=3.0)
    t_end = 2e13
    sw = _ctx(case)
    y, T = _dev(y0), _dev(T0)
    rep = sw.evolve_thermal(_dev(case.nH), case.chem, th, [], y, T, t_end, F=1.0, eps_iter=1e-10)
    yo, To, steps, iters, t, dts, rc = orc.evolve_thermal(case.nH, 1, case.chem, th, np.zeros((0, 3)), np.zeros(0),
                                                          y0, T0, t_end, F=1.0, eps_iter=1e-10)
    assert rc == 0 and rep.converged and rep.steps == steps
    assert rel(T.cpu().numpy(), To) < 1e-9
    assert rel(y.cpu().numpy(), yo) < 1e-9
    assert np.all(To < T0)                     # every cell cooled
    sw.close()


@pytest.mark.parametrize("otsa", [1, 0])
def test_fixed_steps_with_a_source_match_oracle(orc, otsa):
    case = wl.hii_region(n=16, nside=2, box_kpc=1.6)
    th = _th(on_the_spot=otsa, e_diff=wl.diffuse_band_heat(case.chem))
    T0 = np.full(case.nH.shape, 100.0)
    t_rec = 1.0 / (case.chem["alphaB"] * 1e-3)
    dt = t_rec / 400
    sw = _ctx(case)
    nH, y, T = _dev(case.nH), _dev(case.y0), _dev(T0)
    y_o, T_o = case.y0.copy(), T0.copy()
    for _ in range(3):        # the state carries over between calls
        rep = sw.evolve_thermal(nH, case.chem, th, _srcs(case), y, T, 4 * dt, dt_fixed=dt, eps_iter=1e-6)
        assert rep.steps == 4 and rep.converged and rep.sub_overflow == 0
        y_o, T_o, steps, iters, t, dts, rc = orc.evolve_thermal(case.nH, case.nside, case.chem, th, case.pos, case.Q,
                                                                y_o, T_o, 4 * dt, dt_fixed=dt, eps_iter=1e-9)
        assert rc == 0 and steps == 4
        yg, Tg = y.cpu().numpy(), T.cpu().numpy()
        assert rel(yg, y_o) < 1e-4 and rel(1 - yg, 1 - y_o) < 1e-4
        assert rel(Tg, T_o) < 1e-4
    assert T_o.max() > 5e3                     # the source has heated the gas near it
    assert (rep.sweeps == 0) == bool(otsa)
    sw.close()


def test_fixed_steps_with_a_plane_flux_and_bins_match_oracle(orc):
    case = wl.shadow_clump(n=16, nside=2)
    frac, sig, _ = wl.blackbody_bins()
    th = _th(e_bin=list(wl.blackbody_heat()), e_diff=wl.diffuse_band_heat(case.chem))
    T0 = np.full(case.nH.shape, 100.0)
    t_rec = 1.0 / (case.chem["alphaB"] * 2e-4)
    dt = t_rec / 2000
    sw = _ctx(case, bins=(frac, sig))
    nH, y, T = _dev(case.nH), _dev(case.y0), _dev(T0)
    rep = sw.evolve_thermal(nH, case.chem, th, [], y, T, 6 * dt, dt_fixed=dt, eps_iter=1e-6)
    y_o, T_o, steps, *_ = orc.evolve_thermal(case.nH, case.nside, case.chem, th, case.pos, case.Q, case.y0, T0,
                                             6 * dt, dt_fixed=dt, eps_iter=1e-9, sigma_bins=sig, frac_bins=frac,
                                             plane=case.plane)
    assert rep.converged and rep.steps == steps == 6
    yg, Tg = y.cpu().numpy(), T.cpu().numpy()
    assert rel(yg, y_o) < 1e-4 and rel(1 - yg, 1 - y_o) < 1e-4
    assert rel(Tg, T_o) < 1e-4
    assert T_o.max() > 1e4                     # the hard bins heat the lit face
    sw.close()


def test_specific_energy_is_conserved_without_heating_or_cooling():
    case = wl.hii_region(n=8, nside=1, box_kpc=0.5, nH=1e-2)
    rng = np.random.default_rng(3)
    y0 = rng.uniform(0.0, 0.5, case.nH.shape)
    T0 = rng.uniform(5e3, 3e4, case.nH.shape)
    th = _th(on_the_spot=1, cool_mask=0, e_bin=[0.0], e_diff=0.0)
    sw = _ctx(case)
    y, T = _dev(y0), _dev(T0)
    rep = sw.evolve_thermal(_dev(case.nH), case.chem, th, [], y, T, 2e14, F=1.0, eps_iter=1e-9)
    assert rep.converged and rep.steps > 3
    yg, Tg = y.cpu().numpy(), T.cpu().numpy()
    assert np.max(np.abs(yg - y0)) > 0.05
    assert np.allclose((2 - yg) * Tg, (2 - y0) * T0, rtol=1e-12)
    sw.close()


def test_heated_stromgren_volume_gpu():
    nH, Q = 1e-3, 5e48
    case = wl.hii_region(n=32, nside=1, box_kpc=6.6, nH=nH, Q=Q, source_at="corner")
    th = _th(on_the_spot=1, e_bin=[3.72 * EV])
    sw = _ctx(case)
    y, T = _dev(case.y0), _dev(np.full(case.nH.shape, 100.0))
    rep = sw.evolve_thermal(_dev(case.nH), case.chem, th, _srcs(case), y, T, 4.0 / (2.59e-13 * nH), F=1.0)
    assert rep.converged and rep.sweeps == 0
    yg, Tg = y.cpu().numpy(), T.cpu().numpy()
    T_ion = float(np.sum(Tg * (1 - yg)) / np.sum(1 - yg))
    assert 5e3 < T_ion < 3e4
    aB = 2.753e-14 * (2 * 157807.0 / T_ion) ** 1.5 / (1 + (2 * 157807.0 / T_ion / 2.74) ** 0.407) ** 2.242
    vol = 8 * float(np.sum(1 - yg)) * case.chem["dx"] ** 3
    assert vol == pytest.approx(Q / (nH * nH * aB) * (1 - math.exp(-4.0)), rel=0.10)
    sw.close()


def test_invalid_thermal_parameters_are_rejected():
    case = wl.hii_region(n=8, nside=1, box_kpc=1.6)
    sw = _ctx(case)
    nH, y = _dev(case.nH), _dev(case.y0)
    T = _dev(np.full(case.nH.shape, 100.0))
    for bad in (dict(kB=0.0), dict(T_min=0.0), dict(T_min=1e4, T_max=1e3), dict(e_bin=[-1.0]),
                dict(e_diff=float("nan")), dict(z=-1.0), dict(T_min=200.0)):
        with pytest.raises(art.ArtError) as ex:
            sw.evolve_thermal(nH, case.chem, _th(**bad), _srcs(case), y, T, 1e12)
        assert ex.value.status == art.ART_E_INVALID, bad
    sw.close()


def test_fixed_steps_test2_geometry_match_oracle(orc):
    """Test 2's geometry (a point source beside a dense cold clump, 4 blackbody
    bins, the diffuse field transferred) over fixed steps: y, 1 - y and T
    within 1e-4 of the oracle after every call."""
    case = wl.point_clump(n=16, nside=2)
    frac, sig, _ = wl.blackbody_bins()
    th = _th(e_bin=list(wl.blackbody_heat()), e_diff=wl.diffuse_band_heat(case.chem))
    T0 = np.full(case.nH.shape, 100.0)
    dt = 1.0 / (case.chem["alphaB"] * 1e-3) / 800
    sw = _ctx(case, bins=(frac, sig))
    nH, y, T = _dev(case.nH), _dev(case.y0), _dev(T0)
    y_o, T_o = case.y0.copy(), T0.copy()
    for _ in range(2):
        rep = sw.evolve_thermal(nH, case.chem, th, _srcs(case), y, T, 3 * dt, dt_fixed=dt, eps_iter=1e-6)
        assert rep.converged and rep.steps == 3
        y_o, T_o, steps, *_ = orc.evolve_thermal(case.nH, case.nside, case.chem, th, case.pos, case.Q, y_o, T_o,
                                                 3 * dt, dt_fixed=dt, eps_iter=1e-9, sigma_bins=sig, frac_bins=frac)
        yg, Tg = y.cpu().numpy(), T.cpu().numpy()
        assert rel(yg, y_o) < 1e-4 and rel(1 - yg, 1 - y_o) < 1e-4
        assert rel(Tg, T_o) < 1e-4
    clump = case.nH > 1.5e-3
    assert T_o.max() > 5e3 and np.all(T_o[clump] < 1e3)   # heated near the source, the clump still cold
    sw.close()
