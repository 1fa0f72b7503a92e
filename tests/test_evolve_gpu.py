"""GPU time-dependent mode (App. B-D at fixed temperature) against the FP64
oracle and the closed forms its oracle pins use.

* Fixed step sequence (dt_fixed), iterations converged well below the
  parity bound (eps_iter 1e-6 on the GPU, whose FP32 rates leave a residual
  near 1e-7; 1e-9 in the oracle): the state after every step follows the
  oracle's within 1e-4 relative in y and 1 - y (the FP32 rates' error,
  amplified by the chemistry as in the equilibrium iteration).
* Adaptive steps (F = 1): the on-the-spot Stromgren sphere grows as
  R_S (1 - e^{-t/t_rec})^{1/3} within 5 % at 32^3, and pure recombination
  follows 1 - y = 1 / (1 + alpha_B n_H t) within the first-order error of the
  sub-steps.
* A long evolution ends at the equilibrium of art_iterate_ionization.
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


def _ctx(case, bins=None):
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    if bins is not None:
        sw.set_source_spectrum(bins[1], bins[0])
    if case.plane is not None:
        sw.set_plane_source(*case.plane)
    return sw


def _srcs(case):
    return [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]


def _dev(a):
    return torch.as_tensor(a, dtype=torch.float64, device="cuda").clone()


@pytest.mark.parametrize("otsa", [False, True])
def test_fixed_steps_match_oracle(orc, otsa):
    case = wl.hii_region(n=16, nside=2, box_kpc=1.6)
    chem = dict(case.chem, alphaA=case.chem["alphaB"]) if otsa else case.chem
    t_rec = 1.0 / (chem["alphaB"] * 1e-3)
    dt = t_rec / 400
    sw = _ctx(case)
    nH, y = _dev(case.nH), _dev(case.y0)
    y_o = case.y0.copy()
    for _ in range(3):      # 3 calls of 4 steps each: the state carries over
        rep = sw.evolve(nH, chem, _srcs(case), y, 4 * dt, dt_fixed=dt, eps_iter=1e-6)
        assert rep.steps == 4 and rep.converged and rep.sub_overflow == 0
        y_o, steps, iters, tr, dts, rc = orc.evolve(case.nH, case.nside, chem, case.pos, case.Q, y_o, 4 * dt,
                                                    dt_fixed=dt, eps_iter=1e-9)
        assert rc == 0 and steps == 4
        yg = y.cpu().numpy()
        assert rel(yg, y_o) < 1e-4
        assert rel(1 - yg, 1 - y_o) < 1e-4
    assert (rep.sweeps == 0) == otsa
    sw.close()


def test_fixed_steps_with_a_plane_flux_and_bins_match_oracle(orc):
    case = wl.shadow_clump(n=16, nside=2)
    frac, sig, _ = wl.blackbody_bins()
    t_rec = 1.0 / (case.chem["alphaB"] * 2e-4)
    dt = t_rec / 2000
    sw = _ctx(case, bins=(frac, sig))
    nH, y = _dev(case.nH), _dev(case.y0)
    rep = sw.evolve(nH, case.chem, [], y, 6 * dt, dt_fixed=dt, eps_iter=1e-6)
    y_o, steps, *_ = orc.evolve(case.nH, case.nside, case.chem, case.pos, case.Q, case.y0, 6 * dt, dt_fixed=dt,
                                eps_iter=1e-9, sigma_bins=sig, frac_bins=frac, plane=case.plane)
    assert rep.converged and rep.steps == steps == 6
    yg = y.cpu().numpy()
    assert rel(yg, y_o) < 1e-4
    assert rel(1 - yg, 1 - y_o) < 1e-4
    sw.close()


def test_stromgren_sphere_growth_gpu():
    n, nH, Q = 32, 1e-3, 5e48
    case = wl.hii_region(n=n, nside=1, box_kpc=6.6, nH=nH, Q=Q, source_at="corner")
    chem = dict(case.chem, alphaA=case.chem["alphaB"])
    aB, dx = chem["alphaB"], chem["dx"]
    t_rec = 1.0 / (aB * nH)
    rs = (3 * Q / (4 * math.pi * nH * nH * aB)) ** (1 / 3)
    sw = _ctx(case)
    nH_d, y = _dev(case.nH), _dev(case.y0)
    t = 0.0
    for f in (0.1, 0.5, 1.0):
        rep = sw.evolve(nH_d, chem, _srcs(case), y, f * t_rec - t, F=1.0)
        t = f * t_rec
        assert rep.converged and rep.sweeps == 0
        vol = 8 * float(torch.sum(1 - y)) * dx ** 3
        r = (3 * vol / (4 * math.pi)) ** (1 / 3)
        assert r / rs == pytest.approx((1 - math.exp(-f)) ** (1 / 3), rel=0.05)
    sw.close()


def test_pure_recombination_gpu():
    case = wl.hii_region(n=4, nside=1, box_kpc=0.01, nH=1.0)
    chem = dict(case.chem, alphaA=case.chem["alphaB"], gcoll=0.0)
    aB = chem["alphaB"]
    sw = _ctx(case)
    for scale in (1.0, 0.01):
        y = _dev(np.zeros_like(case.nH))
        rep = sw.evolve(_dev(case.nH), chem, [], y, 2.0 / aB, eps_e=0.2 * scale, eps_hi=0.002 * scale)
        exact = 1.0 / (1.0 + 2.0)
        err = float(torch.max(torch.abs((1 - y) - exact))) / exact
        assert err < 0.25 * scale
    sw.close()


def test_long_evolution_reaches_the_equilibrium():
    case = wl.hii_region(n=16, nside=2, box_kpc=1.6)
    t_rec = 1.0 / (case.chem["alphaB"] * 1e-3)
    sw = _ctx(case)
    nH = _dev(case.nH)
    y_eq = _dev(case.y0)
    sw.iterate(nH, case.chem, _srcs(case), y_eq, tol=1e-6, max_iter=400)
    y = _dev(case.y0)
    rep = sw.evolve(nH, case.chem, _srcs(case), y, 30 * t_rec, eps_iter=1e-6)
    assert rep.converged
    a, b = y.cpu().numpy(), y_eq.cpu().numpy()
    assert rel(a, b) < 1e-3
    assert rel(1 - a, 1 - b) < 1e-3
    sw.close()


def test_invalid_options_are_rejected():
    case = wl.hii_region(n=8, nside=1, box_kpc=1.6)
    sw = _ctx(case)
    nH, y = _dev(case.nH), _dev(case.y0)
    for kw in (dict(F=0.0), dict(eps_iter=0.0), dict(eps_e=0.0, eps_hi=0.0), dict(max_steps=0),
               dict(dt_fixed=-1.0)):
        with pytest.raises(art.ArtError) as ex:
            sw.evolve(nH, case.chem, _srcs(case), y, 1e12, **kw)
        assert ex.value.status == art.ART_E_INVALID
    with pytest.raises(art.ArtError) as ex:
        sw.evolve(nH, case.chem, _srcs(case), y, float("inf"))
    assert ex.value.status == art.ART_E_INVALID
    # too few steps for t_end: not converged, y holds the state reached
    with pytest.raises(art.ArtError) as ex:
        sw.evolve(nH, case.chem, _srcs(case), y, 1e20, max_steps=2)
    assert ex.value.status == art.ART_E_NOT_CONVERGED
    sw.close()
