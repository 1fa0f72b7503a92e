"""Pins of the oracle's time-dependent mode (App. B-D at fixed temperature):

* pure recombination of an ionized cell has the closed form
  1 - y = 1 / (1 + alpha_B n_H t); the sub-cycled BDF step converges to it at
  first order as the chemical-timestep factors shrink;
* a point source in a uniform medium on the spot grows the Stromgren sphere
  R(t) = R_S (1 - e^{-t/t_rec})^{1/3} (sharp front: the mean free path of
  51 pc is far below R_S = 5.4 kpc, the paper's Test-1 numbers), and halving
  F leaves it unchanged;
* a long evolution ends at the equilibrium of the fixed-point iteration.
"""
import math

import numpy as np
import pytest

from paper_1410_0763_gb300 import workloads as wl


def _recombining(n=2, nH=1.0):
    case = wl.hii_region(n=n, nside=1, box_kpc=0.01, nH=nH)
    chem = dict(case.chem, alphaA=case.chem["alphaB"], gcoll=0.0)
    return case, chem


@pytest.mark.parametrize("scale", [1.0, 0.1, 0.01])
def test_pure_recombination_closed_form(orc, scale):
    case, chem = _recombining()
    aB, nH = chem["alphaB"], 1.0
    t_rec = 1.0 / (aB * nH)
    y0 = np.zeros_like(case.nH)                      # fully ionized
    errs = []
    for t in (0.5 * t_rec, 2.0 * t_rec, 10.0 * t_rec):
        y, steps, iters, tr, dts, rc = orc.evolve(case.nH, 1, chem, np.zeros((0, 3)), np.zeros(0), y0, t,
                                                  eps_e=0.2 * scale, eps_hi=0.002 * scale)
        assert rc == 0 and tr == t
        exact = 1.0 / (1.0 + aB * nH * t)            # n_e / n_H
        errs.append(abs((1 - y[0, 0, 0]) - exact) / exact)
    # first order in the sub-step factor: the error scales with it
    assert max(errs) < 0.25 * scale


def _stromgren(orc, n, F):
    nH, Q = 1e-3, 5e48
    case = wl.hii_region(n=n, nside=1, box_kpc=6.6, nH=nH, Q=Q, source_at="corner")
    chem = dict(case.chem, alphaA=case.chem["alphaB"])
    aB, dx = chem["alphaB"], chem["dx"]
    t_rec = 1.0 / (aB * nH)
    rs = (3 * Q / (4 * math.pi * nH * nH * aB)) ** (1 / 3)
    y, t, out = case.y0.copy(), 0.0, []
    for f in (0.1, 0.25, 0.5, 1.0):
        y, steps, iters, tr, dts, rc = orc.evolve(case.nH, 1, chem, case.pos, case.Q, y, f * t_rec - t, F=F)
        assert rc == 0
        t = f * t_rec
        vol = 8 * np.sum(1 - y) * dx ** 3            # the source sits on the box corner
        out.append(((3 * vol / (4 * math.pi)) ** (1 / 3) / rs, (1 - math.exp(-f)) ** (1 / 3)))
    return out


def test_stromgren_sphere_growth(orc):
    # the paper's printed Test-1 scales: t_rec = 122.4 Myr, R_S = 5.4 kpc
    case = wl.hii_region(n=16, nside=1, box_kpc=6.6, source_at="corner")
    aB = case.chem["alphaB"]
    assert 1 / (aB * 1e-3) / wl.MYR == pytest.approx(122.4, rel=2e-3)
    r1 = _stromgren(orc, 16, 1.0)
    for got, want in r1:
        assert got == pytest.approx(want, rel=0.06)
    r_half = _stromgren(orc, 16, 0.5)
    for (a, _), (b, _) in zip(r1, r_half):
        assert a == pytest.approx(b, rel=0.01)


def test_long_evolution_reaches_the_equilibrium(orc):
    case = wl.hii_region(n=8, nside=1, box_kpc=1.6)
    ch = case.chem
    t_rec = 1.0 / (ch["alphaB"] * 1e-3)
    y_eq, it, hist, conv = orc.iterate(case.nH, 1, ch, case.pos, case.Q, case.y0, 1e-10, 400)
    assert conv
    y, steps, iters, tr, dts, rc = orc.evolve(case.nH, 1, ch, case.pos, case.Q, case.y0, 30 * t_rec,
                                              eps_iter=1e-8)
    assert rc == 0
    assert np.max(np.abs(y - y_eq) / y_eq) < 1e-3
    assert np.max(np.abs((1 - y) - (1 - y_eq)) / (1 - y_eq)) < 1e-3
