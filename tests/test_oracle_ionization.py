"""Pins of the oracle's ionization side: Eq. (gamma_diff) band integral, the
photon-conserving point-source rate of App. A, the equilibrium balance of
App. B and the fixed-point iteration of App. D.

* the band integral is checked against numerical quadrature;
* the point-source rate against the inverse-square law far from the source,
  against e^{-tau} with tau integrated by dense sampling of the straight line
  (an independent path integral), and against exact photon conservation along
  one ray (adjacent shells telescope to Q (1 - e^{-tau}));
* the balance root against a bracketing root finder on the balance equation;
* the iteration against the paper's printed Test-1 numbers (t_rec = 122.4 Myr,
  R_S = 5.4 kpc fix alpha_B), a Stromgren-volume check, monotone ionization
  from a neutral start, and the paper's finding that the diffuse field
  enlarges the ionized region relative to the on-the-spot approximation.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

from paper_1410_0763_gb300 import workloads as wl


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows[f[0]] = (float(f[1]), float(f[3]))
    return rows


def test_paper_numbers_fix_alpha_b_and_sigma0():
    """The paper's printed Test-1 numbers (tests/golden/paper_test1_values.txt)."""
    g = _golden("paper_test1_values.txt")
    nH, Q = 1e-3, 5e48
    t_rec = 1.0 / (wl.ALPHA_B_1E4 * nH) / wl.MYR
    assert t_rec == pytest.approx(g["t_rec"][0], rel=g["t_rec"][1])
    rs = (3 * Q / (4 * math.pi * nH * nH * wl.ALPHA_B_1E4)) ** (1 / 3) / wl.KPC
    assert rs == pytest.approx(g["R_S"][0], rel=g["R_S"][1])
    mfp = 1.0 / (1e-3 * wl.SIGMA0) / wl.PC
    assert mfp == pytest.approx(g["lambda_mfp"][0], rel=g["lambda_mfp"][1])
    assert 6.6 * wl.KPC / 128 / wl.PC == pytest.approx(g["Delta_H"][0], rel=g["Delta_H"][1])


def test_band_integral_vs_quadrature(orc):
    c = wl.chem_constants()
    nu0, nu1 = c["nu0"], c["nu0"] + c["dnu"]
    f = lambda nu: c["sigma0"] * (nu / nu0) ** -3 / (c["h"] * nu)
    ref, _ = integrate.quad(f, nu0, nu1, epsrel=1e-13)
    assert orc.band_integral(c["sigma0"], c["h"], nu0, nu1) == pytest.approx(ref, rel=1e-12)


def _shell_geometry(src, cell):
    """r_in, r_out of the straight line from src through the centre of cell (slab test)."""
    c = np.array(cell, dtype=float) + 0.5
    d = c - src
    L = np.linalg.norm(d)
    n = d / L
    lo, hi = -np.inf, np.inf
    for i in range(3):
        if abs(n[i]) < 1e-300:
            continue
        t1 = (cell[i] - src[i]) / n[i]
        t2 = (cell[i] + 1 - src[i]) / n[i]
        lo = max(lo, min(t1, t2))
        hi = min(hi, max(t1, t2))
    return max(lo, 0.0), hi, n


def test_point_source_inverse_square_far_field(orc):
    n = 48
    kap = np.zeros((1, n, n, n))
    dx = 1e20
    sig = 6.3e-18
    Q = 1e50
    src = np.array([[0.3, 0.4, 0.45]])
    g = orc.point_sources(kap, [sig], src, [[Q]], dx)
    for cell in [(40, 2, 3), (30, 35, 10), (44, 44, 44), (20, 0, 33)]:
        x, y, z = cell
        r = np.linalg.norm(np.array(cell) + 0.5 - src[0]) * dx
        thin = Q * sig / (4 * math.pi * r * r)
        assert g[z, y, x] == pytest.approx(thin, rel=2e-3)


def test_point_source_attenuation_is_line_integral(orc):
    rng = np.random.default_rng(12)
    n = 20
    kap = 0.3 * np.exp(rng.standard_normal((n, n, n)))
    src = np.array([7.31, 9.77, 4.12])
    sig, dx, Q = 1e-17, 1.0, 1.0
    for cell in [(18, 2, 15), (0, 19, 19), (12, 10, 4), (3, 3, 17)]:
        x, y, z = cell
        k2 = kap.copy()
        k2[z, y, x] = 0.0          # phi = 1 in the target cell
        g = orc.point_sources(k2[None], [sig], src[None], [[Q]], dx)[z, y, x]
        rin, rout, nvec = _shell_geometry(src, cell)
        # dense midpoint sampling of kappa along the line from the source to r_in
        m = 200000
        t = (np.arange(m) + 0.5) / m * rin
        p = src[None, :] + t[:, None] * nvec[None, :]
        idx = np.clip(np.floor(p).astype(int), 0, n - 1)
        tau = kap[idx[:, 2], idx[:, 1], idx[:, 0]].sum() * rin / m
        vol = 4 * math.pi / 3 * (rout ** 3 - rin ** 3)
        expect = Q * math.exp(-tau) * sig * (rout - rin) / (vol * dx * dx)
        assert g == pytest.approx(expect, rel=2e-4)


def test_point_source_photon_conservation_along_a_ray(orc):
    # cells on one straight line from the source have adjacent shells
    # [r_in, r_out], so the photons they absorb, n_HI Gamma V_shell, add up
    # exactly to the photons removed from that ray: Q (1 - e^{-tau_total})
    # (App. A, in minus out).  The source sits on the axis of a row of cells.
    rng = np.random.default_rng(2)
    n = 16
    kap = 0.4 * np.exp(rng.standard_normal((n, n, n)))
    sig, dx, Q = 1e-17, 1.0, 1.0
    y0, z0, x0 = 5, 9, 3.3
    src = np.array([[x0, y0 + 0.5, z0 + 0.5]])
    g = orc.point_sources(kap[None], [sig], src, [[Q]], dx)
    total = 0.0
    for x in range(3, n):
        rin = max(x - x0, 0.0)
        rout = x + 1 - x0
        vshell = 4 * math.pi / 3 * (rout ** 3 - rin ** 3) * dx ** 3
        nHI = kap[z0, y0, x] / (sig * dx)
        total += nHI * g[z0, y0, x] * vshell
    tau = kap[z0, y0, 3] * (4 - x0) + kap[z0, y0, 4:].sum()
    assert total == pytest.approx(Q * -math.expm1(-tau), rel=1e-12)


def test_balance_root(orc):
    rng = np.random.default_rng(4)
    nH = 10 ** rng.uniform(-4, 1, 200)
    g = 10 ** rng.uniform(-18, -8, 200)
    g[:5] = 0.0
    aB, gc = wl.ALPHA_B_1E4, wl.GAMMA_COLL_1E4
    y = orc.balance_eq(nH, aB, gc, g)
    for i in range(200):
        a, c = aB * nH[i], gc * nH[i]
        if g[i] == 0.0:
            # no photons: y = 1 and the collisional equilibrium y = a/(a + c)
            # are both roots; the stable one (any free electron grows) is kept
            assert y[i] == pytest.approx(aB / (aB + gc), rel=1e-13)
            continue
        f = lambda yy: a * (1 - yy) ** 2 - yy * (c * (1 - yy) + g[i])
        # f(0) = a > 0 > f(1) = -g: exactly one root in (0, 1)
        ref = optimize.brentq(f, 0.0, 1.0, xtol=1e-300, rtol=1e-15)
        assert y[i] == pytest.approx(ref, rel=1e-12, abs=1e-300)


def _small_hii(n=16, nside=2, box_kpc=1.6, Q=5e48, nH=1e-3):
    case = wl.hii_region(n=n, nside=nside, box_kpc=box_kpc, nH=nH, Q=Q)
    return case


def test_iteration_converges_and_ionizes_monotonically(orc):
    case = _small_hii()
    y = case.y0.copy()
    ys = [y]
    # run one iteration at a time from the neutral start
    for _ in range(12):
        y, it, hist, conv = orc.iterate(case.nH, case.nside, case.chem, case.pos, case.Q, y,
                                        tol=1e-6, max_iter=1)
        ys.append(y)
    for a, b in zip(ys, ys[1:]):
        assert np.all(b <= a * (1 + 1e-12))      # n_e never decreases
    y, it, hist, conv = orc.iterate(case.nH, case.nside, case.chem, case.pos, case.Q, case.y0,
                                    tol=1e-6, max_iter=200)
    assert conv and hist[-1] < 1e-6
    assert np.all(np.diff(np.log(hist[-5:])) < 0.5)


def test_stromgren_volume_without_diffuse(orc):
    # with alpha_A = alpha_B the recombination emissivity vanishes and the
    # equilibrium is a case-B Stromgren sphere around the source
    n = 24
    nH, Q = 1e-1, 5e48
    rs = (3 * Q / (4 * math.pi * nH * nH * wl.ALPHA_B_1E4)) ** (1 / 3)
    dx = 2.5 * rs / n
    case = wl.hii_region(n=n, nside=2, box_kpc=n * dx / wl.KPC, nH=nH, Q=Q)
    chem = dict(case.chem, alphaA=case.chem["alphaB"])
    y, it, hist, conv = orc.iterate(case.nH, 2, chem, case.pos, case.Q, case.y0, tol=1e-6,
                                    max_iter=300)
    assert conv
    vol = np.sum(1 - y) * dx ** 3
    assert vol == pytest.approx(4 * math.pi / 3 * rs ** 3, rel=0.06)


def test_diffuse_field_enlarges_ionized_region(orc):
    # Sec. 4.1: with the recombination radiation transferred the ionized region
    # is larger than with the on-the-spot approximation
    n = 20
    nH, Q = 1e-1, 5e48
    rs = (3 * Q / (4 * math.pi * nH * nH * wl.ALPHA_B_1E4)) ** (1 / 3)
    dx = 2.5 * rs / n
    case = wl.hii_region(n=n, nside=2, box_kpc=n * dx / wl.KPC, nH=nH, Q=Q)
    otsa = dict(case.chem, alphaA=case.chem["alphaB"])
    y_otsa, *_ = orc.iterate(case.nH, 2, otsa, case.pos, case.Q, case.y0, 1e-6, 300)
    y_diff, *_ = orc.iterate(case.nH, 2, case.chem, case.pos, case.Q, case.y0, 1e-6, 300)
    assert np.all(y_diff <= y_otsa * (1 + 1e-9))
    assert np.sum(1 - y_diff) > np.sum(1 - y_otsa)


def test_iteration_source_bins_split_and_scale(orc):
    """Splitting each source's photons over bins of equal cross section leaves
    the iteration unchanged (Gamma is linear in Q per bin, Eq. pc_gamma); a
    bin with a larger cross section and no photons changes nothing either."""
    n, nside = 12, 1
    case = wl.hii_region(n=n, nside=nside, box_kpc=1.2)
    s0 = case.chem["sigma0"]
    y1, it1, h1, c1 = orc.iterate(case.nH, nside, case.chem, case.pos, case.Q, case.y0, 1e-6, 200)
    y2, it2, h2, c2 = orc.iterate(case.nH, nside, case.chem, case.pos, case.Q, case.y0, 1e-6, 200,
                                  sigma_bins=[s0, s0, 3 * s0], frac_bins=[0.25, 0.75, 0.0])
    assert c1 and c2 and it1 == it2
    assert np.allclose(y1, y2, rtol=1e-12, atol=0)


def test_point_sources_at_selected_cells_equal_the_full_evaluation(orc):
    rng = np.random.default_rng(81)
    shape = (9, 10, 11)
    kap = 0.4 * np.exp(rng.standard_normal((2,) + shape))
    sig = [6.3e-18, 2.0e-18]
    pos = np.array([[2.3, 4.1, 7.7], [10.0, 0.0, 4.5]])
    Qb = np.array([[1e48, 2e47], [5e47, 5e47]])
    full = orc.point_sources(kap, sig, pos, Qb, 1e20).ravel()
    cells = rng.choice(full.size, 40, replace=False)
    assert np.array_equal(orc.point_sources_cells(kap, sig, pos, Qb, 1e20, cells), full[cells])
