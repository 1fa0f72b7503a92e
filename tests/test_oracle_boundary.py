"""Pins of the oracle's incident-radiation boundaries (Sec. 4.3, Test 3):

* a boundary intensity I_bc on every ray entering the box (the formal
  solution, Eq. rad_tr2, with I(0) = I_bc instead of vacuum);
* a plane-parallel incident photon flux through one face (a point source at
  infinity), absorbed cell by cell with the photon-conserving rate.

Pinned against what the transfer equation fixes: an empty box keeps I_bc;
linearity in I_bc and S; e^-kappa s attenuation from the entry point of every
ray (side faces included); the equilibrium S = I_bc; per-column photon
conservation of the beam; the unattenuated thin limit; and the symmetries of
the beam's axis and direction.
"""
import math

import numpy as np
import pytest

from paper_1410_0763_gb300 import workloads as wl


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


@pytest.mark.parametrize("shape,nside", [((5, 6, 7), 1), ((4, 9, 6), 2)])
def test_empty_box_keeps_the_boundary_intensity(orc, shape, nside):
    z = np.zeros(shape)
    jin, j, nz = orc.sweep(z, z, nside, i_bc=2.5)
    assert nz == 0
    assert np.allclose(jin, 2.5, rtol=1e-14, atol=0)


def test_linear_in_boundary_intensity_and_source(orc):
    rng = np.random.default_rng(11)
    shape = (6, 7, 8)
    kap = 0.5 * np.exp(rng.standard_normal(shape))
    S = rng.random(shape)
    a, _, _ = orc.sweep(kap, S, 2, i_bc=0.0)
    b, _, _ = orc.sweep(kap, np.zeros(shape), 2, i_bc=1.0)
    c, _, _ = orc.sweep(kap, S, 2, i_bc=0.7)
    assert rel(c, a + 0.7 * b) < 1e-12
    # emissivity form: the same boundary term
    c2, _, _ = orc.sweep(kap, S * kap, 2, field_form=1, i_bc=0.7)
    assert rel(c2, a + 0.7 * b) < 1e-12


def test_equilibrium_source_equal_to_boundary_intensity(orc):
    # I = S everywhere when the rays enter with I_bc = S: every segment starts
    # at S, so every path-averaged incoming intensity is S phi(dtau)
    rng = np.random.default_rng(12)
    shape = (5, 6, 7)
    kap = 0.4 * np.exp(rng.standard_normal(shape))
    S = np.full(shape, 1.3)
    for d in range(12 * 2 * 2):
        cells, ds, iin, iex = orc.trace_ray(kap, S, 2, d, *_some_ray(orc, shape, 2, d), i_bc=1.3)
        assert np.allclose(iin, 1.3, rtol=1e-14) and iex == pytest.approx(1.3, rel=1e-14)


def _some_ray(orc, shape, nside, d):
    (jlo, jhi, klo, khi), _, _ = orc.lattice(shape, nside, d)
    return (jlo + jhi) // 2, (klo + khi) // 2


def test_attenuation_from_every_entry_point(orc):
    # uniform kappa, S = 0: the intensity at the start of each segment is
    # I_bc e^{-kappa s}, s the path length since the ray entered the box --
    # through the entry face or a side face
    shape = (6, 5, 7)
    kap = np.full(shape, 0.35)
    z = np.zeros(shape)
    checked = 0
    for d in range(12 * 4):
        (jlo, jhi, klo, khi), _, _ = orc.lattice(shape, 2, d)
        for j in range(jlo, jhi + 1, 2):
            for k in range(klo, khi + 1, 2):
                cells, ds, iin, iex = orc.trace_ray(kap, z, 2, d, j, k, i_bc=3.0)
                if cells.size == 0:
                    continue
                s = np.concatenate([[0.0], np.cumsum(ds)[:-1]])
                assert np.allclose(iin, 3.0 * np.exp(-0.35 * s), rtol=1e-13)
                assert iex == pytest.approx(3.0 * math.exp(-0.35 * ds.sum()), rel=1e-13)
                checked += 1
    assert checked > 100


# --- plane-parallel incident flux ---

@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("direction", [1, -1])
def test_beam_conserves_photons_per_column(orc, axis, direction):
    # summed over a column, n_HI Gamma V = F A (1 - e^-tau_column): with
    # n_HI V = kappa_b dx^2 / sigma_b, sum_cells Gamma kappa_b / sigma_b = F_b (1 - e^-tau_b)
    rng = np.random.default_rng(20 + axis)
    shape = (5, 6, 7)
    kap = 0.3 * np.exp(rng.standard_normal((2,) + shape))
    sig = np.array([6.3e-18, 1.5e-18])
    F = np.array([1e6, 3e5])
    g = orc.plane_source(kap, sig, axis, direction, F)
    ax = 2 - axis    # numpy axis of the beam in [z][y][x]
    # per bin separately (Gamma sums over bins)
    tot = np.zeros(np.delete(np.array(shape), ax))
    for b in range(2):
        gb = orc.plane_source(kap[b], [sig[b]], axis, direction, [F[b]])
        col = np.sum(gb * kap[b] / sig[b], axis=ax)
        tau = np.sum(kap[b], axis=ax)
        assert np.allclose(col, F[b] * -np.expm1(-tau), rtol=1e-12)
        tot += gb.sum(axis=ax)
    assert np.allclose(g.sum(axis=ax), tot, rtol=1e-13)


def test_beam_thin_limit_and_attenuation_order(orc):
    shape = (4, 5, 6)
    g = orc.plane_source(np.zeros(shape), [6.3e-18], 2, 1, [1e6])
    assert np.allclose(g, 1e6 * 6.3e-18, rtol=1e-15)
    kap = np.full(shape, 0.2)
    up = orc.plane_source(kap, [6.3e-18], 2, 1, [1e6])
    down = orc.plane_source(kap, [6.3e-18], 2, -1, [1e6])
    assert np.all(np.diff(up, axis=0) < 0)          # along +z the rate falls
    assert np.all(np.diff(down, axis=0) > 0)        # along -z it rises
    assert np.allclose(down, up[::-1], rtol=1e-14)


def test_beam_axis_symmetry(orc):
    rng = np.random.default_rng(21)
    kap = 0.4 * np.exp(rng.standard_normal((5, 6, 7)))
    gx = orc.plane_source(kap, [2e-18], 0, 1, [1e6])
    gz = orc.plane_source(np.ascontiguousarray(kap.transpose(2, 1, 0)), [2e-18], 2, 1, [1e6])
    assert np.allclose(gx, gz.transpose(2, 1, 0), rtol=1e-14)
    gy = orc.plane_source(kap, [2e-18], 1, -1, [1e6])
    gy2 = orc.plane_source(np.ascontiguousarray(kap[:, ::-1, :]), [2e-18], 1, 1, [1e6])
    assert np.allclose(gy, gy2[:, ::-1, :], rtol=1e-14)


def test_iteration_with_a_beam_is_a_fixed_point(orc):
    """The oracle's iteration with a plane-parallel flux converges to a state
    where every cell balances case-B recombination against the beam, the
    diffuse field and collisions; the clump shadows the cells behind it."""
    case = wl.shadow_clump(n=12, nside=1, box_kpc=6.6)
    ch = case.chem
    y, it, hist, conv = orc.iterate(case.nH, case.nside, ch, case.pos, case.Q, case.y0, 1e-8, 400,
                                    plane=case.plane)
    assert conv
    kap = y * case.nH * ch["sigma0"] * ch["dx"]
    ne = (1 - y) * case.nH
    eps = ch["h"] * ch["nu0"] * (ch["alphaA"] - ch["alphaB"]) * ne * ne * ch["dx"] / (4 * math.pi * ch["dnu"])
    jin, _, _ = orc.sweep(kap, eps, case.nside, field_form=1)
    G = orc.band_integral(ch["sigma0"], ch["h"], ch["nu0"], ch["nu0"] + ch["dnu"])
    g = 4 * math.pi * G * jin + orc.plane_source(kap, [ch["sigma0"]], 0, 1, [case.plane[2]])
    y_check = orc.balance_eq(case.nH.ravel(), ch["alphaB"], ch["gcoll"], g.ravel()).reshape(y.shape)
    assert rel(y, y_check) < 1e-6
    # behind the clump (along +x, on its axis) the gas is more neutral than beside it
    mid = case.n // 2
    assert y[mid, mid, -1] > y[0, 0, -1]
