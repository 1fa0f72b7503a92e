"""Pins of the oracle's energy equation (App. C) and temperature-dependent
rates, each against something other than the oracle itself.

* Fits: the case-A and case-B recombination coefficients against the
  textbook table (`golden/hydrogen_rate_values.txt`); the Compton
  coefficient against Ikeuchi & Ostriker's published value, rescaled from
  T_CMB = 2.7 K, and its (1 + z)^4 scaling; collisional-ionization cooling
  removes exactly the ionization potential h nu_0 per ionization; the fits at
  1e4 K reproduce the fixed-temperature constants of the equilibrium runs;
  recombination cooling removes 0.5-1.2 k T per recombination, more in case
  A; the free-free Gaunt factor lies in [1.1, 1.44].
* The implicit energy update: the analytic derivative of the cooling rate
  that its Newton steps use against central differences; closed forms with
  no cooling (heat shared by 1 + x particles) and with Compton cooling alone
  (a linear equation); with every term, the root of the implicit equation
  found by an independent bracketing solver (scipy's brentq).
* One cell over long times at fixed optically thin rates: ionization
  equilibrium at the final temperature and thermal balance H = C; the
  on-the-spot form (less cooling) ends hotter.
* The grid evolution: with neither heating nor cooling, the specific energy
  (2 - y) T of every cell is conserved while its composition changes.
"""
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
KB = 1.380649e-16
EV = 1.602176634e-12
H_PLANCK = 6.62607015e-27
NU0 = 13.598 * EV / H_PLANCK


def golden():
    rows = []
    for line in open(os.path.join(HERE, "golden", "hydrogen_rate_values.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append((f[0], float(f[1]), float(f[2]), float(f[4])))
    return rows


def test_recombination_coefficients_match_the_textbook_table(orc):
    n = 0
    for name, T, v, tol in golden():
        if name.startswith("alpha"):
            assert orc.rate_fit(name, T)[0] == pytest.approx(v, rel=tol), (name, T)
            n += 1
    assert n == 6


def test_compton_coefficient_matches_the_published_value(orc):
    (_, _, v, tol), = [r for r in golden() if r[0] == "compton_2.7K"]
    c0 = orc.rate_fit("compton", 0, z=0.0, kB=KB)
    assert c0 == pytest.approx(v * (2.7255 / 2.7) ** 4, rel=tol)
    assert orc.rate_fit("compton", 0, z=1.0, kB=KB) == pytest.approx(16 * c0, rel=1e-12)


def test_collisional_ionization_cooling_is_the_ionization_potential_per_ionization(orc):
    T = np.geomspace(3e3, 1e7, 25)
    per_ion = orc.rate_fit("cool_ci", T) / orc.rate_fit("gamma_coll", T)
    assert np.allclose(per_ion, H_PLANCK * NU0, rtol=5e-3)


def test_fits_at_1e4_reproduce_the_fixed_temperature_constants(orc):
    from paper_1410_0763_gb300 import workloads as wl
    c = wl.chem_constants()
    assert orc.rate_fit("alpha_B", 1e4)[0] == pytest.approx(c["alphaB"], rel=2e-3)
    assert orc.rate_fit("gamma_coll", 1e4)[0] == pytest.approx(c["gcoll"], rel=5e-3)


def test_recombination_cooling_per_recombination(orc):
    T = np.array([5e3, 1e4, 2e4])
    per_a = orc.rate_fit("cool_rec_A", T) / (orc.rate_fit("alpha_A", T) * KB * T)
    per_b = orc.rate_fit("cool_rec_B", T) / (orc.rate_fit("alpha_B", T) * KB * T)
    assert np.all((per_b > 0.5) & (per_b < 1.2)) and np.all((per_a > 0.5) & (per_a < 1.2))
    assert np.all(orc.rate_fit("cool_rec_A", T) > orc.rate_fit("cool_rec_B", T))


def test_free_free_gaunt_factor(orc):
    T = np.geomspace(1e3, 1e8, 30)
    g = orc.rate_fit("cool_ff", T) / (1.42e-27 * np.sqrt(T))
    assert np.all((g >= 1.1 - 1e-12) & (g <= 1.44 + 1e-12))
    assert g[np.argmin(np.abs(np.log10(T) - 5.5))] == pytest.approx(1.44, rel=2e-2)


def _th(**kw):
    d = dict(kB=KB, e_bin=[3 * EV], e_diff=0.5 * EV, z=-1.0, T_min=10.0, T_max=1e9, cool_mask=31)
    d.update(kw)
    return d


@pytest.mark.parametrize("otsa", [0, 1])
def test_cooling_derivative_matches_central_differences(orc, otsa):
    th = _th(on_the_spot=otsa, z=2.0)
    for T in np.geomspace(30.0, 3e8, 60):
        for y in (0.0, 0.3, 0.999):
            h = 1e-5 * T
            fd = (orc.cooling(th, 1e-2, y, T + h) - orc.cooling(th, 1e-2, y, T - h)) / (2 * h)
            d = orc.cooling_deriv(th, 1e-2, y, T)
            scale = abs(orc.cooling(th, 1e-2, y, T)) / T + 1e-300
            assert abs(d - fd) <= 1e-6 * max(abs(fd), scale), (T, y, d, fd)


def test_energy_step_without_cooling_shares_the_heat(orc):
    th = _th(cool_mask=0)
    for nH, y0, T0, y1, H, dt in [(1e-3, 0.9, 100.0, 0.5, 1e-27, 1e13), (1.0, 0.1, 2e4, 0.2, 0.0, 1e10),
                                  (1e-2, 1.0, 50.0, 0.999, 3e-26, 1e12)]:
        e0 = 1.5 * KB * nH * (2 - y0) * T0
        want = (e0 + H * dt) / (1.5 * KB * nH * (2 - y1))
        assert orc.energy_step(th, nH, y0, T0, y1, H, dt) == pytest.approx(want, rel=1e-12)


def test_energy_step_with_compton_cooling_alone(orc):
    th = _th(cool_mask=16, z=9.0)
    k = orc.rate_fit("compton", 0, z=9.0, kB=KB)
    Tg = 2.7255 * 10
    for nH, y0, T0, y1, H, dt in [(1e-4, 0.0, 1e4, 0.0, 0.0, 1e15), (1e-3, 0.3, 5e3, 0.25, 1e-28, 3e15)]:
        A = 1.5 * KB * nH * (2 - y1)
        B = 1.5 * KB * nH * (2 - y0) * T0 + H * dt
        ne = (1 - y1) * nH
        want = (B + dt * k * ne * Tg) / (A + dt * k * ne)
        assert orc.energy_step(th, nH, y0, T0, y1, H, dt) == pytest.approx(want, rel=1e-11)


def test_energy_step_root_matches_brentq(orc):
    from scipy.optimize import brentq
    rng = np.random.default_rng(5)
    for case_b in (0, 1):
        th = _th(on_the_spot=case_b, z=3.0)
        for _ in range(40):
            nH = 10 ** rng.uniform(-4, 1)
            y0, y1 = rng.uniform(0, 1, 2)
            T0 = 10 ** rng.uniform(2, 5)
            H = 10 ** rng.uniform(-30, -22) * nH
            dt = 10 ** rng.uniform(8, 14)
            A = 1.5 * KB * nH * (2 - y1)
            B = 1.5 * KB * nH * (2 - y0) * T0 + H * dt

            def f(T):
                return A * T + dt * orc.cooling(th, nH, y1, T) - B

            Tg = orc.energy_step(th, nH, y0, T0, y1, H, dt)
            assert abs(f(Tg)) <= 1e-9 * B
            grid = np.geomspace(10.0, 1e9, 400)
            fv = np.array([f(t) for t in grid])
            if np.all(np.diff(fv) > 0) and fv[0] < 0 < fv[-1]:   # a single root
                assert Tg == pytest.approx(brentq(f, 10.0, 1e9, xtol=1e-12, rtol=1e-14), rel=1e-10)


def test_optically_thin_cell_reaches_ionization_and_thermal_equilibrium(orc):
    nH, g, E = 1e-2, 1e-12, 3 * EV
    finals = {}
    for otsa in (0, 1):
        th = _th(on_the_spot=otsa)
        # near equilibrium a call takes one sub-step (the chemical timestep
        # diverges), a fixed-point step of the update: repeat the call
        y, T, n = orc.thermal_cell(th, nH, 1.0, 100.0, g, g * E, 0.0, 3e15)   # ~7 cooling times
        assert n > 10
        for _ in range(12):
            y, T, _n = orc.thermal_cell(th, nH, y, T, g, g * E, 0.0, 3e15)
        aB, gc = orc.rate_fit("alpha_B", T)[0], orc.rate_fit("gamma_coll", T)[0]
        a, c = aB * nH, gc * nH
        y_eq = 2 * a / (2 * a + c + g + math.sqrt(4 * a * g + (c + g) ** 2))
        assert y == pytest.approx(y_eq, rel=1e-7)
        # photo-heating, plus the local recombination photons (alpha_A - alpha_B) n_e^2 e_diff
        dal = 0.0 if otsa else orc.rate_fit("alpha_A", T)[0] - aB
        heat = y * nH * g * E + dal * ((1 - y) * nH) ** 2 * th["e_diff"]
        assert orc.cooling(th, nH, y, T) == pytest.approx(heat, rel=1e-7)
        assert 5e3 < T < 3e4
        finals[otsa] = T
    assert finals[1] > finals[0]


def test_grid_evolution_without_heating_or_cooling_conserves_specific_energy(orc):
    from paper_1410_0763_gb300 import workloads as wl
    case = wl.hii_region(n=6, nside=1, box_kpc=0.5, nH=1e-2)
    rng = np.random.default_rng(3)
    y0 = rng.uniform(0.0, 0.5, case.nH.shape)
    T0 = rng.uniform(5e3, 3e4, case.nH.shape)
    th = _th(on_the_spot=1, cool_mask=0, e_bin=[0.0], e_diff=0.0)
    t_rec = 1.0 / (2.6e-13 * 1e-2)
    y, T, steps, iters, t, dts, rc = orc.evolve_thermal(case.nH, 1, case.chem, th, np.zeros((0, 3)), np.zeros(0),
                                                        y0, T0, 0.5 * t_rec, F=1.0, eps_iter=1e-9)
    assert rc == 0 and steps > 3
    assert np.max(np.abs(y - y0)) > 0.05       # recombining (cool cells) or collisionally ionized (hot ones)
    assert np.allclose((2 - y) * T, (2 - y0) * T0, rtol=1e-12)


def test_heated_stromgren_volume_uses_alpha_B_at_the_ionized_temperature(orc):
    """On the spot, a source in a corner of a uniform medium starting cold and
    neutral: after 4 recombination times the region is photo-heated to
    5e3-3e4 K and its volume is the Stromgren volume Q / (n_H^2 alpha_B(T))
    taken at the mean temperature of the ionized gas (within 10 %; the
    growth factor (1 - e^-4) is 0.98)."""
    from paper_1410_0763_gb300 import workloads as wl
    nH, Q = 1e-3, 5e48
    case = wl.hii_region(n=16, nside=1, box_kpc=6.6, nH=nH, Q=Q, source_at="corner")
    th = _th(on_the_spot=1, e_bin=[3 * EV], e_diff=0.0)
    T0 = np.full(case.nH.shape, 100.0)
    y, T, steps, iters, t, dts, rc = orc.evolve_thermal(case.nH, 1, case.chem, th, case.pos, case.Q, case.y0, T0,
                                                        4 * 1.0 / (2.59e-13 * nH), F=1.0)
    assert rc == 0
    ion = (1 - y) > 0.5
    T_ion = float(np.sum(T * (1 - y)) / np.sum(1 - y))
    assert 5e3 < T_ion < 3e4 and np.all(T[y > 0.99] < 1e3)
    dx = case.chem["dx"]
    vol = 8 * float(np.sum(1 - y)) * dx ** 3     # the corner source lights one octant
    v_s = Q / (nH * nH * orc.rate_fit("alpha_B", T_ion)[0])
    assert vol == pytest.approx(v_s * (1 - math.exp(-4.0)), rel=0.10), (vol / v_s, T_ion, int(ion.sum()))


# ---------------------------------------------------------------------------
# Pins of the cooling and collisional fits against physics and independent
# published values (tests/golden/rate_fit_pins.txt).
# ---------------------------------------------------------------------------
def pins():
    path = os.path.join(os.path.dirname(__file__), "golden", "rate_fit_pins.txt")
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def _fit(orc, name, T):
    return np.array([orc.rate_fit(name, float(t))[0] for t in np.atleast_1d(T)])


def _dlog_dlogT(orc, name, T, h=1e-4):
    return (np.log(_fit(orc, name, T * (1 + h))) - np.log(_fit(orc, name, T * (1 - h)))) / \
        (np.log1p(h) - np.log1p(-h))


def _activation_temperature(orc, name, T, h=1e-4):
    """-d ln f / d(1/T): the energy (in K) of the Boltzmann factor that dominates at low T."""
    return -(np.log(_fit(orc, name, T / (1 + h))) - np.log(_fit(orc, name, T / (1 - h)))) / \
        ((1 + h) / T - (1 - h) / T)


def test_case_b_recombination_cooling_obeys_the_maxwellian_identity(orc):
    """For a rate that is a Maxwellian average of a cross-section, the kinetic energy carried
    away per unit volume is k T alpha (3/2 + d ln alpha / d ln T) exactly (differentiate
    alpha(T) = <sigma v> under the integral).  The case-B cooling fit must agree with the
    case-B recombination fit (pinned to the textbook table) to the fits' few-percent accuracy."""
    T = np.array([3e3, 5e3, 1e4, 2e4, 4e4, 1e5, 3e5])
    pred = KB * T * _fit(orc, "alpha_B", T) * (1.5 + _dlog_dlogT(orc, "alpha_B", T))
    assert np.all(np.abs(_fit(orc, "cool_rec_B", T) / pred - 1.0) < 0.02)


def test_case_a_recombination_cooling_near_the_maxwellian_identity(orc):
    """The same identity for case A.  The case-A cooling fit (Cen 1992, the paper's choice) is an
    older fit than the case-A recombination fit: it lies 11-13 % above the identity at the
    photo-ionized temperatures 3e3-1e4 K (and further above at higher T), so the pin is 15 %."""
    T = np.array([3e3, 5e3, 7e3, 1e4])
    pred = KB * T * _fit(orc, "alpha_A", T) * (1.5 + _dlog_dlogT(orc, "alpha_A", T))
    r = _fit(orc, "cool_rec_A", T) / pred
    assert np.all(np.abs(r - 1.0) < 0.15)


def test_collisional_rates_have_the_hydrogen_level_energies(orc):
    """At low T the collisional ionization rate and the excitation cooling are dominated by
    the Boltzmann factor of their thresholds: the ionization energy I_H and the n = 2
    excitation energy 3/4 I_H of the Bohr levels."""
    p = pins()
    T_ion = p["hydrogen_ionization_energy"] / p["boltzmann_constant_eV"]
    T = 300.0
    assert _activation_temperature(orc, "gamma_coll", T)[0] == pytest.approx(T_ion, rel=2e-3)
    assert _activation_temperature(orc, "cool_ci", T)[0] == pytest.approx(T_ion, rel=2e-3)
    assert _activation_temperature(orc, "cool_ce", T)[0] == pytest.approx(0.75 * T_ion, rel=2e-3)


def test_collisional_ionization_against_an_independent_fit(orc):
    """Voronov (1997)'s fit to the measured cross-sections, at the photo-ionized temperatures:
    the two fits agree within 20 % from 3e3 to 1e4 K (Cen's fit falls below Voronov's at higher
    T).  This also pins the fixed-temperature constant Gamma_coll(1e4 K)."""
    p = pins()
    T = np.array([3e3, 5e3, 7e3, 1e4])
    U = p["voronov_H_dE"] / (p["boltzmann_constant_eV"] * T)
    vor = p["voronov_H_A"] * (1 + p["voronov_H_P"] * np.sqrt(U)) * U ** p["voronov_H_K"] * np.exp(-U) / \
        (p["voronov_H_X"] + U)
    assert np.all(np.abs(_fit(orc, "gamma_coll", T) / vor - 1.0) < 0.20)
    from paper_1410_0763_gb300 import workloads as wl
    g1e4 = wl.hii_region(n=8, nside=1).chem["gcoll"]
    assert abs(g1e4 / vor[-1] - 1.0) < 0.20


def test_free_free_cooling_reaches_the_born_limit_at_high_temperature(orc):
    """Thermal bremsstrahlung per n_e n_i is C g T^1/2, C = 2^5 pi e^6 / (3 h m_e c^3)
    (2 pi k / (3 m_e))^1/2 (Rybicki & Lightman Eq. 5.15a), from the fundamental constants.
    In the Born approximation (k T >> I_H) the thermally averaged Gaunt factor at u = h nu / k T
    is (sqrt 3 / pi) e^{u/2} K_0(u/2), whose average over the emitted spectrum e^-u is
    2 sqrt 3 / pi (integrated numerically here).  At 1e9 K the fit must give that power within
    1 %; at every temperature its Gaunt factor must lie in Rybicki & Lightman's range."""
    from scipy import integrate, special
    p = pins()
    e, h, me, c, k = (p["electron_charge_esu"], p["planck_constant_cgs"], p["electron_mass_g"],
                      p["speed_of_light_cgs"], p["boltzmann_constant_cgs"])
    coef = 2 ** 5 * np.pi * e ** 6 / (3 * h * me * c ** 3) * np.sqrt(2 * np.pi * k / (3 * me))
    born = integrate.quad(lambda u: np.exp(-u) * np.sqrt(3) / np.pi * special.k0e(u / 2), 0, np.inf)[0]
    assert born == pytest.approx(2 * np.sqrt(3) / np.pi, rel=1e-6)
    assert _fit(orc, "cool_ff", 1e9)[0] / (coef * np.sqrt(1e9)) == pytest.approx(born, rel=1e-2)
    T = np.logspace(3, 9, 25)
    g = _fit(orc, "cool_ff", T) / (coef * np.sqrt(T))
    assert np.all((g > p["gaunt_range_lo"] * 0.99) & (g < p["gaunt_range_hi"]))
