"""Seeded synthetic inputs for the diffuse-radiation sweep and the RT/ionization
iteration.

This module holds input recipes only -- random fields, grid shapes, physical
constants and source lists -- and none of the method's arithmetic.  The tests
feed the same arrays to the CUDA path and to the FP64 oracle; the benchmark
uses the same recipes.

Workloads (the paper's own test problems are parameter recipes in its text,
Sec. 4, not datasets; these stand in for them):

* ``lognormal_iid``   -- 16^3, N_side 1: kappa = 0.5 exp(Z), Z ~ N(0,1) i.i.d.
  per cell, S ~ U[0,1) (seed 1).  FP64 path.
* ``grf``             -- 64^3, N_side 4: periodic Gaussian random field with
  power spectrum P(k) ~ k^-3, lognormal density rho = exp(s g - s^2/2), s = 1,
  kappa = rho/<rho> * tau_box/N (tau_box = 10), S = rho/<rho> (seed 2).
* ``hii_region``      -- 128^3, N_side 8: uniform n_H = 1e-3 cm^-3, T = 1e4 K,
  box 6.6 kpc, one source of 5e48 ionizing photons/s at the box centre,
  x0 = 1e-4 (the Test-1 medium of Sec. 4.1 with the source moved to the centre).
* ``batch48``         -- 48 grids, N in {32,48,64,96}, N_side in {2,4,8}, the
  ``grf`` recipe with s ~ U[0.5,1.5] (seed 4 + grid index).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Physical constants (cgs) and hydrogen rate coefficients at T = 1e4 K.
# alpha_B is the value implied by the paper's printed recombination time
# (t_rec = 122.4 Myr at n_H = 1e-3, Sec. 4.1) and Stromgren radius (5.4 kpc);
# sigma0 is implied by the printed mean free path (51.4 pc at n_HI = 1e-3,
# Sec. 4.2).  alpha_A and the collisional ionization rate come from the fits
# the paper cites (Table tab:rate) and are not printed in it.
# ---------------------------------------------------------------------------
H_PLANCK = 6.62607015e-27      # erg s
K_BOLTZ = 1.380649e-16         # erg / K
NU0 = 3.2898419603e15          # Hz, hydrogen ionization threshold (13.6 eV)
KPC = 3.0856775814913673e21    # cm
PC = KPC * 1e-3
MYR = 3.15576e13               # s
SIGMA0 = 6.30e-18              # cm^2, HI cross section at nu0
ALPHA_B_1E4 = 2.59e-13         # cm^3/s, case B at 1e4 K
ALPHA_A_1E4 = 4.18e-13         # cm^3/s, case A at 1e4 K
GAMMA_COLL_1E4 = 6.24e-16      # cm^3/s, HI collisional ionization at 1e4 K


def chem_constants(T: float = 1e4, dx_cm: float = 6.6 * KPC / 128) -> dict:
    """Rate coefficients and spectral constants for the fixed-temperature runs."""
    if T != 1e4:
        raise ValueError("only T = 1e4 K is tabulated")
    return dict(alphaA=ALPHA_A_1E4, alphaB=ALPHA_B_1E4, gcoll=GAMMA_COLL_1E4, sigma0=SIGMA0,
                h=H_PLANCK, nu0=NU0, dnu=K_BOLTZ * T / H_PLANCK, dx=dx_cm)


# ---------------------------------------------------------------------------
# Random fields
# ---------------------------------------------------------------------------
def gaussian_random_field(n: int, slope: float, rng: np.random.Generator) -> np.ndarray:
    """Periodic Gaussian random field on n^3, P(k) ~ k^slope, zero mean, unit variance."""
    w = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(w)
    kz = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kx = np.fft.rfftfreq(n)[None, None, :]
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** (0.5 * slope)
    g = np.fft.irfftn(wk * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g


def lognormal_density(n: int, sigma: float, slope: float, rng: np.random.Generator) -> np.ndarray:
    """rho/<rho> for rho = exp(sigma g - sigma^2/2), g a unit-variance GRF."""
    g = gaussian_random_field(n, slope, rng)
    rho = np.exp(sigma * g - 0.5 * sigma * sigma)
    return rho / rho.mean()


# ---------------------------------------------------------------------------
# Sweep workloads
# ---------------------------------------------------------------------------
@dataclass
class SweepCase:
    name: str
    nside: int
    kappa: np.ndarray          # [bins][z][y][x] or [z][y][x], per cell width
    src: np.ndarray            # same shape: S (field_form 0) or eps*dx (field_form 1)
    field_form: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.kappa.shape[-3:]


def lognormal_iid(n: int = 16, nside: int = 1, seed: int = 1) -> SweepCase:
    rng = np.random.default_rng(seed)
    kappa = 0.5 * np.exp(rng.standard_normal((n, n, n)))
    S = rng.random((n, n, n))
    return SweepCase("lognormal_iid", nside, kappa, S, 0, dict(seed=seed, n=n))


def grf(n: int = 64, nside: int = 4, seed: int = 2, sigma: float = 1.0, slope: float = -3.0,
        tau_box: float = 10.0) -> SweepCase:
    rng = np.random.default_rng(seed)
    rho = lognormal_density(n, sigma, slope, rng)
    kappa = rho * (tau_box / n)
    S = rho.copy()
    return SweepCase("grf", nside, kappa, S, 0,
                     dict(seed=seed, n=n, sigma=sigma, slope=slope, tau_box=tau_box))


def batch48(seed0: int = 4, count: int = 48):
    """48 grids of uneven size and angular resolution (grf recipe per grid)."""
    meta_rng = np.random.default_rng(seed0 * 1000 + 7)
    sizes = meta_rng.choice([32, 48, 64, 96], size=count)
    nsides = meta_rng.choice([2, 4, 8], size=count)
    sigmas = meta_rng.uniform(0.5, 1.5, size=count)
    return [grf(int(sizes[i]), int(nsides[i]), seed0 + i, float(sigmas[i])) for i in range(count)]


# ---------------------------------------------------------------------------
# Ionization workloads
# ---------------------------------------------------------------------------
@dataclass
class HIICase:
    name: str
    nside: int
    n: int
    nH: np.ndarray             # [z][y][x] cm^-3
    y0: np.ndarray             # initial neutral fraction
    pos: np.ndarray            # [nsrc][3] (x, y, z) in cell widths
    Q: np.ndarray              # [nsrc] photons/s
    chem: dict
    tol: float = 1e-6
    box_cm: float = 6.6 * KPC
    plane: tuple | None = None  # (axis, direction, photons/s/cm^2) of a plane-parallel incident flux


def hii_region(n: int = 128, nside: int = 8, box_kpc: float = 6.6, nH: float = 1e-3,
               Q: float = 5e48, x0: float = 1e-4, source_at: str = "center") -> HIICase:
    dx = box_kpc * KPC / n
    pos = np.array([[n / 2, n / 2, n / 2]]) if source_at == "center" else np.array([[0.0, 0.0, 0.0]])
    return HIICase("hii_region", nside, n, np.full((n, n, n), nH), np.full((n, n, n), 1.0 - x0),
                   pos, np.array([Q]), chem_constants(1e4, dx), 1e-6, box_kpc * KPC)


def hii_random(n: int = 128, nside: int = 8, seed: int = 100, box_kpc: float = 6.6, nH_mean: float = 1e-3,
               x0: float = 1e-4) -> HIICase:
    """Surrogate training setup: lognormal density (sigma uniform in [0, 1.5],
    P(k) ~ k^-3, mean nH_mean), 1-8 sources uniform in the box with Q uniform in
    [1e48, 1e49] s^-1."""
    rng = np.random.default_rng(seed)
    sigma = float(rng.uniform(0.0, 1.5))
    rho = lognormal_density(n, sigma, -3.0, rng) if sigma > 0 else np.ones((n, n, n))
    nsrc = int(rng.integers(1, 9))
    pos = rng.uniform(0.5, n - 0.5, size=(nsrc, 3))
    Q = rng.uniform(1e48, 1e49, size=nsrc)
    dx = box_kpc * KPC / n
    return HIICase("hii_random", nside, n, nH_mean * rho, np.full((n, n, n), 1.0 - x0), pos, Q,
                   chem_constants(1e4, dx), 1e-6, box_kpc * KPC)


def shadow_clump(n: int = 128, nside: int = 8, box_kpc: float = 6.6, nH: float = 2e-4,
                 overdensity: float = 200.0, r_kpc: float = 0.8, offset_kpc: float = 1.7,
                 flux: float = 1e6, x0: float = 1e-4) -> HIICase:
    """The geometry of the paper's Test 3 (Sec. 4.3): uniform n_H with a sphere
    of radius r_kpc at overdensity x n_H, centred offset_kpc from the box
    centre along +x, lit by a plane-parallel photon flux (photons/s/cm^2)
    entering the x = 0 face along +x.  No point sources.  The gas is held at
    1e4 K (the rates of chem_constants), not at the paper's 8000 K / 40 K."""
    dx = box_kpc * KPC / n
    c = (np.arange(n) + 0.5) * dx
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    mid = 0.5 * box_kpc * KPC
    r2 = (x - mid - offset_kpc * KPC) ** 2 + (y - mid) ** 2 + (z - mid) ** 2
    dens = np.where(r2 <= (r_kpc * KPC) ** 2, overdensity * nH, nH)
    return HIICase("shadow_clump", nside, n, dens, np.full((n, n, n), 1.0 - x0), np.zeros((0, 3)),
                   np.zeros(0), chem_constants(1e4, dx), 1e-6, box_kpc * KPC, (0, 1, flux))


def point_clump(n: int = 128, nside: int = 8, box_kpc: float = 6.6, nH: float = 1e-3, overdensity: float = 200.0,
                r_kpc: float = 0.56, offset_kpc: float = 0.8, Q: float = 5e48, x0: float = 1e-4) -> HIICase:
    """The geometry of the paper's Test 2 (Sec. 4.2): a point source of Q
    photons/s at the box centre, uniform n_H, and a sphere of radius r_kpc at
    overdensity x n_H centred offset_kpc from the source along +x."""
    dx = box_kpc * KPC / n
    c = (np.arange(n) + 0.5) * dx
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    mid = 0.5 * box_kpc * KPC
    r2 = (x - mid - offset_kpc * KPC) ** 2 + (y - mid) ** 2 + (z - mid) ** 2
    dens = np.where(r2 <= (r_kpc * KPC) ** 2, overdensity * nH, nH)
    return HIICase("point_clump", nside, n, dens, np.full((n, n, n), 1.0 - x0), np.array([[n / 2, n / 2, n / 2]]),
                   np.array([Q]), chem_constants(1e4, dx), 1e-6, box_kpc * KPC)


def blackbody_bins(T: float = 1e5, edges_ev=(13.6, 24.6, 54.4, 100.0, 500.0), n_quad: int = 4000):
    """Photon fractions and photon-weighted cross sections of a blackbody of
    temperature T over bins above the HI threshold (hydrogenic sigma0 (nu/nu0)^-3):
    frac_b = int_b B_nu/(h nu) / int_all, sigma_b = int_b sigma n_nu / int_b n_nu.
    Returns (frac [nb], sigma [nb], edges in Hz)."""
    ev = 1.602176634e-12
    nu_edges = np.array(edges_ev) * ev / H_PLANCK
    x = lambda nu: H_PLANCK * nu / (K_BOLTZ * T)
    frac, sig = [], []
    for lo, hi in zip(nu_edges[:-1], nu_edges[1:]):
        nu = np.linspace(lo, hi, n_quad)
        n_nu = nu ** 2 / np.expm1(x(nu))              # photon number per frequency (B_nu / h nu)
        s = SIGMA0 * (nu / NU0) ** -3
        w = np.trapezoid(n_nu, nu)
        frac.append(w)
        sig.append(np.trapezoid(s * n_nu, nu) / w)
    frac = np.array(frac) / np.sum(frac)
    return frac, np.array(sig), nu_edges


def blackbody_heat(T: float = 1e5, edges_ev=(13.6, 24.6, 54.4, 100.0, 500.0), n_quad: int = 4000):
    """Mean energy above the HI threshold (erg) of a photo-ionization by each bin of a
    blackbody of temperature T (the bins of `blackbody_bins`):
    e_b = int_b sigma n_nu (h nu - h nu0) / int_b sigma n_nu."""
    ev = 1.602176634e-12
    nu_edges = np.array(edges_ev) * ev / H_PLANCK
    out = []
    for lo, hi in zip(nu_edges[:-1], nu_edges[1:]):
        nu = np.linspace(lo, hi, n_quad)
        w = SIGMA0 * (nu / NU0) ** -3 * nu ** 2 / np.expm1(H_PLANCK * nu / (K_BOLTZ * T))
        out.append(np.trapezoid(w * H_PLANCK * (nu - NU0), nu) / np.trapezoid(w, nu))
    return np.array(out)


def diffuse_band_heat(chem: dict, n_quad: int = 4000) -> float:
    """Mean energy above threshold (erg) of a photo-ionization by the recombination
    band [nu0, nu0 + dnu] with a flat J_nu: int sigma/(h nu) (h nu - h nu0) / int sigma/(h nu)."""
    nu = np.linspace(chem["nu0"], chem["nu0"] + chem["dnu"], n_quad)
    w = (nu / chem["nu0"]) ** -3 / nu
    return float(np.trapezoid(w * chem["h"] * (nu - chem["nu0"]), nu) / np.trapezoid(w, nu))


def clumpy_sweep(n: int = 256, nside: int = 8, seed: int = 5, tau_box: float = 10.0, nbins: int = 4) -> SweepCase:
    """Sweep input on the clumpy medium of `clumpy` (lognormal sigma 1.5, P(k) ~ k^-3, plus 200
    spheres at 100x the mean density; seed 5), in the 4 bins of a 1e5 K blackbody above 13.6 eV:
    kappa_b = rho/<rho> * tau_box/N * sigma_b/sigma_0 (the grf recipe's box optical depth 10 in
    the first bin, sigma_b the bins' photon-weighted cross sections) and S_b = rho/<rho> in every
    bin.  Arrays are [bin][z][y][x]."""
    case = clumpy(n=n, nside=nside, seed=seed)
    rho = case.nH / case.nH.mean()
    _, sig, _ = blackbody_bins()
    sig = sig[:nbins]
    kappa = np.stack([rho * (tau_box / n) * (s / SIGMA0) for s in sig])
    src = np.stack([rho] * nbins)
    return SweepCase("clumpy_sweep", nside, kappa, src, 0, dict(seed=seed, n=n, tau_box=tau_box, nbins=nbins,
                                                                 sigma_ratio=[float(s / SIGMA0) for s in sig]))


def clumpy(n: int = 256, nside: int = 8, seed: int = 5, sigma: float = 1.5, n_clumps: int = 200,
           overdensity: float = 100.0, n_src: int = 8, Q: float = 5e48, box_kpc: float = 6.6,
           nH_mean: float = 1e-3, x0: float = 1e-4) -> HIICase:
    """Clumpy medium: lognormal density (sigma, P(k) ~ k^-3) plus n_clumps spheres
    (centres uniform, radius uniform in [2, 8] cells) at overdensity x the mean,
    then scaled to mean n_H nH_mean; n_src sources of Q photons/s at uniform
    positions."""
    rng = np.random.default_rng(seed)
    rho = lognormal_density(n, sigma, -3.0, rng)
    centres = rng.uniform(0, n, size=(n_clumps, 3))
    radii = rng.uniform(2.0, 8.0, size=n_clumps)
    g = np.arange(n) + 0.5
    for c, r in zip(centres, radii):
        lo = np.maximum(np.floor(c - r).astype(int), 0)
        hi = np.minimum(np.ceil(c + r).astype(int) + 1, n)
        zz, yy, xx = np.meshgrid(g[lo[2]:hi[2]], g[lo[1]:hi[1]], g[lo[0]:hi[0]], indexing="ij")
        inside = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= r * r
        blk = rho[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        blk[inside] = overdensity
    rho /= rho.mean()
    pos = rng.uniform(0.5, n - 0.5, size=(n_src, 3))
    dx = box_kpc * KPC / n
    return HIICase("clumpy", nside, n, nH_mean * rho, np.full((n, n, n), 1.0 - x0), pos, np.full(n_src, Q),
                   chem_constants(1e4, dx), 1e-6, box_kpc * KPC)
