"""FP64 CPU oracle for the diffuse-radiation ray-tracing scheme of Tanaka et al.
(2014) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (``paper_1410_0763_gb300``)
never imports it and shares no code with it.  The arithmetic lives in
``oracle.c`` (plain C, FP64); this module only compiles it with gcc and
marshals numpy arrays through ctypes.

Every function cites the passage of the paper it follows; see ``oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, -O2, OpenMP when present)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class SweepCfg(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("nside", C.c_int),
                ("tie_tol", C.c_double), ("field_form", C.c_int), ("nthreads", C.c_int),
                ("i_bc", C.c_double), ("averaging", C.c_int)]


class Chem(C.Structure):
    _fields_ = [("alphaA", C.c_double), ("alphaB", C.c_double), ("gcoll", C.c_double),
                ("sigma0", C.c_double), ("h", C.c_double), ("nu0", C.c_double),
                ("dnu", C.c_double), ("dx", C.c_double)]


class EvolveOpt(C.Structure):
    _fields_ = [("F", C.c_double), ("eps_iter", C.c_double), ("eps_e", C.c_double), ("eps_hi", C.c_double),
                ("dt_fixed", C.c_double), ("max_steps", C.c_int), ("max_iter", C.c_int), ("max_sub", C.c_int)]


class Thermal(C.Structure):
    _fields_ = [("on_the_spot", C.c_int), ("cool_mask", C.c_int), ("e_bin", C.c_double * 4),
                ("e_diff", C.c_double), ("z", C.c_double), ("kB", C.c_double), ("T_min", C.c_double),
                ("T_max", C.c_double)]


_D = C.POINTER(C.c_double)
_L = C.POINTER(C.c_long)


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = C.CDLL(path)
            lib.orc_n_dirs.argtypes = [C.c_int]
            lib.orc_healpix_dirs.argtypes = [C.c_int, _D]
            lib.orc_sweep_dir.argtypes = [C.POINTER(SweepCfg), _D, _D, C.c_int, _D, _D]
            lib.orc_sweep_range.argtypes = [C.POINTER(SweepCfg), _D, _D, C.c_int, C.c_int, _D]
            lib.orc_sweep_range.restype = C.c_long
            lib.orc_sweep_range_count.argtypes = [C.POINTER(SweepCfg), _D, _D, C.c_int, C.c_int, _D,
                                                  C.POINTER(C.c_longlong)]
            lib.orc_sweep_range_count.restype = C.c_long
            lib.orc_sweep.argtypes = [C.POINTER(SweepCfg), _D, _D, _D, _D]
            lib.orc_sweep.restype = C.c_long
            lib.orc_lattice.argtypes = [C.POINTER(SweepCfg), C.c_int, _L, C.POINTER(C.c_int), _D]
            lib.orc_trace_ray.argtypes = [C.POINTER(SweepCfg), _D, _D, C.c_int, C.c_long, C.c_long,
                                          _L, _D, _D, C.c_int, _D]
            lib.orc_jin_cells.argtypes = [C.POINTER(SweepCfg), _D, _D, _L, C.c_int, _D]
            lib.orc_band_integral.argtypes = [C.c_double] * 4
            lib.orc_band_integral.restype = C.c_double
            lib.orc_point_sources.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _D, _D, C.c_int,
                                              _D, _D, C.c_double, C.c_int, _D]
            lib.orc_balance_eq.argtypes = [C.c_long, _D, C.c_double, C.c_double, _D, _D]
            lib.orc_iterate.argtypes = [C.POINTER(SweepCfg), C.POINTER(Chem), _D, C.c_int, _D, _D,
                                        C.c_double, C.c_int, _D, _D, C.POINTER(C.c_int)]
            lib.orc_iterate_bins.argtypes = [C.POINTER(SweepCfg), C.POINTER(Chem), _D, C.c_int, _D, _D,
                                             C.c_int, _D, _D, C.c_double, C.c_int, _D, _D, C.POINTER(C.c_int)]
            lib.orc_iterate_ext.argtypes = [C.POINTER(SweepCfg), C.POINTER(Chem), _D, C.c_int, _D, _D,
                                            C.c_int, _D, _D, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                            _D, _D, C.POINTER(C.c_int)]
            lib.orc_point_sources_cells.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _D, _D, C.c_int, _D, _D,
                                                     C.c_double, _L, C.c_int, _D]
            lib.orc_plane_source.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _D, _D, C.c_int, C.c_int, _D, _D]
            lib.orc_evolve.argtypes = [C.POINTER(SweepCfg), C.POINTER(Chem), _D, C.c_int, _D, _D, C.c_int, _D, _D,
                                       C.c_int, C.c_int, C.c_double, C.POINTER(EvolveOpt), C.c_double, _D,
                                       C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double), _D]
            for f in ("alpha_A", "alpha_B", "gamma_coll", "cool_rec_A", "cool_rec_B", "cool_ci", "cool_ce",
                      "cool_ff"):
                getattr(lib, "orc_" + f).argtypes = [C.c_double]
                getattr(lib, "orc_" + f).restype = C.c_double
            lib.orc_compton_coef.argtypes = [C.c_double, C.c_double]
            lib.orc_compton_coef.restype = C.c_double
            TP = C.POINTER(Thermal)
            lib.orc_cooling.argtypes = [TP, C.c_double, C.c_double, C.c_double]
            lib.orc_cooling.restype = C.c_double
            lib.orc_cooling_deriv.argtypes = [TP, C.c_double, C.c_double, C.c_double]
            lib.orc_cooling_deriv.restype = C.c_double
            lib.orc_energy_step.argtypes = [TP] + [C.c_double] * 6
            lib.orc_energy_step.restype = C.c_double
            lib.orc_thermal_cell.argtypes = [TP] + [C.c_double] * 9 + [C.c_int, _D, _D]
            lib.orc_evolve_thermal.argtypes = [C.POINTER(SweepCfg), C.POINTER(Chem), TP, _D, C.c_int, _D, _D,
                                               C.c_int, _D, _D, C.c_int, C.c_int, C.c_double,
                                               C.POINTER(EvolveOpt), C.c_double, _D, _D, C.POINTER(C.c_int),
                                               C.POINTER(C.c_int), C.POINTER(C.c_double), _D]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def default_threads() -> int:
    return max(1, min(os.cpu_count() or 1, 64))


def _cfg(shape, nside, field_form=0, tie_tol=1e-12, nthreads=None, i_bc=0.0, averaging=0) -> SweepCfg:
    nz, ny, nx = shape
    return SweepCfg(nx, ny, nz, nside, tie_tol, int(field_form),
                    default_threads() if nthreads is None else int(nthreads), float(i_bc), int(averaging))


def n_dirs(nside: int) -> int:
    return 12 * nside * nside


def healpix_dirs(nside: int) -> np.ndarray:
    """HEALPix RING pixel centres as unit vectors, shape (12 nside^2, 3)."""
    out = np.empty((n_dirs(nside), 3))
    if _lib_handle().orc_healpix_dirs(nside, _dp(out)) != 0:
        raise ValueError("nside must be >= 1")
    return out


def sweep(kappa, src, nside, field_form=0, tie_tol=1e-12, nthreads=None, i_bc=0.0, averaging=0):
    """Full sweep (Sec. 2.2).  kappa, src: [z][y][x]; i_bc: intensity of every ray
    entering the box (0: vacuum); averaging 0: the paper's cell average, 1: the
    exact path average.  Returns (J_in, J, n_w_zero)."""
    k, s = _f64(kappa), _f64(src)
    jin = np.empty_like(k)
    j = np.empty_like(k)
    cfg = _cfg(k.shape, nside, field_form, tie_tol, nthreads, i_bc, averaging)
    nz = _lib_handle().orc_sweep(C.byref(cfg), _dp(k), _dp(s), _dp(jin), _dp(j))
    if nz < 0:
        raise MemoryError("oracle sweep: allocation failed")
    return jin, j, int(nz)


def sweep_range(kappa, src, nside, d0, d1, field_form=0, tie_tol=1e-12, nthreads=None):
    """Sum over directions d0..d1-1 (RING order) of Ibar^{ave,in}, not divided by N_d."""
    k, s = _f64(kappa), _f64(src)
    acc = np.empty_like(k)
    cfg = _cfg(k.shape, nside, field_form, tie_tol, nthreads)
    nz = _lib_handle().orc_sweep_range(C.byref(cfg), _dp(k), _dp(s), int(d0), int(d1), _dp(acc))
    if nz < 0:
        raise MemoryError("oracle sweep: allocation failed")
    return acc, int(nz)


def sweep_range_count(kappa, src, nside, d0, d1, field_form=0, tie_tol=1e-12, nthreads=None):
    """Like sweep_range, also returning the number of segments marched."""
    k, s = _f64(kappa), _f64(src)
    acc = np.empty_like(k)
    n = C.c_longlong(0)
    cfg = _cfg(k.shape, nside, field_form, tie_tol, nthreads)
    nz = _lib_handle().orc_sweep_range_count(C.byref(cfg), _dp(k), _dp(s), int(d0), int(d1), _dp(acc),
                                             C.byref(n))
    if nz < 0:
        raise MemoryError("oracle sweep: allocation failed")
    return acc, int(n.value)


def sweep_dir(kappa, src, nside, d, field_form=0, tie_tol=1e-12, i_bc=0.0, averaging=0):
    """Per-cell A (sum ds*Ibar_in, or the exact average's deposit) and W (sum ds) of one direction."""
    k, s = _f64(kappa), _f64(src)
    A = np.empty_like(k)
    W = np.empty_like(k)
    cfg = _cfg(k.shape, nside, field_form, tie_tol, 1, i_bc, averaging)
    if _lib_handle().orc_sweep_dir(C.byref(cfg), _dp(k), _dp(s), int(d), _dp(A), _dp(W)) != 0:
        raise ValueError("bad direction index")
    return A, W


def lattice(shape, nside, d, tie_tol=1e-12):
    """(jlo, jhi, klo, khi), (a, b, c, sign_a), (qb, qc, |n_a|) of direction d."""
    r = np.zeros(4, dtype=np.int64)
    ax = (C.c_int * 4)()
    q = np.zeros(3)
    cfg = _cfg(shape, nside, 0, tie_tol, 1)
    if _lib_handle().orc_lattice(C.byref(cfg), int(d), r.ctypes.data_as(_L), ax, _dp(q)) != 0:
        raise ValueError("bad direction index")
    return tuple(int(v) for v in r), tuple(ax), tuple(q)


def trace_ray(kappa, src, nside, d, j, k, field_form=0, tie_tol=1e-12, maxseg=100000, i_bc=0.0):
    """Segments (cell, ds, I_in) of lattice ray (j, k) of direction d, and the exit intensity."""
    kk, s = _f64(kappa), _f64(src)
    cells = np.zeros(maxseg, dtype=np.int64)
    ds = np.zeros(maxseg)
    iin = np.zeros(maxseg)
    iex = C.c_double(0.0)
    cfg = _cfg(kk.shape, nside, field_form, tie_tol, 1, i_bc)
    n = _lib_handle().orc_trace_ray(C.byref(cfg), _dp(kk), _dp(s), int(d), int(j), int(k),
                                    cells.ctypes.data_as(_L), _dp(ds), _dp(iin), maxseg,
                                    C.byref(iex))
    if n < 0 or n > maxseg:
        raise ValueError("trace_ray failed")
    return cells[:n].copy(), ds[:n].copy(), iin[:n].copy(), iex.value


def jin_cells(kappa, src, nside, cells, field_form=0, tie_tol=1e-12, nthreads=None, i_bc=0.0, averaging=0):
    """J^in at the given flat cell indices, computed one cell at a time."""
    k, s = _f64(kappa), _f64(src)
    c = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
    out = np.empty(c.shape[0])
    cfg = _cfg(k.shape, nside, field_form, tie_tol, nthreads, i_bc, averaging)
    bad = _lib_handle().orc_jin_cells(C.byref(cfg), _dp(k), _dp(s), c.ctypes.data_as(_L),
                                      int(c.shape[0]), _dp(out))
    if bad:
        raise RuntimeError(f"{bad} (cell, direction) pairs with no ray")
    return out


def band_integral(sigma0, h, nu0, nu1) -> float:
    """int_{nu0}^{nu1} sigma(nu)/(h nu) dnu for sigma = sigma0 (nu/nu0)^-3 (Eq. gamma_diff)."""
    return float(_lib_handle().orc_band_integral(sigma0, h, nu0, nu1))


def point_sources(kappa_bins, sigma_bins, pos, Q, dx, nthreads=None):
    """Photon-conserving point-source rate per neutral atom (App. A).

    kappa_bins: [bins][z][y][x] (per cell width); sigma_bins: [bins] cm^2;
    pos: [nsrc][3] in cell widths (x, y, z); Q: [nsrc][bins] photons/s.
    """
    kb = _f64(kappa_bins)
    if kb.ndim == 3:
        kb = kb[None]
    nb, nz, ny, nx = kb.shape
    sg = _f64(sigma_bins).reshape(nb)
    p = _f64(pos).reshape(-1, 3)
    q = _f64(Q).reshape(p.shape[0], nb)
    out = np.empty((nz, ny, nx))
    _lib_handle().orc_point_sources(nx, ny, nz, nb, _dp(kb), _dp(sg), p.shape[0], _dp(p), _dp(q),
                                    float(dx), default_threads() if nthreads is None else nthreads,
                                    _dp(out))
    return out


def balance_eq(nH, alphaB, gcoll, g):
    """Equilibrium neutral fraction y (App. B, dt -> infinity)."""
    n = _f64(nH)
    gg = _f64(g)
    y = np.empty_like(n)
    _lib_handle().orc_balance_eq(n.size, _dp(n), float(alphaB), float(gcoll), _dp(gg), _dp(y))
    return y


def point_sources_cells(kappa_bins, sigma, pos, Qb, dx, cells):
    """Point-source rates (App. A) at the given flat cell indices only; arguments as point_sources."""
    k = _f64(kappa_bins)
    if k.ndim == 3:
        k = k[None]
    nb = k.shape[0]
    nz, ny, nx = k.shape[1:]
    sig = _f64(sigma).reshape(nb)
    p = _f64(pos).reshape(-1, 3)
    q = _f64(Qb).reshape(p.shape[0], nb)
    c = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
    out = np.empty(c.shape[0])
    if _lib_handle().orc_point_sources_cells(nx, ny, nz, nb, _dp(k), _dp(sig), p.shape[0], _dp(p), _dp(q), float(dx),
                                             c.ctypes.data_as(_L), int(c.shape[0]), _dp(out)) != 0:
        raise ValueError("cell index out of range")
    return out


def plane_source(kappa_bins, sigma, axis, direction, flux):
    """Photo-ionization rate of a plane-parallel incident flux (the Test-3 setup, Sec. 4.3): flux[b]
    photons/s/cm^2 in bin b travelling along +axis (direction 1) or -axis (-1); axis 0, 1, 2 = x, y, z.
    kappa_bins: [bin][z][y][x] per cell width.  Returns Gamma [z][y][x] in s^-1."""
    k = _f64(kappa_bins)
    if k.ndim == 3:
        k = k[None]
    nb = k.shape[0]
    sig = _f64(sigma).reshape(nb)
    F = _f64(flux).reshape(nb)
    nz, ny, nx = k.shape[1:]
    out = np.empty((nz, ny, nx))
    if _lib_handle().orc_plane_source(nx, ny, nz, nb, _dp(k), _dp(sig), int(axis), int(direction), _dp(F),
                                      _dp(out)) != 0:
        raise ValueError("axis must be 0-2 and direction +-1")
    return out


def iterate(nH, nside, chem: dict, pos, Q, y0, tol=1e-6, max_iter=200, nthreads=None, sigma_bins=None,
            frac_bins=None, plane=None):
    """RT / balance fixed-point iteration (App. D).  Point sources emit Q * frac_b in bin b with cross
    section sigma_b (default: one bin at sigma0); plane = (axis, direction, flux) adds a plane-parallel
    incident flux split over the bins the same way.  Returns (y, iters, residuals, converged)."""
    n = _f64(nH)
    y = _f64(y0).copy()
    p = _f64(pos).reshape(-1, 3)
    q = _f64(Q).reshape(p.shape[0])
    sig = _f64([chem["sigma0"]] if sigma_bins is None else sigma_bins)
    frac = _f64([1.0] if frac_bins is None else frac_bins)
    hist = np.zeros(max_iter)
    it = C.c_int(0)
    ch = Chem(chem["alphaA"], chem["alphaB"], chem["gcoll"], chem["sigma0"], chem["h"],
              chem["nu0"], chem["dnu"], chem["dx"])
    cfg = _cfg(n.shape, nside, 1, 1e-12, nthreads)
    pa, pd, pf = plane if plane is not None else (0, 1, 0.0)
    rc = _lib_handle().orc_iterate_ext(C.byref(cfg), C.byref(ch), _dp(n), p.shape[0], _dp(p), _dp(q),
                                       int(sig.size), _dp(sig), _dp(frac), int(pa), int(pd), float(pf),
                                       float(tol), int(max_iter), _dp(y), _dp(hist), C.byref(it))
    if rc < 0:
        raise MemoryError("oracle iterate: allocation failed")
    return y, it.value, hist[: it.value].copy(), rc == 0



def evolve(nH, nside, chem: dict, pos, Q, y0, t_end, F=10.0, eps_iter=1e-3, eps_e=0.2, eps_hi=0.002,
           dt_fixed=0.0, max_steps=100000, max_iter=100, max_sub=1000000, sigma_bins=None, frac_bins=None,
           plane=None, nthreads=None):
    """Time-dependent mode (App. B-D) at fixed temperature from t = 0 to t_end (s).  Returns
    (y, steps, iterations, t_reached, dts, rc): rc 0 when t_end is reached with every step converged,
    1 if some step's iteration hit max_iter, 2 if max_steps ran out."""
    n = _f64(nH)
    y = _f64(y0).copy()
    p = _f64(pos).reshape(-1, 3)
    q = _f64(Q).reshape(p.shape[0])
    sig = _f64([chem["sigma0"]] if sigma_bins is None else sigma_bins)
    frac = _f64([1.0] if frac_bins is None else frac_bins)
    ch = Chem(chem["alphaA"], chem["alphaB"], chem["gcoll"], chem["sigma0"], chem["h"],
              chem["nu0"], chem["dnu"], chem["dx"])
    cfg = _cfg(n.shape, nside, 1, 1e-12, nthreads)
    pa, pd, pf = plane if plane is not None else (0, 1, 0.0)
    opt = EvolveOpt(float(F), float(eps_iter), float(eps_e), float(eps_hi), float(dt_fixed), int(max_steps),
                    int(max_iter), int(max_sub))
    dts = np.zeros(max_steps)
    steps, iters, t = C.c_int(0), C.c_int(0), C.c_double(0.0)
    rc = _lib_handle().orc_evolve(C.byref(cfg), C.byref(ch), _dp(n), p.shape[0], _dp(p), _dp(q), int(sig.size),
                                  _dp(sig), _dp(frac), int(pa), int(pd), float(pf), C.byref(opt), float(t_end),
                                  _dp(y), C.byref(steps), C.byref(iters), C.byref(t), _dp(dts))
    if rc < 0:
        raise MemoryError("oracle evolve: allocation failed")
    return y, steps.value, iters.value, t.value, dts[: steps.value].copy(), rc


def _thermal(th: dict) -> Thermal:
    e = list(th.get("e_bin", [0.0])) + [0.0] * 4
    return Thermal(int(th.get("on_the_spot", 0)), int(th.get("cool_mask", 31)), (C.c_double * 4)(*e[:4]),
                   float(th.get("e_diff", 0.0)), float(th.get("z", -1.0)), float(th["kB"]),
                   float(th.get("T_min", 10.0)), float(th.get("T_max", 1e9)))


def rate_fit(name: str, T, z: float = 0.0, kB: float = 1.380649e-16):
    """Temperature fits of the energy equation (App. C; see oracle.c for the sources):
    alpha_A, alpha_B, gamma_coll (cm^3/s); cool_rec_A, cool_rec_B, cool_ci, cool_ce, cool_ff
    (erg cm^3/s); compton (erg/s/K per electron, independent of T)."""
    lib = _lib_handle()
    if name == "compton":
        return float(lib.orc_compton_coef(float(z), float(kB)))
    f = getattr(lib, "orc_" + name)
    return np.array([f(float(t)) for t in np.atleast_1d(np.asarray(T, dtype=np.float64))])


def cooling(th: dict, nH: float, y: float, T: float) -> float:
    """Cooling rate C(n, T) in erg/s/cm^3 (App. C) of hydrogen with neutral fraction y."""
    t = _thermal(th)
    return float(_lib_handle().orc_cooling(C.byref(t), float(nH), float(y), float(T)))


def cooling_deriv(th: dict, nH: float, y: float, T: float) -> float:
    """dC/dT (erg/s/cm^3/K) of `cooling`, from the fits' analytic logarithmic derivatives."""
    t = _thermal(th)
    return float(_lib_handle().orc_cooling_deriv(C.byref(t), float(nH), float(y), float(T)))


def energy_step(th: dict, nH, y0, T0, y1, H1, dt) -> float:
    """The implicit energy update of App. C for one cell: T at t + dt."""
    t = _thermal(th)
    return float(_lib_handle().orc_energy_step(C.byref(t), float(nH), float(y0), float(T0), float(y1),
                                               float(H1), float(dt)))


def thermal_cell(th: dict, nH, y0, T0, gpt, hpt, gdiff, dt, eps_e=0.2, eps_hi=0.002, max_sub=1000000):
    """One cell over dt at fixed rates: chemistry sub-steps (App. B, D) each followed by the
    implicit energy update (App. C).  Returns (y, T, sub-steps)."""
    t = _thermal(th)
    y, T = C.c_double(0.0), C.c_double(0.0)
    n = _lib_handle().orc_thermal_cell(C.byref(t), float(nH), float(y0), float(T0), float(gpt), float(hpt),
                                       float(gdiff), float(dt), float(eps_e), float(eps_hi), int(max_sub),
                                       C.byref(y), C.byref(T))
    return y.value, T.value, n


def evolve_thermal(nH, nside, chem: dict, thermal: dict, pos, Q, y0, T0, t_end, F=10.0, eps_iter=1e-3,
                   eps_e=0.2, eps_hi=0.002, dt_fixed=0.0, max_steps=100000, max_iter=100, max_sub=1000000,
                   sigma_bins=None, frac_bins=None, plane=None, nthreads=None):
    """Time-dependent mode with the energy equation (App. B-D) from t = 0 to t_end (s).  Returns
    (y, T, steps, iterations, t_reached, dts, rc), rc as in `evolve`."""
    n = _f64(nH)
    y = _f64(y0).copy()
    T = np.broadcast_to(_f64(T0), n.shape).copy()
    p = _f64(pos).reshape(-1, 3)
    q = _f64(Q).reshape(p.shape[0])
    sig = _f64([chem["sigma0"]] if sigma_bins is None else sigma_bins)
    frac = _f64([1.0] if frac_bins is None else frac_bins)
    ch = Chem(chem["alphaA"], chem["alphaB"], chem["gcoll"], chem["sigma0"], chem["h"],
              chem["nu0"], chem["dnu"], chem["dx"])
    th = _thermal(thermal)
    cfg = _cfg(n.shape, nside, 1, 1e-12, nthreads)
    pa, pd, pf = plane if plane is not None else (0, 1, 0.0)
    opt = EvolveOpt(float(F), float(eps_iter), float(eps_e), float(eps_hi), float(dt_fixed), int(max_steps),
                    int(max_iter), int(max_sub))
    dts = np.zeros(max_steps)
    steps, iters, t = C.c_int(0), C.c_int(0), C.c_double(0.0)
    rc = _lib_handle().orc_evolve_thermal(C.byref(cfg), C.byref(ch), C.byref(th), _dp(n), p.shape[0], _dp(p),
                                          _dp(q), int(sig.size), _dp(sig), _dp(frac), int(pa), int(pd), float(pf),
                                          C.byref(opt), float(t_end), _dp(y), _dp(T), C.byref(steps),
                                          C.byref(iters), C.byref(t), _dp(dts))
    if rc < 0:
        raise MemoryError("oracle evolve_thermal: allocation failed")
    return y, T, steps.value, iters.value, t.value, dts[: steps.value].copy(), rc


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
