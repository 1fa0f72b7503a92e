"""Thin ctypes binding of libart (include/art.h).

Argument marshalling only: every step of the sweep runs in the CUDA library.
The module-level functions carry the C names; :class:`ArtSweep` wraps one
context.  Buffers are torch CUDA tensors (device pointers, stream-ordered on
the current torch stream) or numpy arrays (host pointers; the call copies and
synchronizes).  Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

ART_OK, ART_E_INVALID, ART_E_CUDA, ART_E_OOM, ART_E_NOT_CONVERGED, ART_E_TIMEOUT, ART_E_STATE = range(7)
ART_FP32, ART_FP64 = 0, 1
ART_AVG_PAPER, ART_AVG_EXACT = 0, 1
ART_FIELDS_S, ART_FIELDS_EPS = 0, 1
_STATUS = {0: "ART_OK", 1: "ART_E_INVALID", 2: "ART_E_CUDA", 3: "ART_E_OOM",
           4: "ART_E_NOT_CONVERGED", 5: "ART_E_TIMEOUT", 6: "ART_E_STATE"}


class ArtGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx_cm", C.c_double)]


class ArtOptions(C.Structure):
    _fields_ = [("precision", C.c_int), ("averaging", C.c_int), ("field_form", C.c_int),
                ("tile_b", C.c_int), ("tile_c", C.c_int), ("slab", C.c_int), ("dir_split", C.c_int),
                ("tie_tol", C.c_double), ("variant", C.c_int), ("persistent", C.c_int), ("graph", C.c_int),
                ("dir_begin", C.c_int), ("dir_end", C.c_int), ("early_launch", C.c_int)]


class ArtSweepStats(C.Structure):
    _fields_ = [("segments", C.c_int64), ("n_dirs", C.c_int32), ("n_classes", C.c_int32),
                ("launches", C.c_int32), ("ctas_per_launch", C.c_int32), ("tile_b", C.c_int32),
                ("tile_c", C.c_int32), ("slab", C.c_int32), ("dir_split", C.c_int32),
                ("device_bytes", C.c_int64), ("variant", C.c_int32), ("group", C.c_int32),
                ("n_grids", C.c_int32), ("work_items", C.c_int32), ("persistent", C.c_int32),
                ("bins_per_launch", C.c_int32)]


class ArtChem(C.Structure):
    _fields_ = [("alphaA", C.c_double), ("alphaB", C.c_double), ("gcoll", C.c_double), ("sigma0", C.c_double),
                ("h", C.c_double), ("nu0", C.c_double), ("dnu", C.c_double)]


class ArtEvolveOptions(C.Structure):
    _fields_ = [("t_end", C.c_double), ("F", C.c_double), ("eps_iter", C.c_double), ("eps_e", C.c_double),
                ("eps_hi", C.c_double), ("dt_fixed", C.c_double), ("max_steps", C.c_int), ("max_iter", C.c_int),
                ("max_sub", C.c_int)]


class ArtEvolveReport(C.Structure):
    _fields_ = [("steps", C.c_int32), ("iterations", C.c_int32), ("sweeps", C.c_int32), ("converged", C.c_int32),
                ("sub_overflow", C.c_int64), ("t", C.c_double), ("dt_min", C.c_double), ("dt_max", C.c_double),
                ("seconds", C.c_double)]


class ArtThermal(C.Structure):
    _fields_ = [("on_the_spot", C.c_int32), ("cool_mask", C.c_int32), ("e_bin", C.c_double * 4),
                ("e_diff", C.c_double), ("z", C.c_double), ("kB", C.c_double), ("T_min", C.c_double),
                ("T_max", C.c_double)]


class ArtSource(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("z", C.c_double), ("Q", C.c_double)]


class ArtIterReport(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("residual", C.c_double),
                ("seconds", C.c_double)]


class ArtProfile(C.Structure):
    _fields_ = [("sweep_ms", C.c_double), ("sweep_launches", C.c_int64), ("reduce_ms", C.c_double),
                ("reduce_launches", C.c_int64)]


class ArtNetOptions(C.Structure):
    _fields_ = [("dilation", C.c_int * 4), ("seed", C.c_uint64), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("adam_eps", C.c_double)]


class ArtWarmOptions(C.Structure):
    _fields_ = [("coarse_factor", C.c_int), ("coarse_nside", C.c_int), ("use_net", C.c_int),
                ("phase1_max_iter", C.c_int), ("phase1_tol", C.c_double), ("judge_tol", C.c_double),
                ("coarse_solve", C.c_int), ("coarse_tol", C.c_double), ("judge_after", C.c_int)]


class ArtWarmReport(C.Structure):
    _fields_ = [("total", ArtIterReport), ("surrogate_iterations", C.c_int32), ("plain_sweeps", C.c_int32),
                ("fell_back", C.c_int32), ("judge_error", C.c_double), ("coarse_iterations", C.c_int32)]


ART_NET_PARAMS = 59713
NET_LAYERS = [(4, 32), (32, 32), (32, 32), (32, 1)]   # (c_in, c_out)


class ArtDataset(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("n_samples", C.c_int),
                ("X", C.c_void_p), ("t", C.c_void_p), ("w", C.c_void_p)]


class ArtTrainOpts(C.Structure):
    _fields_ = [("steps", C.c_int), ("seed", C.c_uint64), ("reset", C.c_int), ("net", ArtNetOptions),
                ("stream", C.c_void_p)]


class ArtTrainReport(C.Structure):
    _fields_ = [("steps", C.c_int32), ("first_epoch_loss", C.c_double), ("last_epoch_loss", C.c_double),
                ("seconds", C.c_double)]


ART_WARM_NONE, ART_WARM_COARSE, ART_WARM_SURROGATE = 0, 1, 2


class ArtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> C.CDLL:
    """Load libart.so; raises if it is missing (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libart.so not built ({path}); run paper_1410_0763_gb300.build.build()")
        lib = C.CDLL(path)
        P = C.c_void_p
        lib.art_options_default.argtypes = [C.POINTER(ArtOptions)]
        lib.art_create.argtypes = [C.POINTER(ArtGrid), C.c_int, C.c_int, C.POINTER(ArtOptions), C.POINTER(P)]
        lib.art_batch_create.argtypes = [C.POINTER(ArtGrid), C.POINTER(C.c_int), C.c_int, C.c_int,
                                         C.POINTER(ArtOptions), C.POINTER(P)]
        lib.art_autotune.argtypes = [P, C.c_int, C.POINTER(C.c_int), P]
        lib.art_sum_partials.argtypes = [P, C.c_int, C.c_int64, P, P]
        lib.art_set_source_spectrum.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.art_set_source_spectrum.restype = C.c_int
        lib.art_sum_partials.restype = C.c_int
        lib.art_destroy.argtypes = [P]
        lib.art_last_error.argtypes = [P]
        lib.art_last_error.restype = C.c_char_p
        lib.art_get_stats.argtypes = [P, C.POINTER(ArtSweepStats)]
        lib.art_set_fields.argtypes = [P, P, P, C.c_int, P]
        lib.art_set_band.argtypes = [P, C.POINTER(C.c_double)]
        lib.art_set_boundary_intensity.argtypes = [P, C.POINTER(C.c_double)]
        lib.art_plane_source.argtypes = [P, P, C.POINTER(C.c_double), C.c_int, C.c_int, C.POINTER(C.c_double), P, P]
        lib.art_plane_source.restype = C.c_int
        lib.art_set_plane_source.argtypes = [P, C.c_int, C.c_int, C.c_double]
        lib.art_set_plane_source.restype = C.c_int
        lib.art_set_relaxation.argtypes = [P, C.c_double]
        lib.art_set_relaxation.restype = C.c_int
        lib.art_ablation_sweep.argtypes = [P, C.c_int, P, P]
        lib.art_ablation_sweep.restype = C.c_int
        lib.art_evolve_options_default.argtypes = [C.POINTER(ArtEvolveOptions)]
        lib.art_evolve_options_default.restype = C.c_int
        lib.art_thermal_default.argtypes = [C.POINTER(ArtThermal)]
        lib.art_thermal_default.restype = C.c_int
        lib.art_evolve_thermal.argtypes = [P, C.POINTER(ArtChem), C.POINTER(ArtThermal), P, C.POINTER(ArtSource),
                                           C.c_int, C.POINTER(ArtEvolveOptions), P, P, C.POINTER(ArtEvolveReport),
                                           P]
        lib.art_evolve_thermal.restype = C.c_int
        lib.art_evolve_ionization.argtypes = [P, C.POINTER(ArtChem), P, C.POINTER(ArtSource), C.c_int,
                                              C.POINTER(ArtEvolveOptions), P, C.POINTER(ArtEvolveReport), P]
        lib.art_evolve_ionization.restype = C.c_int
        lib.art_sweep.argtypes = [P, P, P, P, C.c_int, P]
        lib.art_sweep_check.argtypes = [P, P]
        lib.art_sweep_check.restype = C.c_int
        lib.art_sweep_set_wait.argtypes = [P, C.c_double, C.c_int]
        lib.art_sweep_set_wait.restype = C.c_int
        lib.art_sweep_stream.argtypes = [P, C.c_int, P, P, P, P, P, P]
        lib.art_sweep_stream.restype = C.c_int
        lib.art_count_segments.argtypes = [C.POINTER(ArtGrid), C.c_int, C.c_double, C.POINTER(C.c_int64)]
        lib.art_band_integral.argtypes = [C.c_double] * 5 + [C.POINTER(C.c_double)]
        lib.art_measure_pipes.argtypes = [C.POINTER(C.c_double)] * 4
        lib.art_point_sources.argtypes = [P, P, C.POINTER(C.c_double), C.POINTER(ArtSource), C.POINTER(C.c_double),
                                          C.c_int, P, P]
        lib.art_iterate_ionization.argtypes = [P, C.POINTER(ArtChem), P, C.POINTER(ArtSource), C.c_int, C.c_double,
                                               C.c_int, C.c_int, P, C.POINTER(C.c_double), C.POINTER(ArtIterReport),
                                               P]
        lib.art_train_opts_default.argtypes = [C.POINTER(ArtTrainOpts)]
        lib.art_train_opts_default.restype = C.c_int
        lib.art_surrogate_train.argtypes = [P, C.POINTER(ArtDataset), C.POINTER(ArtTrainOpts),
                                            C.POINTER(ArtTrainReport)]
        lib.art_surrogate_train.restype = C.c_int
        lib.art_surrogate_network.argtypes = [P, C.POINTER(P)]
        lib.art_surrogate_network.restype = C.c_int
        lib.art_sweep_noalloc.argtypes = [C.POINTER(ArtGrid), C.c_int, P, P, P, P, C.c_char_p, C.c_size_t]
        lib.art_profile_enable.argtypes = [P, C.c_int]
        lib.art_profile_read.argtypes = [P, C.POINTER(ArtProfile), C.c_int]
        lib.art_net_options_default.argtypes = [C.POINTER(ArtNetOptions)]
        lib.art_net_create.argtypes = [C.POINTER(ArtNetOptions), C.POINTER(P)]
        lib.art_net_destroy.argtypes = [P]
        lib.art_net_last_error.argtypes = [P]
        lib.art_net_last_error.restype = C.c_char_p
        lib.art_net_get_params.argtypes = [P, P]
        lib.art_net_set_params.argtypes = [P, P]
        lib.art_net_forward.argtypes = [P, C.c_int, C.c_int, C.c_int, P, P, P]
        lib.art_net_gradients.argtypes = [P, C.c_int, C.c_int, C.c_int, P, P, P, C.POINTER(C.c_double), P, P]
        lib.art_net_train_step.argtypes = [P, C.c_int, C.c_int, C.c_int, P, P, P, C.POINTER(C.c_double), P]
        lib.art_surrogate_sample.argtypes = [P, C.POINTER(ArtChem), P, P, C.c_int, C.c_int, P, P, P, P, P]
        lib.art_surrogate_collect.argtypes = [P, C.POINTER(ArtChem), P, C.POINTER(ArtSource), C.c_int, P, C.c_int,
                                              C.c_int, C.c_int, P, P, P, P]
        lib.art_net_train.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P, C.c_int, C.c_uint64,
                                      C.POINTER(C.c_double), P]
        lib.art_warm_options_default.argtypes = [C.POINTER(ArtWarmOptions)]
        lib.art_net_check.argtypes = [P, P]
        lib.art_net_check.restype = C.c_int
        lib.art_net_set_test_stall.argtypes = [P, C.c_int]
        lib.art_net_set_test_stall.restype = C.c_int
        lib.art_net_set_plane_group.argtypes = [P, C.c_int]
        lib.art_net_set_plane_group.restype = C.c_int
        lib.art_iterate_ionization_warm.argtypes = [P, P, C.POINTER(ArtChem), P, C.POINTER(ArtSource), C.c_int,
                                                    C.c_double, C.c_int, C.POINTER(ArtWarmOptions), P,
                                                    C.POINTER(C.c_double), C.POINTER(ArtWarmReport), P]
        for f in ("art_net_options_default", "art_net_create", "art_net_destroy", "art_net_get_params",
                  "art_net_set_params", "art_net_forward", "art_net_gradients", "art_net_train_step",
                  "art_surrogate_sample", "art_warm_options_default", "art_iterate_ionization_warm",
                  "art_surrogate_collect", "art_net_train",
                  "art_batch_create", "art_autotune"):
            getattr(lib, f).restype = C.c_int
        for f in ("art_point_sources", "art_iterate_ionization", "art_sweep_noalloc", "art_measure_pipes", "art_band_integral", "art_profile_enable", "art_profile_read", "art_options_default", "art_create", "art_count_segments", "art_destroy", "art_get_stats", "art_set_fields",
                  "art_set_band", "art_set_boundary_intensity", "art_sweep"):
            getattr(lib, f).restype = C.c_int
        _lib = lib
        return lib


# ---------------------------------------------------------------------------
# C names
# ---------------------------------------------------------------------------
def art_options_default() -> ArtOptions:
    o = ArtOptions()
    load().art_options_default(C.byref(o))
    return o


def art_create(grid: ArtGrid, n_side: int, nu_bins: int, opt: ArtOptions | None):
    h = C.c_void_p()
    st = load().art_create(C.byref(grid), int(n_side), int(nu_bins), C.byref(opt) if opt else None, C.byref(h))
    if st != ART_OK:
        raise ArtError(st, "art_create failed")
    return h


def art_batch_create(grids, n_side, nu_bins: int, opt: ArtOptions | None):
    n = len(grids)
    ga = (ArtGrid * n)(*grids)
    na = (C.c_int * n)(*[int(x) for x in n_side])
    h = C.c_void_p()
    st = load().art_batch_create(ga, na, n, int(nu_bins), C.byref(opt) if opt else None, C.byref(h))
    if st != ART_OK:
        raise ArtError(st, "art_batch_create failed")
    return h


def art_autotune(ctx, reps: int, stream: int) -> tuple[int, int]:
    best = C.c_int(0)
    st = load().art_autotune(ctx, int(reps), C.byref(best), C.c_void_p(stream))
    return st, best.value


def art_sum_partials(parts, out, stream=None):
    """Fixed-order (part-order, Kahan) sum of device float32 parts [n_parts][n] into out [n]."""
    n_parts = int(parts.shape[0])
    n = int(out.numel())
    pp, pd, _p = _ptr(parts.reshape(-1), np.float32, n_parts * n)
    op, od, _o = _ptr(out, np.float32, n)
    if not (pd and od):
        raise TypeError("art_sum_partials takes device buffers")
    st = load().art_sum_partials(C.c_void_p(pp), n_parts, n, C.c_void_p(op), C.c_void_p(_stream(stream)))
    if st != ART_OK:
        raise ArtError(st, "art_sum_partials failed")
    return out


def art_destroy(ctx) -> int:
    return load().art_destroy(ctx)


def art_last_error(ctx) -> str:
    return load().art_last_error(ctx).decode()


def art_get_stats(ctx) -> ArtSweepStats:
    s = ArtSweepStats()
    _check(ctx, load().art_get_stats(ctx, C.byref(s)))
    return s


def art_set_fields(ctx, kappa_ptr: int, src_ptr: int, on_device: int, stream: int) -> int:
    return load().art_set_fields(ctx, C.c_void_p(kappa_ptr), C.c_void_p(src_ptr), int(on_device),
                                 C.c_void_p(stream))


def art_set_band(ctx, G) -> int:
    arr = (C.c_double * len(G))(*[float(g) for g in G])
    return load().art_set_band(ctx, arr)


def art_set_boundary_intensity(ctx, I_bc) -> int:
    arr = None if I_bc is None else (C.c_double * len(I_bc))(*[float(v) for v in I_bc])
    return load().art_set_boundary_intensity(ctx, arr)


def art_sweep(ctx, J_ptr: int, Jin_ptr: int, gamma_ptr: int, on_device: int, stream: int) -> int:
    return load().art_sweep(ctx, C.c_void_p(J_ptr or None), C.c_void_p(Jin_ptr or None),
                            C.c_void_p(gamma_ptr or None), int(on_device), C.c_void_p(stream))


def art_band_integral(sigma0, h, nu0, nu_lo, nu_hi) -> float:
    out = C.c_double(0.0)
    st = load().art_band_integral(float(sigma0), float(h), float(nu0), float(nu_lo), float(nu_hi), C.byref(out))
    if st != ART_OK:
        raise ArtError(st, "art_band_integral: bad arguments")
    return out.value


def art_sweep_noalloc(shape, n_side: int, kappa_ptr: int, S_ptr: int, Jin_ptr: int, stream: int):
    """The allocation-free FP32 sweep (device pointers).  Returns (status, message)."""
    nz, ny, nx = shape
    buf = C.create_string_buffer(256)
    st = load().art_sweep_noalloc(C.byref(ArtGrid(nx, ny, nz, 1.0)), int(n_side), C.c_void_p(kappa_ptr),
                                  C.c_void_p(S_ptr), C.c_void_p(Jin_ptr), C.c_void_p(stream), buf, 256)
    return st, buf.value.decode()


def art_measure_pipes() -> dict:
    """Results per clock per SM of MUFU ex2, MUFU rcp, scalar FP32 FFMA and FP32 FMAs issued
    as packed FP32x2 instructions (ffma2, two per instruction) on the current GPU."""
    a, b, c, d = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    st = load().art_measure_pipes(C.byref(a), C.byref(b), C.byref(c), C.byref(d))
    if st != ART_OK:
        raise ArtError(st, "art_measure_pipes failed")
    return {"ex2": a.value, "rcp": b.value, "ffma": c.value, "ffma2": d.value}


def art_profile_enable(ctx, enable: bool) -> int:
    return load().art_profile_enable(ctx, int(bool(enable)))


def art_profile_read(ctx, reset: bool = True) -> ArtProfile:
    p = ArtProfile()
    _check(ctx, load().art_profile_read(ctx, C.byref(p), int(bool(reset))))
    return p


def art_count_segments(shape, n_side: int, tie_tol: float = 1e-12) -> int:
    nz, ny, nx = shape
    out = C.c_int64(0)
    st = load().art_count_segments(C.byref(ArtGrid(nx, ny, nz, 1.0)), int(n_side), float(tie_tol), C.byref(out))
    if st != ART_OK:
        raise ArtError(st, "art_count_segments failed")
    return int(out.value)


def _check(ctx, st: int):
    if st != ART_OK:
        raise ArtError(st, art_last_error(ctx) if ctx else "")


# ---------------------------------------------------------------------------
# Buffer marshalling
# ---------------------------------------------------------------------------
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype, n):
    """(pointer, on_device, keepalive) for a torch CUDA tensor or numpy array of n elements."""
    if x is None:
        return 0, None, None
    if _is_torch(x) and not x.is_cuda:
        x = x.numpy()          # CPU (e.g. pinned) tensor: a host buffer
    if _is_torch(x):
        import torch
        want = torch.float64 if dtype == np.float64 else torch.float32
        if x.dtype != want or not x.is_contiguous() or not x.is_cuda:
            raise TypeError(f"expected a contiguous CUDA tensor of {want}")
        if x.numel() != n:
            raise ValueError(f"expected {n} elements, got {x.numel()}")
        return x.data_ptr(), 1, x
    a = np.asarray(x)
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype).name}")
    if a.size != n:
        raise ValueError(f"expected {n} elements, got {a.size}")
    return a.ctypes.data, 0, a


def _stream(stream) -> int:
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover
        pass
    return 0


def _sources(sources):
    arr = (ArtSource * max(1, len(sources)))()
    for i, s in enumerate(sources):
        arr[i] = ArtSource(float(s[0]), float(s[1]), float(s[2]), float(s[3]))
    return arr


class ArtSweep:
    """One sweep context: a grid (nz, ny, nx) with its N_side, or a batch --
    `shape` a list of (nz, ny, nx) and `nside` an int or one per grid -- and
    the number of frequency bins.  Batch arrays are the grids' [z][y][x]
    arrays concatenated inside each bin (see `offsets`)."""

    def __init__(self, shape, nside, nbins: int = 1, precision: str = "fp32", field_form: int = 0,
                 dx_cm: float = 1.0, tile_b: int = 0, tile_c: int = 0, slab: int = 0, dir_split: int = 0,
                 tie_tol: float = 1e-12, variant: int = 0, persistent: int = 0, graph: bool = False,
                 dir_range=None, early_launch: bool = True, averaging: int = 0):
        batch = len(shape) > 0 and not np.isscalar(shape[0])
        shapes = [tuple(int(v) for v in s) for s in (shape if batch else [shape])]
        nsides = [int(v) for v in nside] if not np.isscalar(nside) else [int(nside)] * len(shapes)
        if len(nsides) != len(shapes):
            raise ValueError("one n_side per grid")
        self.batch = batch
        self.shapes = shapes
        self.shape = shapes[0]
        self.nsides = nsides
        self.nside, self.nbins = nsides[0], int(nbins)
        self.dtype = np.float64 if precision == "fp64" else np.float32
        opt = art_options_default()
        opt.precision = ART_FP64 if precision == "fp64" else ART_FP32
        opt.field_form = int(field_form)
        opt.tile_b, opt.tile_c, opt.slab, opt.dir_split = tile_b, tile_c, slab, dir_split
        opt.tie_tol = tie_tol
        opt.variant = int(variant)
        opt.persistent = int(persistent)
        opt.graph = 1 if graph else 0
        opt.early_launch = 1 if early_launch else -1
        opt.averaging = int(averaging)
        if dir_range is not None:
            opt.dir_begin, opt.dir_end = int(dir_range[0]), int(dir_range[1])
        grids = [ArtGrid(nx, ny, nz, dx_cm) for (nz, ny, nx) in shapes]
        if batch:
            self._ctx = art_batch_create(grids, nsides, nbins, opt)
        else:
            self._ctx = art_create(grids[0], nsides[0], nbins, opt)
        sizes = [nz * ny * nx for (nz, ny, nx) in shapes]
        self.offsets = [int(v) for v in np.concatenate([[0], np.cumsum(sizes)[:-1]])]
        self.ncell = int(sum(sizes))

    def autotune(self, reps: int = 3, stream=None) -> int:
        """Time every compiled kernel variant on the current fields; keep the fastest."""
        st, best = art_autotune(self._ctx, reps, _stream(stream))
        _check(self._ctx, st)
        return best

    def close(self):
        if getattr(self, "_ctx", None):
            art_destroy(self._ctx)
            self._ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def stats(self) -> ArtSweepStats:
        return art_get_stats(self._ctx)

    def profile(self, enable: bool = True):
        _check(self._ctx, art_profile_enable(self._ctx, enable))

    def profile_read(self, reset: bool = True) -> ArtProfile:
        return art_profile_read(self._ctx, reset)

    def point_sources(self, kappa, sigma, sources, gamma, Qb=None, stream=None):
        """Point-source rates (App. A) into `gamma` (device); kappa device [bins][z][y][x] FP32."""
        kp, kd, _k = _ptr(kappa, np.float32, self.ncell * self.nbins)
        gp, gd, _g = _ptr(gamma, np.float32, self.ncell)
        if not (kd and gd):
            raise TypeError("point_sources takes device buffers")
        src = _sources(sources)
        sig = (C.c_double * self.nbins)(*[float(x) for x in sigma])
        q = None
        if Qb is not None:
            qa = np.ascontiguousarray(np.asarray(Qb, dtype=np.float64).reshape(len(sources), self.nbins))
            q = qa.ctypes.data_as(C.POINTER(C.c_double))
        _check(self._ctx, load().art_point_sources(self._ctx, C.c_void_p(kp), sig, src, q, len(sources),
                                                    C.c_void_p(gp), C.c_void_p(_stream(stream))))
        return gamma

    def plane_source(self, kappa, sigma, axis, direction, flux, gamma, stream=None):
        """Plane-parallel incident flux (Test-3 setup, Sec. 4.3) into `gamma` (device): flux[b]
        photons/s/cm^2 along +axis (direction 1) or -axis (-1); kappa device [bins][z][y][x] FP32."""
        kp, kd, _k = _ptr(kappa, np.float32, self.ncell * self.nbins)
        gp, gd, _g = _ptr(gamma, np.float32, self.ncell)
        if not (kd and gd):
            raise TypeError("plane_source takes device buffers")
        sig = (C.c_double * self.nbins)(*[float(x) for x in sigma])
        fl = (C.c_double * self.nbins)(*[float(x) for x in flux])
        _check(self._ctx, load().art_plane_source(self._ctx, C.c_void_p(kp), sig, int(axis), int(direction), fl,
                                                   C.c_void_p(gp), C.c_void_p(_stream(stream))))
        return gamma

    def set_plane_source(self, axis=0, direction=1, flux=0.0):
        """Plane-parallel incident flux of the iteration (photons/s/cm^2; 0 removes it)."""
        _check(self._ctx, load().art_set_plane_source(self._ctx, int(axis), int(direction), float(flux)))

    def evolve(self, nH, chem: dict, sources, y, t_end, stream=None, **opts):
        """Time-dependent mode (App. B-D) from t = 0 to t_end (s); nH, y: device FP64 [z][y][x], y updated
        in place.  opts: F, eps_iter, eps_e, eps_hi, dt_fixed, max_steps, max_iter, max_sub.  Returns the
        report; raises ArtError unless t_end was reached with every step converged."""
        npp, nd_, _n = _ptr(nH, np.float64, self.ncell)
        yp, yd, _y = _ptr(y, np.float64, self.ncell)
        if not (nd_ and yd):
            raise TypeError("evolve takes device buffers")
        o = ArtEvolveOptions()
        load().art_evolve_options_default(C.byref(o))
        o.t_end = float(t_end)
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, type(getattr(o, k))(v))
        src = _sources(sources)
        rep = ArtEvolveReport()
        ch = self._chem(chem)
        st = load().art_evolve_ionization(self._ctx, C.byref(ch), C.c_void_p(npp), src, len(sources), C.byref(o),
                                          C.c_void_p(yp), C.byref(rep), C.c_void_p(_stream(stream)))
        _check(self._ctx, st)
        return rep

    def evolve_thermal(self, nH, chem: dict, thermal: dict, sources, y, T, t_end, stream=None, **opts):
        """Time-dependent mode with the energy equation (App. B-D); nH, y, T: device FP64 [z][y][x],
        y and T updated in place.  thermal: on_the_spot, cool_mask, e_bin (list, erg), e_diff (erg), z,
        kB, T_min, T_max (library defaults for the keys left out).  opts as `evolve`.  Returns the
        report; raises ArtError unless t_end was reached with every step converged."""
        npp, nd_, _n = _ptr(nH, np.float64, self.ncell)
        yp, yd, _y = _ptr(y, np.float64, self.ncell)
        tp, td, _t = _ptr(T, np.float64, self.ncell)
        if not (nd_ and yd and td):
            raise TypeError("evolve_thermal takes device buffers")
        o = ArtEvolveOptions()
        load().art_evolve_options_default(C.byref(o))
        o.t_end = float(t_end)
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, type(getattr(o, k))(v))
        th = ArtThermal()
        load().art_thermal_default(C.byref(th))
        for k, v in thermal.items():
            if k == "e_bin":
                e = [float(x) for x in v] + [0.0] * 4
                th.e_bin = (C.c_double * 4)(*e[:4])
            elif hasattr(th, k):
                setattr(th, k, type(getattr(th, k))(v))
            else:
                raise TypeError(f"unknown thermal parameter {k}")
        src = _sources(sources)
        rep = ArtEvolveReport()
        ch = self._chem(chem)
        st = load().art_evolve_thermal(self._ctx, C.byref(ch), C.byref(th), C.c_void_p(npp), src, len(sources),
                                       C.byref(o), C.c_void_p(yp), C.c_void_p(tp), C.byref(rep),
                                       C.c_void_p(_stream(stream)))
        _check(self._ctx, st)
        return rep

    def set_relaxation(self, omega: float):
        """Over-relaxation factor of the balance update in `iterate` / `iterate_warm` (1: plain)."""
        _check(self._ctx, load().art_set_relaxation(self._ctx, float(omega)))

    def iterate(self, nH, chem: dict, sources, y, tol=1e-6, max_iter=200, stream=None, warm_start=ART_WARM_NONE):
        """RT / balance iteration (App. D); nH, y: device FP64 [z][y][x]; y updated in place.
        warm_start: ART_WARM_NONE, ART_WARM_COARSE or ART_WARM_SURROGATE (after surrogate_train).
        Returns (report, residual history); raises ArtError unless converged."""
        npp, nd_, _n = _ptr(nH, np.float64, self.ncell)
        yp, yd, _y = _ptr(y, np.float64, self.ncell)
        if not (nd_ and yd):
            raise TypeError("iterate takes device buffers")
        ch = ArtChem(chem["alphaA"], chem["alphaB"], chem["gcoll"], chem["sigma0"], chem["h"], chem["nu0"],
                     chem["dnu"])
        src = _sources(sources)
        hist = (C.c_double * max_iter)()
        rep = ArtIterReport()
        st = load().art_iterate_ionization(self._ctx, C.byref(ch), C.c_void_p(npp), src, len(sources), float(tol),
                                           int(max_iter), int(warm_start), C.c_void_p(yp), hist, C.byref(rep),
                                           C.c_void_p(_stream(stream)))
        n = max(0, min(rep.iterations, max_iter))
        if st != ART_OK:
            raise ArtError(st, art_last_error(self._ctx))
        return rep, np.array(hist[:n])

    def surrogate_train(self, X, t, w, n_samples, steps=0, seed=1, reset=False, stream=None):
        """art_surrogate_train: train the context's surrogate network on samples of its grid (device
        arrays as surrogate_collect fills them; w may be None).  Returns the ArtTrainReport."""
        nz, ny, nx = self.shape
        V = nx * ny * nz
        xp, xd, _x = _ptr(X, np.float32, 4 * V * n_samples)
        tp, td, _t = _ptr(t, np.float32, V * n_samples)
        wp, wd, _w = _ptr(w, np.float32, V * n_samples)
        if not (xd and td and (w is None or wd)):
            raise TypeError("surrogate_train takes device buffers")
        data = ArtDataset(nx, ny, nz, int(n_samples), C.c_void_p(xp), C.c_void_p(tp), C.c_void_p(wp or None))
        o = ArtTrainOpts()
        load().art_train_opts_default(C.byref(o))
        o.steps, o.seed, o.reset = int(steps), int(seed), 1 if reset else 0
        o.stream = C.c_void_p(_stream(stream))
        rep = ArtTrainReport()
        _check(self._ctx, load().art_surrogate_train(self._ctx, C.byref(data), C.byref(o), C.byref(rep)))
        return rep

    def set_source_spectrum(self, sigma=None, frac=None):
        """Point-source bins of the iteration: cross sections sigma[b] (cm^2), photon fractions frac[b];
        None restores one bin at sigma0."""
        if sigma is None:
            _check(self._ctx, load().art_set_source_spectrum(self._ctx, 0, None, None))
            return
        n = len(sigma)
        sg = (C.c_double * n)(*[float(v) for v in sigma])
        fr = (C.c_double * n)(*[float(v) for v in frac])
        _check(self._ctx, load().art_set_source_spectrum(self._ctx, n, sg, fr))

    def _chem(self, chem: dict) -> ArtChem:
        return ArtChem(chem["alphaA"], chem["alphaB"], chem["gcoll"], chem["sigma0"], chem["h"], chem["nu0"],
                       chem["dnu"])

    def iterate_warm(self, net, nH, chem: dict, sources, y, tol=1e-6, max_iter=200, coarse_factor=4,
                     coarse_nside=4, use_net=True, phase1_max_iter=40, phase1_tol=1e-3, judge_tol=0.3,
                     coarse_solve=True, coarse_tol=1e-4, judge_after=2, stream=None):
        """The iteration of `iterate`, warm-started by the surrogate (coarse sweep + network).
        Returns (warm report, residual history); raises ArtError unless converged."""
        npp, nd_, _n = _ptr(nH, np.float64, self.ncell)
        yp, yd, _y = _ptr(y, np.float64, self.ncell)
        if not (nd_ and yd):
            raise TypeError("iterate_warm takes device buffers")
        w = ArtWarmOptions()
        load().art_warm_options_default(C.byref(w))
        w.coarse_factor, w.coarse_nside, w.use_net = int(coarse_factor), int(coarse_nside), 1 if use_net else 0
        w.phase1_max_iter, w.phase1_tol, w.judge_tol = int(phase1_max_iter), float(phase1_tol), float(judge_tol)
        w.coarse_solve, w.coarse_tol = 1 if coarse_solve else 0, float(coarse_tol)
        w.judge_after = int(judge_after)
        src = _sources(sources)
        hist = (C.c_double * max_iter)()
        rep = ArtWarmReport()
        st = load().art_iterate_ionization_warm(self._ctx, net._net if net is not None else None,
                                                C.byref(self._chem(chem)), C.c_void_p(npp), src, len(sources),
                                                float(tol), int(max_iter), C.byref(w), C.c_void_p(yp), hist,
                                                C.byref(rep), C.c_void_p(_stream(stream)))
        n = max(0, min(rep.total.iterations, max_iter))
        if st != ART_OK:
            raise ArtError(st, art_last_error(self._ctx))
        return rep, np.array(hist[:n])

    def surrogate_sample(self, nH, chem: dict, y, X=None, t=None, jin=None, jc=None, coarse_factor=4,
                         coarse_nside=4, stream=None):
        """Training sample of state y (device FP64): inputs X [4][V], target t, J^in, prolonged J_c
        (device float32 buffers, each optional)."""
        npp, _, _n = _ptr(nH, np.float64, self.ncell)
        yp, _, _y = _ptr(y, np.float64, self.ncell)
        ptrs = []
        keep = []
        for b, m in ((X, 4 * self.ncell), (t, self.ncell), (jin, self.ncell), (jc, self.ncell)):
            p_, d_, k_ = _ptr(b, np.float32, m)
            if b is not None and not d_:
                raise TypeError("surrogate_sample writes device buffers")
            ptrs.append(p_)
            keep.append(k_)
        _check(self._ctx, load().art_surrogate_sample(self._ctx, C.byref(self._chem(chem)), C.c_void_p(npp),
                                                       C.c_void_p(yp), int(coarse_factor), int(coarse_nside),
                                                       *[C.c_void_p(p_) for p_ in ptrs],
                                                       C.c_void_p(_stream(stream))))

    def surrogate_collect(self, nH, chem: dict, sources, y, X, t, n_iter, w=None, coarse_factor=4,
                          coarse_nside=4, stream=None):
        """Run n_iter plain iterations from y (device FP64, updated) recording one training sample per
        iteration into X (device float32 [n_iter][4][V]), t and w ([n_iter][V], w optional)."""
        npp, _, _n = _ptr(nH, np.float64, self.ncell)
        yp, yd, _y = _ptr(y, np.float64, self.ncell)
        xp, xd, _x = _ptr(X, np.float32, n_iter * 4 * self.ncell)
        tp, td, _t = _ptr(t, np.float32, n_iter * self.ncell)
        wp, wd, _w = _ptr(w, np.float32, n_iter * self.ncell)
        if not (yd and xd and td) or (w is not None and not wd):
            raise TypeError("surrogate_collect takes device buffers")
        src = _sources(sources)
        _check(self._ctx, load().art_surrogate_collect(self._ctx, C.byref(self._chem(chem)), C.c_void_p(npp), src,
                                                        len(sources), C.c_void_p(yp), int(n_iter),
                                                        int(coarse_factor), int(coarse_nside), C.c_void_p(xp),
                                                        C.c_void_p(tp), C.c_void_p(wp),
                                                        C.c_void_p(_stream(stream))))

    def set_fields(self, kappa, src, stream=None):
        n = self.ncell * self.nbins
        kp, kd, _k = _ptr(kappa, self.dtype, n)
        sp, sd, _s = _ptr(src, self.dtype, n)
        if kd != sd:
            raise TypeError("kappa and src must both be host or both be device buffers")
        _check(self._ctx, art_set_fields(self._ctx, kp, sp, kd, _stream(stream) if kd else 0))

    def set_band(self, G):
        if len(G) != self.nbins:
            raise ValueError("one band integral per bin")
        _check(self._ctx, art_set_band(self._ctx, G))

    def ablation_sweep(self, mode, J_in, stream=None):
        """Thread-per-ray sweep of Sec. 3.1 into J_in (device FP32): mode 0 float atomics, mode 1 the
        paper's four ray groups (benchmark only)."""
        jp, jd, _j = _ptr(J_in, np.float32, self.ncell)
        if not jd:
            raise TypeError("ablation_sweep takes a device buffer")
        _check(self._ctx, load().art_ablation_sweep(self._ctx, int(mode), C.c_void_p(jp), C.c_void_p(_stream(stream))))
        return J_in

    def set_boundary_intensity(self, I_bc):
        """Intensity of every ray entering the box, one value per bin (None: vacuum)."""
        if I_bc is not None and len(I_bc) != self.nbins:
            raise ValueError("one boundary intensity per bin")
        _check(self._ctx, art_set_boundary_intensity(self._ctx, I_bc))

    def sweep(self, J=None, J_in=None, gamma=None, stream=None):
        n = self.ncell * self.nbins
        bufs = [(J, n), (J_in, n), (gamma, self.ncell)]
        ptrs, kinds, keep = [], set(), []
        for b, m in bufs:
            p, dev, k = _ptr(b, self.dtype, m)
            ptrs.append(p)
            keep.append(k)
            if b is not None:
                kinds.add(dev)
        if len(kinds) > 1:
            raise TypeError("outputs must all be host or all be device buffers")
        on_dev = kinds.pop() if kinds else 1
        _check(self._ctx, art_sweep(self._ctx, ptrs[0], ptrs[1], ptrs[2], on_dev,
                                    _stream(stream) if on_dev else 0))
        return J, J_in, gamma

    def check(self, stream=None) -> int:
        """art_sweep_check: synchronize `stream` and return the status of the sweeps since the last
        check (ART_OK, ART_E_TIMEOUT when a wait of the wavefront sweep ran out)."""
        return int(load().art_sweep_check(self._ctx, C.c_void_p(_stream(stream))))

    def set_wait(self, seconds: float = 2.0, stall_unit: int = -1):
        """art_sweep_set_wait: bound of the wavefront sweep's waits, and the stalled-unit test hook."""
        _check(self._ctx, load().art_sweep_set_wait(self._ctx, float(seconds), int(stall_unit)))

    def wave_counters(self) -> dict:
        """Counters of a library built with ART_WAVE_STATS=1 (a profiling aid): warp cycles at the
        wavefront sweep's step barriers and in its units, lane-0 cycles in the poll loops and the
        number of polls, summed since the last call (all zero in other builds)."""
        lib = load()
        lib.art_wave_counters.argtypes = [C.c_void_p, C.POINTER(C.c_longlong)]
        lib.art_wave_counters.restype = C.c_int
        out = (C.c_longlong * 4)()
        _check(self._ctx, lib.art_wave_counters(self._ctx, out))
        return dict(barrier_cycles=int(out[0]), unit_cycles=int(out[1]), poll_cycles=int(out[2]),
                    polls=int(out[3]))

    def sweep_stream(self, kappas, srcs, J=None, J_in=None, gamma=None, stream=None):
        """Sweeps of len(kappas) field sets held in host memory (art_sweep_stream): the copies of
        the next and the previous set overlap the current sweep.  kappas, srcs: lists of host
        arrays as set_fields takes them; J, J_in, gamma: lists of host output arrays, one per set,
        or None.  Returns (J, J_in, gamma)."""
        n = len(kappas)
        if len(srcs) != n:
            raise ValueError("one source field per kappa field")
        nf = self.ncell * self.nbins
        keep = []

        def table(lst, m):
            if lst is None:
                return None
            if len(lst) != n:
                raise ValueError("one buffer per set")
            ps = []
            for a in lst:
                p, dev, k = _ptr(a, self.dtype, m)
                if dev:
                    raise TypeError("sweep_stream takes host buffers")
                ps.append(p)
                keep.append(k)
            return (C.c_void_p * max(n, 1))(*ps)

        tabs = [table(kappas, nf), table(srcs, nf), table(J, nf), table(J_in, nf), table(gamma, self.ncell)]
        _check(self._ctx, load().art_sweep_stream(self._ctx, n, *tabs, C.c_void_p(_stream(stream))))
        return J, J_in, gamma


class ArtNet:
    """The 3D-convolution surrogate (include/art_net.h): 4 -> 32 -> 32 -> 32 -> 1 channels,
    3x3x3 kernels with per-layer dilations, BF16 tensor-core kernels, FP32 master weights."""

    def __init__(self, dilation=(1, 2, 4, 8), seed: int = 1, lr: float = 1e-3, beta1: float = 0.9,
                 beta2: float = 0.999, adam_eps: float = 1e-8):
        o = ArtNetOptions()
        load().art_net_options_default(C.byref(o))
        for i, d in enumerate(dilation):
            o.dilation[i] = int(d)
        o.seed, o.lr, o.beta1, o.beta2, o.adam_eps = int(seed), float(lr), float(beta1), float(beta2), float(adam_eps)
        h = C.c_void_p()
        st = load().art_net_create(C.byref(o), C.byref(h))
        if st != ART_OK:
            raise ArtError(st, "art_net_create failed")
        self._net = h
        self.dilation = tuple(int(d) for d in dilation)

    def close(self):
        if getattr(self, "_net", None):
            load().art_net_destroy(self._net)
            self._net = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != ART_OK:
            raise ArtError(st, load().art_net_last_error(self._net).decode())

    def check(self, stream=None) -> int:
        """Synchronize and return the bounded-wait status of the network's kernels (ART_OK or ART_E_TIMEOUT)."""
        return load().art_net_check(self._net, C.c_void_p(_stream(stream)))

    def set_plane_group(self, planes: int):
        """Output planes per convolution work item: 1, 2, 4, or 0 for the automatic choice."""
        self._check(load().art_net_set_plane_group(self._net, int(planes)))

    def set_test_stall(self, on: bool):
        self._check(load().art_net_set_test_stall(self._net, 1 if on else 0))

    def get_params(self) -> np.ndarray:
        out = np.empty(ART_NET_PARAMS, dtype=np.float32)
        self._check(load().art_net_get_params(self._net, out.ctypes.data))
        return out

    def set_params(self, p):
        a = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        if a.size != ART_NET_PARAMS:
            raise ValueError(f"expected {ART_NET_PARAMS} parameters")
        self._check(load().art_net_set_params(self._net, a.ctypes.data))

    @staticmethod
    def split_params(flat):
        """params layout -> [(W [27][c_out][c_in], b [c_out])] per layer."""
        out, off = [], 0
        for ci, co in NET_LAYERS:
            W = np.asarray(flat[off:off + 27 * co * ci]).reshape(27, co, ci)
            off += 27 * co * ci
            b = np.asarray(flat[off:off + co])
            off += co
            out.append((W, b))
        return out

    @staticmethod
    def join_params(layers):
        return np.concatenate([np.concatenate([np.ravel(W), np.ravel(b)]) for W, b in layers])

    def _dev(self, x, n, name):
        p_, d_, k_ = _ptr(x, np.float32, n)
        if not d_:
            raise TypeError(f"{name} must be a CUDA float32 tensor")
        return p_

    def forward(self, X, o, shape, stream=None):
        nz, ny, nx = shape
        V = nx * ny * nz
        self._check(load().art_net_forward(self._net, nx, ny, nz, C.c_void_p(self._dev(X, 4 * V, "X")),
                                           C.c_void_p(self._dev(o, V, "o")), C.c_void_p(_stream(stream))))
        return o

    def gradients(self, X, t, shape, w=None, stream=None):
        nz, ny, nx = shape
        V = nx * ny * nz
        loss = C.c_double(0.0)
        g = np.empty(ART_NET_PARAMS, dtype=np.float32)
        wp = self._dev(w, V, "w") if w is not None else 0
        self._check(load().art_net_gradients(self._net, nx, ny, nz, C.c_void_p(self._dev(X, 4 * V, "X")),
                                             C.c_void_p(self._dev(t, V, "t")), C.c_void_p(wp), C.byref(loss),
                                             g.ctypes.data, C.c_void_p(_stream(stream))))
        return loss.value, g

    def train(self, X, t, shape, n_samples, steps, w=None, seed=0, stream=None):
        """`steps` Adam steps over n_samples samples (device X [n][4][V], t and w [n][V]); returns the
        loss per step."""
        nz, ny, nx = shape
        V = nx * ny * nz
        hist = np.zeros(max(steps, 1), dtype=np.float64)
        wp = self._dev(w, n_samples * V, "w") if w is not None else 0
        self._check(load().art_net_train(self._net, nx, ny, nz, int(n_samples),
                                         C.c_void_p(self._dev(X, n_samples * 4 * V, "X")),
                                         C.c_void_p(self._dev(t, n_samples * V, "t")), C.c_void_p(wp), int(steps),
                                         int(seed),
                                         hist.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(_stream(stream))))
        return hist[:steps]

    def train_step(self, X, t, shape, w=None, want_loss=True, stream=None):
        nz, ny, nx = shape
        V = nx * ny * nz
        loss = C.c_double(float("nan"))
        wp = self._dev(w, V, "w") if w is not None else 0
        self._check(load().art_net_train_step(self._net, nx, ny, nz, C.c_void_p(self._dev(X, 4 * V, "X")),
                                              C.c_void_p(self._dev(t, V, "t")), C.c_void_p(wp),
                                              C.byref(loss) if want_loss else None, C.c_void_p(_stream(stream))))
        return loss.value
