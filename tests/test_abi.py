"""The C-ABI library loads and exports every entry point include/*.h declares;
host-only entry points work without a GPU; the library's per-slab segment
tables agree with the oracle's independent marcher on the exact segment
count."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_1410_0763_gb300 import art, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return art.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(art_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 9
    raw = ctypes.CDLL(art.library_path())
    for n in names:
        assert hasattr(raw, n), n


def test_options_default(lib):
    o = art.art_options_default()
    assert o.precision == art.ART_FP32 and o.field_form == art.ART_FIELDS_S
    assert o.tie_tol == 1e-12 and o.tile_b == 0 and o.slab == 0


@pytest.mark.parametrize("dims,nside,bins", [((0, 4, 4), 1, 1), ((4, 4, 4), 0, 1), ((4, 4, 4), 1, 0),
                                             ((4, -1, 4), 2, 1)])
def test_create_rejects_bad_arguments_without_touching_the_gpu(lib, dims, nside, bins):
    nz, ny, nx = dims
    h = ctypes.c_void_p()
    st = lib.art_create(ctypes.byref(art.ArtGrid(nx, ny, nz, 1.0)), nside, bins, None, ctypes.byref(h))
    assert st == art.ART_E_INVALID and not h.value


@pytest.mark.parametrize("dims,nsides,n", [([(4, 4, 4)], [1], 0), ([(4, 4, 4), (0, 4, 4)], [1, 1], 2),
                                             ([(4, 4, 4), (5, 5, 5)], [1, 0], 2),
                                             ([(4, 4, 4)], [1], 5000)])
def test_batch_create_rejects_bad_arguments_without_touching_the_gpu(lib, dims, nsides, n):
    grids = (art.ArtGrid * max(1, len(dims)))(*[art.ArtGrid(nx, ny, nz, 1.0) for (nz, ny, nx) in dims])
    ns = (ctypes.c_int * len(nsides))(*nsides)
    h = ctypes.c_void_p()
    st = lib.art_batch_create(grids, ns, n, 1, None, ctypes.byref(h))
    assert st == art.ART_E_INVALID and not h.value
    assert lib.art_batch_create(None, ns, 1, 1, None, ctypes.byref(h)) == art.ART_E_INVALID
    assert lib.art_autotune(None, 1, None, None) == art.ART_E_INVALID


@pytest.mark.parametrize("rng", [(3, 3), (5, 2), (-1, 4), (0, 13)])
def test_bad_direction_shards_are_rejected_without_touching_the_gpu(lib, rng):
    o = art.art_options_default()
    o.dir_begin, o.dir_end = rng
    h = ctypes.c_void_p()
    st = lib.art_create(ctypes.byref(art.ArtGrid(4, 4, 4, 1.0)), 1, 1, ctypes.byref(o), ctypes.byref(h))
    assert st == art.ART_E_INVALID and not h.value


def test_null_context_calls_fail_cleanly(lib):
    assert lib.art_sweep(None, None, None, None, 1, None) == art.ART_E_INVALID
    assert lib.art_set_fields(None, None, None, 0, None) == art.ART_E_INVALID
    assert lib.art_set_boundary_intensity(None, None) == art.ART_E_INVALID
    assert lib.art_plane_source(None, None, None, 0, 1, None, None, None) == art.ART_E_INVALID
    assert lib.art_set_plane_source(None, 0, 1, 1.0) == art.ART_E_INVALID
    assert lib.art_set_relaxation(None, 1.3) == art.ART_E_INVALID
    assert lib.art_evolve_ionization(None, None, None, None, 0, None, None, None, None) == art.ART_E_INVALID
    assert lib.art_evolve_options_default(None) == art.ART_E_INVALID
    assert lib.art_ablation_sweep(None, 0, None, None) == art.ART_E_INVALID
    o = art.ArtEvolveOptions()
    assert lib.art_evolve_options_default(ctypes.byref(o)) == art.ART_OK
    assert (o.F, o.eps_iter, o.eps_e, o.eps_hi, o.dt_fixed) == (10.0, 1e-3, 0.2, 0.002, 0.0)
    w = art.ArtWarmOptions()
    assert lib.art_warm_options_default(ctypes.byref(w)) == art.ART_OK and w.judge_after == 2
    assert lib.art_evolve_thermal(None, None, None, None, None, 0, None, None, None, None, None) == \
        art.ART_E_INVALID
    assert lib.art_thermal_default(None) == art.ART_E_INVALID
    assert lib.art_sweep_stream(None, 1, None, None, None, None, None, None) == art.ART_E_INVALID
    assert lib.art_sweep_check(None, None) == art.ART_E_INVALID
    assert lib.art_wave_counters(None, None) == art.ART_E_INVALID
    assert lib.art_iterate_ionization(None, None, None, None, 0, 1e-6, 10, art.ART_WARM_SURROGATE, None, None,
                                      None, None) == art.ART_E_INVALID
    assert lib.art_surrogate_train(None, None, None, None) == art.ART_E_INVALID
    assert lib.art_surrogate_network(None, None) == art.ART_E_INVALID
    assert lib.art_train_opts_default(None) == art.ART_E_INVALID
    to = art.ArtTrainOpts()
    assert lib.art_train_opts_default(ctypes.byref(to)) == art.ART_OK
    assert (to.steps, to.seed, to.reset, list(to.net.dilation)) == (0, 1, 0, [1, 2, 4, 8])
    assert lib.art_sweep_set_wait(None, 1.0, -1) == art.ART_E_INVALID
    th = art.ArtThermal()
    assert lib.art_thermal_default(ctypes.byref(th)) == art.ART_OK
    assert (th.on_the_spot, th.cool_mask, list(th.e_bin), th.e_diff, th.z, th.kB, th.T_min, th.T_max) == \
        (0, 31, [0.0] * 4, 0.0, 0.0, 1.380649e-16, 10.0, 1e9)
    assert lib.art_destroy(None) == art.ART_OK
    assert lib.art_last_error(None) == b"null context"


@pytest.mark.parametrize("shape,nside", [((8, 8, 8), 1), ((6, 7, 8), 2), ((9, 12, 10), 3), ((16, 16, 16), 4)])
def test_segment_count_matches_oracle_marcher(lib, orc, shape, nside):
    kap = np.ones(shape)
    src = np.zeros(shape)
    total = 0
    for d in range(12 * nside * nside):
        (jlo, jhi, klo, khi), _, _ = orc.lattice(shape, nside, d)
        for k in range(klo, khi + 1):
            for j in range(jlo, jhi + 1):
                cells, _, _, _ = orc.trace_ray(kap, src, nside, d, j, k)
                total += len(cells)
    assert art.art_count_segments(shape, nside) == total
