"""Pins of the oracle's transfer step and averaging (Sec. 2.2).

* closed forms: kappa = 0 (emissivity inputs) gives the path integral of the
  emissivity; uniform kappa and S give I = S (1 - e^{-kappa l}) after a path
  length l; along an axis-aligned direction cell m (counted from the upwind
  face) sees Ibar_in = S (1 - e^{-kappa m}) phi(kappa);
* energy: per ray, emission escaping its own segment = absorbed incoming +
  escaped at the exit, exactly; per direction, sum_cells kappa A equals the
  absorbed incoming radiation of all rays;
* the emissivity and source-function input forms agree;
* J^in computed cell by cell equals the full sweep; sharded direction ranges
  add up to the full sweep.
"""
import numpy as np
import pytest

from paper_1410_0763_gb300 import workloads as wl


def phi(x):
    x = np.asarray(x, dtype=float)
    out = np.ones_like(x)
    nz = x > 0
    out[nz] = -np.expm1(-x[nz]) / x[nz]
    return out


def test_kappa_zero_gives_emissivity_path_integral(orc):
    rng = np.random.default_rng(3)
    shape = (8, 8, 8)
    kap = np.zeros(shape)
    eps = rng.random(shape)
    nside = 2
    for d in [0, 7, 22, 40]:
        (jlo, jhi, klo, khi), _, _ = orc.lattice(shape, nside, d)
        for (j, k) in [(jlo + 3, klo + 4), (2, 3), (4, 1), (jhi - 3, khi - 2)]:
            cells, ds, iin, iex = orc.trace_ray(kap, eps, nside, d, j, k, field_form=1)
            if len(cells) == 0:
                continue
            cum = np.concatenate([[0.0], np.cumsum(eps.ravel()[cells] * ds)])
            assert np.allclose(iin, cum[:-1], rtol=1e-13, atol=1e-15)
            assert iex == pytest.approx(cum[-1], rel=1e-13)


def test_uniform_medium_closed_form(orc):
    shape = (10, 10, 10)
    kap0, S0 = 0.37, 0.8
    kap = np.full(shape, kap0)
    src = np.full(shape, S0)
    nside = 2
    for d in [1, 9, 25, 33]:
        (jlo, jhi, klo, khi), _, _ = orc.lattice(shape, nside, d)
        for j in range(jlo, jhi + 1, 3):
            for k in range(klo, khi + 1, 4):
                cells, ds, iin, iex = orc.trace_ray(kap, src, nside, d, j, k)
                if len(cells) == 0:
                    continue
                l = np.concatenate([[0.0], np.cumsum(ds)])
                assert np.allclose(iin, S0 * (1 - np.exp(-kap0 * l[:-1])), rtol=1e-12, atol=1e-15)
                assert iex == pytest.approx(S0 * (1 - np.exp(-kap0 * l[-1])), rel=1e-12)


def test_axial_direction_cell_average(orc):
    # N_side = 1 pixel 5 is n = (-1, 0, 0) exactly (phi = pi, z = 0 ring).
    n = 12
    shape = (n, n, n)
    v = orc.healpix_dirs(1)
    d = 5
    assert np.allclose(v[d], [-1, 0, 0], atol=1e-15)
    kap0, S0 = 0.6, 1.3
    A, W = orc.sweep_dir(np.full(shape, kap0), np.full(shape, S0), 1, d)
    ibar = A / W
    # upwind face is x = n (the ray travels towards -x): cell x sits at m = n-1-x
    m = (n - 1 - np.arange(n))[None, None, :]
    expect = S0 * (1 - np.exp(-kap0 * m)) * phi(kap0)
    assert np.allclose(ibar, np.broadcast_to(expect, shape), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("form", [0, 1])
def test_energy_identity_per_ray(orc, form):
    # sum_j S_j (1 - e^{-dtau_j}) = sum_j dtau_j Ibar_in_j + I_exit (Eq. rt and
    # the path average after it, summed along the ray)
    rng = np.random.default_rng(5)
    shape = (9, 8, 7)
    kap = 0.5 * np.exp(rng.standard_normal(shape))
    S = rng.random(shape)
    src = S if form == 0 else kap * S
    nside = 2
    for d in [2, 11, 30, 47]:
        (jlo, jhi, klo, khi), _, _ = orc.lattice(shape, nside, d)
        for j in range(jlo, jhi + 1, 2):
            for k in range(klo, khi + 1, 3):
                cells, ds, iin, iex = orc.trace_ray(kap, src, nside, d, j, k, field_form=form)
                if len(cells) == 0:
                    continue
                dtau = kap.ravel()[cells] * ds
                emitted = np.sum(S.ravel()[cells] * -np.expm1(-dtau))
                absorbed = np.sum(dtau * iin * phi(dtau))
                assert emitted == pytest.approx(absorbed + iex, rel=1e-12, abs=1e-14)


def test_direction_absorption_matches_rays(orc):
    # sum over cells of kappa * A (A = sum ds * Ibar_in) equals the incoming
    # radiation absorbed along every ray of the family
    rng = np.random.default_rng(6)
    shape = (7, 7, 7)
    kap = 0.4 * np.exp(rng.standard_normal(shape))
    S = rng.random(shape)
    nside = 2
    for d in [3, 17, 44]:
        A, _ = orc.sweep_dir(kap, S, nside, d)
        (jlo, jhi, klo, khi), _, _ = orc.lattice(shape, nside, d)
        tot = 0.0
        for k in range(klo, khi + 1):
            for j in range(jlo, jhi + 1):
                cells, ds, iin, _ = orc.trace_ray(kap, S, nside, d, j, k)
                dtau = kap.ravel()[cells] * ds
                tot += np.sum(iin * -np.expm1(-dtau))
        assert np.sum(kap * A) == pytest.approx(tot, rel=1e-12)


def test_emissivity_form_equals_source_form(orc):
    case = wl.lognormal_iid(10, 2, seed=11)
    jin0, j0, nz0 = orc.sweep(case.kappa, case.src, 2, field_form=0)
    jin1, j1, nz1 = orc.sweep(case.kappa, case.kappa * case.src, 2, field_form=1)
    assert nz0 == 0 and nz1 == 0
    assert np.allclose(jin0, jin1, rtol=1e-12)
    assert np.allclose(j0, j1, rtol=1e-12)
    assert np.allclose(j0, jin0 + case.src, rtol=1e-14)


def test_optically_thick_limit(orc):
    # deep inside a uniform medium I_in -> S, so Ibar_in = S phi(kappa ds) and
    # J^in -> 0 like 1/kappa: each of the segments through a cell adds
    # S (1 - e^{-kappa ds})/kappa -> S/kappa to A, and W = 1/|n_a|; J -> S
    shape = (12, 12, 12)
    S0 = 0.7
    out = []
    for kap0 in [25.0, 50.0, 100.0]:
        jin, j, _ = orc.sweep(np.full(shape, kap0), np.full(shape, S0), 2)
        core = jin[3:-3, 3:-3, 3:-3]
        out.append(core.mean())
        assert np.all(j[3:-3, 3:-3, 3:-3] > S0)
    assert out[0] > out[1] > out[2]
    assert out[1] / out[0] == pytest.approx(0.5, rel=0.08)
    assert out[2] / out[1] == pytest.approx(0.5, rel=0.05)
    # kappa J^in / S tends to the mean over directions of |n_x|+|n_y|+|n_z|
    # (segments per cell per direction times |n_a|), from below
    l1 = np.abs(orc.healpix_dirs(2)).sum(axis=1).mean()
    assert 0.85 * l1 < 100.0 * out[2] / S0 < l1


def test_cell_by_cell_equals_full_sweep(orc):
    case = wl.grf(16, 2, seed=21)
    jin, _, _ = orc.sweep(case.kappa, case.src, 2)
    rng = np.random.default_rng(1)
    cells = rng.choice(jin.size, 25, replace=False)
    one = orc.jin_cells(case.kappa, case.src, 2, cells)
    assert np.allclose(one, jin.ravel()[cells], rtol=1e-13)


def test_sharded_ranges_add_up(orc):
    case = wl.grf(12, 2, seed=8)
    full, nz = orc.sweep_range(case.kappa, case.src, 2, 0, 48)
    a, _ = orc.sweep_range(case.kappa, case.src, 2, 0, 20)
    b, _ = orc.sweep_range(case.kappa, case.src, 2, 20, 48)
    assert nz == 0
    assert np.allclose(a + b, full, rtol=1e-13)


def test_thread_count_does_not_change_result(orc):
    case = wl.grf(12, 2, seed=9)
    j1, _, _ = orc.sweep(case.kappa, case.src, 2, nthreads=1)
    j4, _, _ = orc.sweep(case.kappa, case.src, 2, nthreads=4)
    assert np.array_equal(j1, j4)
