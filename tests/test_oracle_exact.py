"""Pins of the oracle's exact path averaging (ART_AVG_EXACT), the alternative
to the paper's cell average that the paper's double count of local emission
calls for (Eq. path_averaged_intensity; the exact path average of I over a
segment is S + (I_in - S) phi).

* Energy per direction: with the exact average, absorbed = emitted - escaped
  exactly.  Source-function inputs deposit (I_in - S) phi ds, so
  sum_cells kappa A = -sum_rays I_exit; emissivity inputs deposit the whole
  <I> ds, so sum_cells kappa A = sum_cells eps W - sum_rays I_exit.
* A thick uniform medium is in equilibrium inside: J = S exactly (up to the
  e^-tau of the distance to the boundary); the paper's average is not.
* kappa = 0 with emissivity inputs along an axis: the cell average of the
  linearly growing intensity is eps (m + 1/2) for cell m (the paper's:
  eps m).
"""
import numpy as np
import pytest


def _exits(orc, kap, src, nside, d, form):
    (jlo, jhi, klo, khi), _, _ = orc.lattice(kap.shape, nside, d)
    total = 0.0
    for k in range(klo, khi + 1):
        for j in range(jlo, jhi + 1):
            cells, ds, iin, iex = orc.trace_ray(kap, src, nside, d, j, k, field_form=form)
            total += iex
    return total


@pytest.mark.parametrize("form", [0, 1])
def test_exact_average_conserves_energy_per_direction(orc, form):
    rng = np.random.default_rng(61)
    shape = (5, 6, 7)
    kap = 0.6 * np.exp(rng.standard_normal(shape))
    src = rng.random(shape)
    for d in range(12 * 4):
        A, W = orc.sweep_dir(kap, src, 2, d, field_form=form, averaging=1)
        lhs = np.sum(kap * A)
        esc = _exits(orc, kap, src, 2, d, form)
        if form == 0:
            assert lhs == pytest.approx(-esc, rel=1e-11, abs=1e-12)
        else:
            assert lhs == pytest.approx(np.sum(src * W) - esc, rel=1e-11, abs=1e-12)


def test_thick_uniform_medium_is_in_equilibrium_inside(orc):
    shape = (14, 14, 14)
    kap = np.full(shape, 5.0)
    S = np.full(shape, 0.7)
    _, j_exact, _ = orc.sweep(kap, S, 2, averaging=1)
    _, j_paper, _ = orc.sweep(kap, S, 2)
    inner = (slice(5, 9),) * 3          # at least 5 cells (optical depth 25) from every face
    assert np.allclose(j_exact[inner], 0.7, rtol=1e-9, atol=0)
    assert np.all(j_paper[inner] > 0.7 * 1.1)   # the paper's form also counts the local emission as incoming


def test_empty_medium_emission_average_along_an_axis(orc):
    # N_side 1 has four exactly axial directions; in an emissivity-only medium
    # (kappa = 0) the intensity entering cell m of a ray along +x is eps m
    shape = (3, 3, 9)
    z = np.zeros(shape)
    eps = np.full(shape, 0.25)
    dirs = orc.healpix_dirs(1)
    d = int(np.argmax(dirs[:, 0]))
    assert dirs[d, 0] == pytest.approx(1.0, abs=1e-15)
    A_x, W_x = orc.sweep_dir(z, eps, 1, d, field_form=1, averaging=1)
    A_p, W_p = orc.sweep_dir(z, eps, 1, d, field_form=1, averaging=0)
    m = np.arange(shape[2])
    assert np.allclose((A_x / W_x)[1, 1], 0.25 * (m + 0.5), rtol=1e-14)
    assert np.allclose((A_p / W_p)[1, 1], 0.25 * m, rtol=1e-14, atol=1e-15)


def test_exact_and_paper_outputs_relate_through_the_source(orc):
    # source-function inputs: J - S is the cell average of (I_in - S) phi in
    # exact mode and of I_in phi in paper mode; both J^in outputs equal J - S
    rng = np.random.default_rng(62)
    shape = (6, 7, 5)
    kap = 0.5 * np.exp(rng.standard_normal(shape))
    S = rng.random(shape)
    jin_x, j_x, _ = orc.sweep(kap, S, 2, averaging=1)
    jin_p, j_p, _ = orc.sweep(kap, S, 2)
    assert np.allclose(j_x - S, jin_x, rtol=1e-13, atol=1e-15)
    assert np.allclose(j_p - S, jin_p, rtol=1e-13, atol=1e-15)
    # emissivity inputs with kappa > 0 everywhere: the same J as source-function inputs
    jin_e, j_e, _ = orc.sweep(kap, S * kap, 2, field_form=1, averaging=1)
    assert np.allclose(j_e, j_x, rtol=1e-12)
    assert np.allclose(jin_e, jin_x, rtol=1e-9, atol=1e-12)
