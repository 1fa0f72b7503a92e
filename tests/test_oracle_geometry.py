"""Pins of the oracle's ray geometry (Sec. 2.2 Fig. parallel_ray, Sec. 3.1).

The ray family of a direction is the unit lattice of lines, on planes normal
to the dominant axis a, offset to cell centres: X_b = j + 1/2 + q_b u,
X_c = k + 1/2 + q_c u (u measured along a from the upwind face).  The checks:

* brute force: every (ray, cell) pair is intersected by the slab test and the
  ordered segment list is compared with the oracle's incremental marcher;
* every cell's summed chord length W equals 1/|n_a| -- each cross-section of a
  cell normal to a contains exactly one lattice point, so exactly 1/|n_a| of
  ray length passes through it (the lattice is aligned with the mesh);
* the four parity groups (j mod 2, k mod 2) of Sec. 3.1 visit no cell twice;
* sum over cells of W = sum over rays of chord length.
"""
import numpy as np
import pytest

SHAPE = (6, 7, 8)  # (nz, ny, nx): non-cubic on purpose


def frame_from_vector(n, tie_tol=1e-12):
    m = np.abs(n).max()
    a = int(np.nonzero(np.abs(n) >= m - tie_tol * m)[0][0])
    b, c = [i for i in range(3) if i != a]
    sa = 1 if n[a] >= 0 else -1
    na = abs(n[a])
    qb = float(np.clip(n[b] / na, -1, 1))
    qc = float(np.clip(n[c] / na, -1, 1))
    return a, b, c, sa, na, qb, qc


def brute_segments(shape, n, j, k):
    """All (cell, ds) with ds > 1e-12 for lattice ray (j, k), sorted along the ray."""
    nz, ny, nx = shape
    dims = (nx, ny, nz)
    a, b, c, sa, na, qb, qc = frame_from_vector(n)
    Na, Nb, Nc = dims[a], dims[b], dims[c]
    ia = np.arange(Na)[:, None, None]
    ib = np.arange(Nb)[None, :, None]
    ic = np.arange(Nc)[None, None, :]
    if sa > 0:
        lo_a, hi_a = ia + 0.0, ia + 1.0
    else:
        lo_a, hi_a = Na - ia - 1.0, Na - ia + 0.0

    def interval(p, x0, q):
        if q == 0.0:
            inside = (x0 > p) & (x0 < p + 1)
            return np.where(inside, -np.inf, np.inf), np.where(inside, np.inf, -np.inf)
        u1 = (p - x0) / q
        u2 = (p + 1 - x0) / q
        return np.minimum(u1, u2), np.maximum(u1, u2)

    lo_b, hi_b = interval(ib + 0.0, j + 0.5, qb)
    lo_c, hi_c = interval(ic + 0.0, k + 0.5, qc)
    lo = np.maximum(np.maximum(lo_a, lo_b), lo_c)
    hi = np.minimum(np.minimum(hi_a, hi_b), hi_c)
    du = hi - lo
    sel = np.nonzero(du > 1e-12)
    out = []
    for t in range(len(sel[0])):
        x = [0, 0, 0]
        x[a], x[b], x[c] = sel[0][t], sel[1][t], sel[2][t]
        cell = (x[2] * ny + x[1]) * nx + x[0]
        out.append((lo[sel][t], cell, du[sel][t] / na))
    out.sort()
    return [(cell, ds) for _, cell, ds in out]


@pytest.mark.parametrize("nside", [2, 3])
def test_marcher_matches_brute_force(orc, nside):
    v = orc.healpix_dirs(nside)
    kap = np.ones(SHAPE)
    src = np.zeros(SHAPE)
    rng = np.random.default_rng(0)
    dirs = range(v.shape[0]) if nside == 2 else rng.choice(v.shape[0], 30, replace=False)
    nrays = 0
    for d in dirs:
        (jlo, jhi, klo, khi), _, _ = orc.lattice(SHAPE, nside, d)
        for k in range(klo - 1, khi + 2):
            for j in range(jlo - 1, jhi + 2):
                ref = brute_segments(SHAPE, v[d], j, k)
                cells, ds, _, _ = orc.trace_ray(kap, src, nside, d, j, k)
                # near-ties: the brute force may keep slivers the marcher merges
                ref = [(c, s) for c, s in ref if s > 1e-10]
                got = [(c, s) for c, s in zip(cells, ds) if s > 1e-10]
                assert [c for c, _ in got] == [c for c, _ in ref], (d, j, k)
                assert np.allclose([s for _, s in got], [s for _, s in ref], atol=1e-11)
                nrays += len(ref) > 0
    assert nrays > 100


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_chord_per_cell_is_one_over_na(orc, nside):
    v = orc.healpix_dirs(nside)
    kap = np.ones(SHAPE)
    src = np.zeros(SHAPE)
    for d in range(v.shape[0]):
        _, W = orc.sweep_dir(kap, src, nside, d)
        na = np.abs(v[d]).max()
        assert np.allclose(W, 1.0 / na, rtol=1e-11), d


def test_parity_groups_visit_each_cell_once(orc):
    nside = 2
    v = orc.healpix_dirs(nside)
    kap = np.ones(SHAPE)
    src = np.zeros(SHAPE)
    ncell = int(np.prod(SHAPE))
    for d in range(v.shape[0]):
        (jlo, jhi, klo, khi), _, _ = orc.lattice(SHAPE, nside, d)
        visits = np.zeros((4, ncell), dtype=int)
        total = 0.0
        for k in range(klo, khi + 1):
            for j in range(jlo, jhi + 1):
                cells, ds, _, _ = orc.trace_ray(kap, src, nside, d, j, k)
                g = (j % 2) + 2 * (k % 2)
                np.add.at(visits[g], cells, 1)
                total += ds.sum()
        assert visits.max() <= 1, d
        # sum over cells of W equals the summed chord length of all rays
        _, W = orc.sweep_dir(kap, src, nside, d)
        assert W.sum() == pytest.approx(total, rel=1e-12)
        # each cell is crossed by at most four rays of this direction
        assert visits.sum(axis=0).max() <= 4


def test_segment_count_estimate(orc):
    # rays cross (|n_a| + |n_b| + |n_c|)/|n_a| cells per unit length along a:
    # total segments = that factor times N^3, up to boundary terms
    n = 16
    shape = (n, n, n)
    nside = 2
    v = orc.healpix_dirs(nside)
    kap = np.ones(shape)
    src = np.zeros(shape)
    for d in [0, 5, 13, 20]:
        (jlo, jhi, klo, khi), _, _ = orc.lattice(shape, nside, d)
        nseg = 0
        for k in range(klo, khi + 1):
            for j in range(jlo, jhi + 1):
                cells, _, _, _ = orc.trace_ray(kap, src, nside, d, j, k)
                nseg += len(cells)
        est = np.abs(v[d]).sum() / np.abs(v[d]).max() * n ** 3
        assert abs(nseg - est) / est < 4.0 / n
