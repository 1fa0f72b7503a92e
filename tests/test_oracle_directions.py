"""Pins of the oracle's HEALPix direction set (Sec. 2.3; Gorski et al. 2005).

The checks come from what defines HEALPix, not from its pixel formulas:
equal-area pixels (the solid angle above each ring centre equals the pixels
above it plus half the ring), iso-latitude rings with equally spaced pixels,
the ring populations, the mirror and quarter-turn symmetries, the RING order,
and the N_side = 1 set written out from the base-resolution geometry.
"""
import math

import numpy as np
import pytest


def _rings(v, tol=1e-12):
    """Group directions by z (rings), in RING order."""
    z = v[:, 2]
    rings = []
    start = 0
    for i in range(1, len(z) + 1):
        if i == len(z) or abs(z[i] - z[start]) > tol:
            rings.append((start, i))
            start = i
    return rings


@pytest.mark.parametrize("nside", [1, 2, 3, 4, 8])
def test_count_norm_and_antipodal_sum(orc, nside):
    v = orc.healpix_dirs(nside)
    assert v.shape == (12 * nside * nside, 3)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-14)
    assert np.abs(v.sum(axis=0)).max() < 1e-12


def test_nside1_base_pixels(orc):
    # N_side = 1: three rings of four pixels at z = 2/3, 0, -2/3; the polar
    # rings sit at phi = pi/4 + k pi/2, the equatorial one at phi = k pi/2.
    v = orc.healpix_dirs(1)
    z = v[:, 2]
    assert np.allclose(z[:4], 2 / 3) and np.allclose(z[4:8], 0) and np.allclose(z[8:], -2 / 3)
    phi = np.mod(np.arctan2(v[:, 1], v[:, 0]), 2 * np.pi)
    assert np.allclose(np.sort(phi[:4]), [np.pi / 4, 3 * np.pi / 4, 5 * np.pi / 4, 7 * np.pi / 4])
    assert np.allclose(np.sort(np.mod(phi[4:8] + 1e-9, 2 * np.pi)) - 1e-9,
                       [0, np.pi / 2, np.pi, 3 * np.pi / 2], atol=1e-12)
    assert np.allclose(np.sort(phi[8:]), [np.pi / 4, 3 * np.pi / 4, 5 * np.pi / 4, 7 * np.pi / 4])


@pytest.mark.parametrize("nside", [1, 2, 3, 4, 8, 16])
def test_equal_area_ring_latitudes(orc, nside):
    v = orc.healpix_dirs(nside)
    npix = v.shape[0]
    rings = _rings(v)
    assert len(rings) == 4 * nside - 1
    above = 0
    for (s, e) in rings:
        m = e - s
        z = v[s, 2]
        # solid angle above the ring centre, in pixel units of 4 pi / N_pix
        cap = 2 * math.pi * (1 - z) / (4 * math.pi / npix)
        assert cap == pytest.approx(above + m / 2, abs=1e-9)
        above += m
    assert above == npix


@pytest.mark.parametrize("nside", [1, 2, 3, 4, 8])
def test_ring_populations_spacing_and_order(orc, nside):
    v = orc.healpix_dirs(nside)
    rings = _rings(v)
    for r, (s, e) in enumerate(rings):
        i = r + 1
        expect = 4 * min(i, nside, 4 * nside - i)
        assert e - s == expect
        phi = np.mod(np.arctan2(v[s:e, 1], v[s:e, 0]), 2 * np.pi)
        # RING order: increasing phi within the ring, starting in [0, 2pi/m]
        unwrapped = np.unwrap(phi)
        d = np.diff(unwrapped)
        assert np.allclose(d, 2 * np.pi / expect, atol=1e-12)
        off = np.mod(unwrapped[0], 2 * np.pi / expect) / (2 * np.pi / expect)
        # polar-cap rings are shifted by half a pixel; belt rings alternate
        if i < nside or i > 3 * nside:
            assert off == pytest.approx(0.5, abs=1e-9)
        else:
            assert min(abs(off - 0.5), abs(off), abs(off - 1)) < 1e-9
        if nside <= i <= 3 * nside:
            shifted = abs(off - 0.5) < 1e-9
            assert shifted == ((i - nside) % 2 == 0)
    # rings run from north to south
    zs = [v[s, 2] for s, _ in rings]
    assert all(a > b for a, b in zip(zs, zs[1:]))


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_symmetries(orc, nside):
    v = orc.healpix_dirs(nside)

    def same_set(a, b):
        a = a[np.lexsort(np.round(a, 9).T)]
        b = b[np.lexsort(np.round(b, 9).T)]
        return np.allclose(a, b, atol=1e-12)

    mirror = v * np.array([1, 1, -1])
    assert same_set(v, mirror)
    quarter = np.stack([-v[:, 1], v[:, 0], v[:, 2]], axis=1)
    assert same_set(v, quarter)
