"""Pins for the oracle's HEALPix RING geometry (Gorski et al. 2005).

The paper works on a flat grid (Section 3.1) and names the sphere as future
work (Section 4); the pixelisation itself comes from the HEALPix definition.
"""
import os

import numpy as np
import pytest

import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "healpix_nside1.txt")


def test_nside1_base_pixels(orc):
    rows = np.loadtxt(GOLD)
    z, phi = orc.pix_centers(1)
    assert np.allclose(z, rows[:, 1], atol=1e-15)
    assert np.allclose(phi / np.pi, rows[:, 2], atol=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 3, 4, 8, 16, 64, 512])
def test_ring_counts_and_offsets(orc, nside):
    total = 0
    prev_end = 0
    for i in range(1, 4 * nside):
        nr, st, z, omz, opz, p0 = orc.ring_info(nside, i)
        assert st == prev_end
        prev_end = st + nr
        total += nr
        assert abs((1 - z) - omz) < 1e-15 and abs((1 + z) - opz) < 1e-15
        assert -1 < z < 1
        # mirror symmetry of rings i and 4nside - i
        nr2, _, z2, _, _, p2 = orc.ring_info(nside, 4 * nside - i)
        assert nr2 == nr and abs(z + z2) < 1e-15 and abs(p0 - p2) < 1e-15
    assert total == 12 * nside * nside


@pytest.mark.parametrize("nside", [2, 4, 16, 128])
def test_equal_area_ring_centres(orc, nside):
    """HEALPix pixels all have area 4pi/Npix, and every ring centre sits where
    the polar cap above it holds exactly the pixels of the rings to the north
    plus half of its own ring: 2pi(1 - z_i) = Omega (n_north + n_i/2)."""
    npix = 12 * nside * nside
    omega = 4 * np.pi / npix
    north = 0
    for i in range(1, 2 * nside + 1):
        nr, st, z, omz, opz, p0 = orc.ring_info(nside, i)
        assert st == north
        cap = 2 * np.pi * omz
        assert cap == pytest.approx(omega * (north + nr / 2), rel=1e-13, abs=1e-15)
        north += nr


@pytest.mark.parametrize("nside", [4, 8, 32])
def test_azimuths_equally_spaced_with_healpix_shifts(orc, nside):
    """Within a ring the centres are equally spaced by 2pi/n_r; polar-cap rings
    are offset by half a pixel, and equatorial rings alternate between a half
    pixel and no offset, starting with a half pixel at ring nside."""
    for i in range(1, 4 * nside):
        nr, st, z, omz, opz, p0 = orc.ring_info(nside, i)
        half = np.pi / nr
        if i < nside or i > 3 * nside:
            assert p0 == pytest.approx(half, rel=1e-14)
        else:
            assert p0 == pytest.approx(half if (i - nside) % 2 == 0 else 0.0, abs=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 33])
def test_two_independent_geometries_agree(orc, nside):
    z1, p1 = orc.pix_centers(nside)
    z2, p2 = W.pixel_centers(nside)
    assert np.max(np.abs(z1 - z2)) < 1e-14
    assert np.max(np.abs(p1 - p2)) < 1e-13
