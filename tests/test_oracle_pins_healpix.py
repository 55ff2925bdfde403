"""Pins of the oracle's HEALPix pixel assignment (Gorski et al. 2005, used for the maps of Sect.
2.5): pixel centres map to themselves in both schemes, RING and NESTED name the same pixel, points
near a centre stay in its pixel, and uniform directions fill the equal-area pixels evenly."""
import numpy as np
import pytest

import oracle
from paper_2111_08744_gb300 import inputs as I


@pytest.mark.parametrize("nside", [1, 2, 8, 64])
def test_centres_map_to_themselves(nside):
    for nest in (True, False):
        d = I.healpix_directions(nside, nest=nest)
        np.testing.assert_array_equal(oracle.healpix_pixels(d, nside, nest), np.arange(12 * nside * nside))


def _unit(rng, n):
    v = rng.normal(size=(3, n))
    return v / np.linalg.norm(v, axis=0)


@pytest.mark.parametrize("nside", [4, 32])
def test_ring_and_nested_name_the_same_pixel(nside):
    v = _unit(np.random.Generator(np.random.PCG64(11)), 20000)
    pn = oracle.healpix_pixels(v, nside, True)
    pr = oracle.healpix_pixels(v, nside, False)
    tn, fn = I.pix2ang_nest(nside, pn)
    tr, fr = I.pix2ang_ring(nside, pr)
    np.testing.assert_allclose(tn, tr, atol=1e-12)
    np.testing.assert_allclose(np.cos(fn), np.cos(fr), atol=1e-12)
    np.testing.assert_allclose(np.sin(fn), np.sin(fr), atol=1e-12)


def test_points_near_a_centre_stay_in_its_pixel():
    nside = 16
    rng = np.random.Generator(np.random.PCG64(5))
    c = I.healpix_directions(nside)
    v = c + 0.05 * np.sqrt(4 * np.pi / c.shape[1]) * _unit(rng, c.shape[1])   # 5 % of a pixel size
    for nest in (True, False):
        own = oracle.healpix_pixels(c, nside, nest)
        np.testing.assert_array_equal(oracle.healpix_pixels(v, nside, nest), own)


def test_uniform_directions_fill_equal_area_pixels():
    nside, n = 8, 2_000_000
    v = _unit(np.random.Generator(np.random.PCG64(3)), n)
    for nest in (True, False):
        counts = np.bincount(oracle.healpix_pixels(v, nside, nest), minlength=12 * nside * nside)
        mean = n / counts.size
        chi2 = ((counts - mean) ** 2 / mean).sum()
        # chi-square with 767 degrees of freedom: mean 767, sd ~39
        assert abs(chi2 - (counts.size - 1)) < 6 * np.sqrt(2 * (counts.size - 1)), chi2
