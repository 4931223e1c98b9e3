"""Pins for the oracle's HEALPix RING grid (the pixelisation of the paper's
Sect. 3 maps)."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "healpix_rings_nside1_2.txt")


def test_rings_match_hand_written_table(oracle):
    rows = np.loadtxt(GOLDEN)
    for nside in (1, 2):
        g = oracle.healpix_rings(nside)
        sel = rows[rows[:, 0] == nside]
        assert len(sel) == 4 * nside - 1
        for _, ring, zn, zd, n, p in sel:
            r = int(ring) - 1
            assert g["z"][r] == pytest.approx(zn / zd, abs=1e-15)
            assert g["nr"][r] == int(n)
            assert g["phi0"][r] == pytest.approx(p * np.pi, abs=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 64, 512])
def test_pixel_count_and_offsets(oracle, nside):
    g = oracle.healpix_rings(nside)
    assert g["nr"].sum() == 12 * nside * nside
    assert np.all(np.diff(g["offset"]) == g["nr"][:-1])
    assert np.all(np.diff(g["z"]) < 0)  # north to south
    np.testing.assert_allclose(g["sintheta"] ** 2 + g["z"] ** 2, 1.0, atol=1e-14)
    # north/south mirror symmetry of the grid
    np.testing.assert_allclose(g["z"], -g["z"][::-1], atol=1e-15)
    np.testing.assert_array_equal(g["nr"], g["nr"][::-1])


@pytest.mark.parametrize("nside", [8, 32, 128])
def test_equal_area_moments(oracle, nside):
    """Equal-area pixels integrate low-order functions of z: mean z^2 over all
    pixel centres tends to the sphere average 1/3 (error O(1/nside^2)), and
    the cap boundary ring z = 2/3 splits off the 1/6 of the sphere that
    holds 2 nside (nside - 1) + 2 nside pixels' worth of area."""
    g = oracle.healpix_rings(nside)
    z = np.repeat(g["z"], g["nr"])
    assert abs(np.mean(z ** 2) - 1.0 / 3.0) < 0.2 / nside ** 2
    assert abs(np.mean(z)) < 1e-14
    # area north of z = 2/3 is 1/6 of the sphere: cap rings hold
    # 2 nside (nside-1) pixels and the boundary ring (z = 2/3 exactly) half of 4 nside
    ncap = int(np.sum(g["nr"][: nside - 1]))
    assert ncap == 2 * nside * (nside - 1)
    assert (ncap + 2 * nside) / (12 * nside * nside) == pytest.approx(1.0 / 6.0)
    assert g["z"][nside - 1] == pytest.approx(2.0 / 3.0, abs=1e-15)


def test_pixel_angles_ring_spacing(oracle):
    nside = 8
    th, ph = oracle.pixel_angles(nside)
    g = oracle.healpix_rings(nside)
    for r in range(4 * nside - 1):
        o, n = g["offset"][r], g["nr"][r]
        np.testing.assert_allclose(np.diff(ph[o:o + n]), 2 * np.pi / n, atol=1e-14)
        assert np.all(th[o:o + n] == th[o])


def test_generator_ring_layout_agrees(oracle):
    """The input generator keeps its own copy of the grid (no shared code);
    both must agree."""
    import wf_inputs as gen

    for nside in (1, 2, 16, 256):
        z, p0, nr = gen.ring_layout(nside)
        g = oracle.healpix_rings(nside)
        np.testing.assert_allclose(z, g["z"], atol=1e-15)
        np.testing.assert_allclose(p0, g["phi0"], atol=1e-15)
        np.testing.assert_array_equal(nr, g["nr"])
