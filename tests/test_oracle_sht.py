"""Pins for the oracle's Legendre functions and spherical-harmonic transforms
(the basis change of Sect. 2.1 on the HEALPix grid of Sect. 3)."""
import math

import numpy as np
import pytest
from scipy import special as sp
from numpy.polynomial.legendre import leggauss


def _closed_form(l, m, th):
    """Textbook Y_lm(theta, 0), l <= 2, Condon-Shortley phase."""
    c, s = math.cos(th), math.sin(th)
    table = {
        (0, 0): 1.0 / math.sqrt(4 * math.pi),
        (1, 0): math.sqrt(3 / (4 * math.pi)) * c,
        (1, 1): -math.sqrt(3 / (8 * math.pi)) * s,
        (2, 0): math.sqrt(5 / (16 * math.pi)) * (3 * c * c - 1),
        (2, 1): -math.sqrt(15 / (8 * math.pi)) * s * c,
        (2, 2): math.sqrt(15 / (32 * math.pi)) * s * s,
    }
    return table[(l, m)]


@pytest.mark.parametrize("th", [0.05, 0.7, 1.5707963267948966, 2.3, 3.1])
def test_legendre_low_l_closed_forms(oracle, th):
    for m in range(3):
        lam = oracle.legendre(2, m, math.cos(th))
        for l in range(m, 3):
            assert lam[l - m] == pytest.approx(_closed_form(l, m, th), abs=1e-15)


def test_legendre_against_scipy(oracle):
    rng = np.random.default_rng(3)
    for _ in range(20):
        th = rng.uniform(0.01, math.pi - 0.01)
        m = int(rng.integers(0, 60))
        lam = oracle.legendre(120, m, math.cos(th))
        ref = np.array([sp.sph_harm_y(l, m, th, 0.0).real for l in range(m, 121)])
        np.testing.assert_allclose(lam, ref, atol=1e-13, rtol=1e-11)


@pytest.mark.parametrize("m", [0, 3, 50, 400, 1000])
def test_legendre_orthonormal_by_quadrature(oracle, m):
    """2 pi int lambda_lm lambda_l'm dx = delta_ll' (Gauss-Legendre, exact for
    the polynomial degree involved).  At m = 400 and 1000 the seed sin^m is
    far below the double range near the poles, so this also pins the scaled
    exponent of the seed."""
    lmax = m + 160
    x, wq = leggauss(lmax + 2)
    lam = np.array([oracle.legendre(lmax, m, xi) for xi in x])  # (nodes, l)
    gram = 2 * np.pi * (lam.T * wq) @ lam
    np.testing.assert_allclose(gram, np.eye(lmax - m + 1), atol=1e-11)


def test_legendre_seed_closed_form_high_m(oracle):
    """lambda_mm = (-1)^m sqrt((2m+1)/(4pi) (2m)!/(2^m m!)^2) sin^m theta,
    compared in logs via lgamma at m = 4096."""
    for m, th in [(4096, 1.45), (3000, 1.2), (777, 0.9)]:
        lam = oracle.legendre(m, m, math.cos(th))[0]
        logref = 0.5 * (math.log((2 * m + 1) / (4 * math.pi)) + math.lgamma(2 * m + 1)
                        - 2 * math.lgamma(m + 1) - 2 * m * math.log(2)) + m * math.log(math.sin(th))
        assert lam != 0.0
        assert math.copysign(1, lam) == (-1) ** m
        assert math.log(abs(lam)) == pytest.approx(logref, abs=1e-9)


def _direct_synthesis(oracle, nside, lmax, a):
    th, ph = oracle.pixel_angles(nside)
    l, m = oracle.alm_lm(lmax)
    f = np.zeros(th.size)
    for k in range(l.size):
        Y = sp.sph_harm_y(int(l[k]), int(m[k]), th, ph)
        f += (a[k] * Y).real * (1.0 if m[k] == 0 else 2.0)
    return f


def _random_alm(oracle, lmax, rng):
    l, m = oracle.alm_lm(lmax)
    a = rng.standard_normal(l.size) + 1j * rng.standard_normal(l.size)
    a[m == 0] = a[m == 0].real
    return a


@pytest.mark.parametrize("nside,lmax", [(2, 5), (4, 8), (8, 20)])
def test_synthesis_against_direct_spherical_harmonics(oracle, nside, lmax):
    rng = np.random.default_rng(nside)
    a = _random_alm(oracle, lmax, rng)
    f = oracle.synthesis(nside, lmax, lmax, a)
    np.testing.assert_allclose(f, _direct_synthesis(oracle, nside, lmax, a), atol=1e-12)


def test_synthesis_band_limit(oracle):
    rng = np.random.default_rng(5)
    nside, lmax, L = 8, 20, 9
    a = _random_alm(oracle, lmax, rng)
    l, _ = oracle.alm_lm(lmax)
    cut = np.where(l <= L, a, 0)
    np.testing.assert_allclose(oracle.synthesis(nside, lmax, L, a),
                               oracle.synthesis(nside, lmax, lmax, cut), atol=1e-13)


@pytest.mark.parametrize("nside,lmax", [(4, 8), (8, 24), (16, 40)])
def test_adjoint_dot_product_identity(oracle, nside, lmax):
    """<Y a, f> = Re sum w conj(a) (Y^T f), w = 1 (m = 0) or 2 (m > 0)."""
    rng = np.random.default_rng(11)
    a = _random_alm(oracle, lmax, rng)
    f = rng.standard_normal(oracle.npix(nside))
    lhs = float(np.dot(oracle.synthesis(nside, lmax, lmax, a), f))
    _, m = oracle.alm_lm(lmax)
    w = np.where(m == 0, 1.0, 2.0)
    rhs = float(np.sum(w * (np.conj(a) * oracle.adjoint_synthesis(nside, lmax, lmax, f)).real))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_analysis_of_synthesis_near_identity(oracle):
    """HEALPix quadrature: Omega Y^T Y a ~ a for l well below 2 nside, with
    the error falling as nside grows at fixed lmax."""
    rng = np.random.default_rng(2)
    lmax = 8
    errs = []
    for nside in (8, 16, 32):
        a = _random_alm(oracle, lmax, rng)
        om = 4 * np.pi / oracle.npix(nside)
        back = om * oracle.adjoint_synthesis(nside, lmax, lmax, oracle.synthesis(nside, lmax, lmax, a))
        errs.append(np.max(np.abs(back - a)) / np.max(np.abs(a)))
    assert errs[0] < 5e-2 and errs[2] < errs[1] < errs[0]


def test_subsets_match_full(oracle):
    rng = np.random.default_rng(9)
    nside, lmax = 8, 16
    a = _random_alm(oracle, lmax, rng)
    full = oracle.synthesis(nside, lmax, lmax, a)
    part = oracle.synthesis(nside, lmax, lmax, a, rings=(5, 9))
    g = oracle.healpix_rings(nside)
    lo, hi = g["offset"][5], g["offset"][9]
    np.testing.assert_allclose(part[lo:hi], full[lo:hi], atol=1e-14)
    assert np.all(np.isnan(part[:lo])) and np.all(np.isnan(part[hi:]))
    f = rng.standard_normal(oracle.npix(nside))
    bfull = oracle.adjoint_synthesis(nside, lmax, lmax, f)
    bpart = oracle.adjoint_synthesis(nside, lmax, lmax, f, ms=(3, 7))
    _, m = oracle.alm_lm(lmax)
    sel = (m >= 3) & (m < 7)
    np.testing.assert_allclose(bpart[sel], bfull[sel], atol=1e-13)
