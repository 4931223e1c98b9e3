"""Pins of the oracle's spin-weighted harmonics and polarisation transforms
(the spin-2 basis change behind Eqs. 10-11), each against something the
oracle does not compute itself."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


@pytest.fixture(scope="module")
def oracle():
    import oracle as o

    return o


def wigner_d_explicit(j, a, b, beta):
    """Wigner's explicit sum for d^j_{ab}(beta), term by term in Python."""
    c, s = math.cos(beta / 2), math.sin(beta / 2)
    tot = 0.0
    for k in range(0, 2 * j + 1):
        args = (j + b - k, k, a - b + k, j - a - k)
        if min(args) < 0:
            continue
        num = math.sqrt(math.factorial(j + a) * math.factorial(j - a) * math.factorial(j + b) * math.factorial(j - b))
        den = math.factorial(args[0]) * math.factorial(k) * math.factorial(args[2]) * math.factorial(args[3])
        tot += (-1) ** (a - b + k) * num / den * c ** (2 * j + b - a - 2 * k) * s ** (a - b + 2 * k)
    return tot


def test_spin0_is_the_condon_shortley_legendre(oracle):
    for m in (0, 1, 2, 5, 13):
        for x in (-0.97, -0.3, 0.0, 0.41, 0.999):
            np.testing.assert_allclose(oracle.spin_legendre(40, m, 0, x)[m:], oracle.legendre(40, m, x),
                                       rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("s", [2, -2])
def test_spin2_matches_wigners_explicit_sum(oracle, s):
    for m in range(-8, 9):
        for th in (0.13, 0.9, 1.6, 2.7):
            got = oracle.spin_legendre(10, m, s, math.cos(th))
            for l in range(max(abs(m), 2), 11):
                ref = math.sqrt((2 * l + 1) / (4 * math.pi)) * wigner_d_explicit(l, m, -s, th)
                assert got[l] == pytest.approx(ref, rel=1e-11, abs=1e-13), (m, th, l)


def test_spin2_orthonormal_by_quadrature(oracle):
    x, w = np.polynomial.legendre.leggauss(80)
    lmax = 40
    for m in (-7, -2, 0, 1, 2, 6, 20):
        V = np.array([oracle.spin_legendre(lmax, m, 2, xi) for xi in x])  # nodes x l
        G = 2 * np.pi * (V * w[:, None]).T @ V
        l0 = max(abs(m), 2)
        np.testing.assert_allclose(G[l0:, l0:], np.eye(lmax + 1 - l0), atol=1e-12)


def test_spin2_m0_is_the_second_associated_legendre(oracle):
    """2lambda_l0 = sqrt((2l+1)/(4 pi) (l-2)!/(l+2)!) P_l^2(x) (scipy), one sign for all l."""
    from scipy.special import lpmv

    sgn = None
    for x in (-0.8, -0.1, 0.35, 0.9):
        got = oracle.spin_legendre(30, 0, 2, x)
        for l in range(2, 31):
            ref = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - 2) / math.factorial(l + 2)) * lpmv(2, l, x)
            if sgn is None:
                sgn = np.sign(got[l] / ref)
            assert got[l] == pytest.approx(sgn * ref, rel=1e-10, abs=1e-14)


def _rand_eb(rng, lmax, L):
    from wf_inputs import alm_unit_gaussian

    E = alm_unit_gaussian(rng, lmax)
    B = alm_unit_gaussian(rng, lmax)
    ell, m = __import__("oracle").alm_lm(lmax)
    E[(ell < 2) | (ell > L)] = 0.0
    B[(ell < 2) | (ell > L)] = 0.0
    return E, B


@pytest.mark.parametrize("nside,lmax,L", [(4, 8, 8), (8, 16, 11)])
def test_pol_adjoint_identity(oracle, nside, lmax, L):
    rng = np.random.default_rng(nside)
    E, B = _rand_eb(rng, lmax, L)
    Q, U = oracle.synthesis_pol(nside, lmax, L, E, B)
    q = rng.standard_normal(Q.size)
    u = rng.standard_normal(U.size)
    Et, Bt = oracle.adjoint_pol(nside, lmax, L, q, u)
    ell, m = oracle.alm_lm(lmax)
    w = np.where(m == 0, 1.0, 2.0)
    lhs = np.dot(Q, q) + np.dot(U, u)
    rhs = np.sum(w * (np.conj(E) * Et + np.conj(B) * Bt).real)
    assert lhs == pytest.approx(rhs, rel=1e-11)


def test_axisymmetric_e_and_b_modes(oracle):
    """m = 0: a pure E mode gives U = 0 and Q(theta) = -E_l0 2lambda_l0; a pure
    B mode gives Q = 0 and U(theta) = -B_l0 2lambda_l0."""
    nside, lmax = 8, 16
    ell, m = oracle.alm_lm(lmax)
    z = np.repeat(oracle.healpix_rings(nside)["z"], oracle.healpix_rings(nside)["nr"])
    for l in (2, 5, 11):
        E = np.zeros(ell.size, dtype=np.complex128)
        k = oracle.alm_index(lmax, l, 0)
        E[k] = 0.7
        Q, U = oracle.synthesis_pol(nside, lmax, lmax, E, np.zeros_like(E))
        lam = np.array([oracle.spin_legendre(lmax, 0, 2, zz)[l] for zz in z])
        np.testing.assert_allclose(U, 0.0, atol=1e-13)
        np.testing.assert_allclose(Q, -0.7 * lam, atol=1e-13)
        Q, U = oracle.synthesis_pol(nside, lmax, lmax, np.zeros_like(E), E)
        np.testing.assert_allclose(Q, 0.0, atol=1e-13)
        np.testing.assert_allclose(U, -0.7 * lam, atol=1e-13)


def test_e_b_exchange_rotates_the_polarisation(oracle):
    """(E, B) -> (B, -E) multiplies 2a = -(E + iB) by -i, so Q + iU -> -i (Q + iU):
    the polarisation rotates by 45 degrees, (Q, U) -> (U, -Q)."""
    rng = np.random.default_rng(3)
    E, B = _rand_eb(rng, 12, 12)
    Q, U = oracle.synthesis_pol(8, 12, 12, E, B)
    Q2, U2 = oracle.synthesis_pol(8, 12, 12, B, -E)
    np.testing.assert_allclose(Q2, U, atol=1e-12)
    np.testing.assert_allclose(U2, -Q, atol=1e-12)
