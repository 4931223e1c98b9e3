"""Pins for the oracle's template marginalisation (paper Sect. 3, Eq. 12)."""
import numpy as np
import pytest

import wf_inputs as gen


def _case(oracle, nside, seed):
    P = gen.healpix_problem(nside, 2 * nside, seed, fwhm_arcmin=60.0, b_cut_deg=20.0, n_disks=4,
                            disk_radius_deg=10.0, draws=True)
    d = oracle.synthesis(nside, 2 * nside, 2 * nside, P["a_signal"]) + P["noise"]
    return P, d


def test_projection_properties(oracle):
    nside = 8
    P, d = _case(oracle, nside, 11)
    V = oracle.template_matrix(nside, P["mask"])
    out, c = oracle.marginalize_templates(nside, d, P["mask"])
    np.testing.assert_allclose(V.T @ out, 0.0, atol=1e-10 * np.abs(d).sum())
    again, c2 = oracle.marginalize_templates(nside, out, P["mask"])
    np.testing.assert_allclose(again, out, atol=1e-12)
    np.testing.assert_allclose(c2, 0.0, atol=1e-10)
    # masked pixels carry no template, so they are left as they were
    masked = P["mask"] == 0
    np.testing.assert_array_equal(out[masked], d[masked])


def test_pure_monopole_and_dipole_are_removed(oracle):
    nside = 8
    P, _ = _case(oracle, nside, 12)
    th, ph = oracle.pixel_angles(nside)
    pure = 3.0 - 0.5 * np.sin(th) * np.cos(ph) + 0.25 * np.sin(th) * np.sin(ph) + 2.0 * np.cos(th)
    out, c = oracle.marginalize_templates(nside, pure, P["mask"])
    obs = P["mask"] > 0
    np.testing.assert_allclose(out[obs], 0.0, atol=1e-12)
    np.testing.assert_allclose(c, [3.0, -0.5, 0.25, 2.0], rtol=1e-12)


def test_limit_of_the_dense_finite_sigma_form(oracle):
    """(1 + sigma V V^T)^-1 d solved densely, sigma large, against the limit."""
    nside = 4
    P, d = _case(oracle, nside, 13)
    V = oracle.template_matrix(nside, P["mask"])
    lim, _ = oracle.marginalize_templates(nside, d, P["mask"])
    errs = []
    for sigma in (1e4, 1e6):  # beyond ~1e7 the dense system itself is too ill-conditioned
        dense = np.linalg.solve(np.eye(d.size) + sigma * V @ V.T, d)
        errs.append(np.max(np.abs(dense - lim)))
        assert errs[-1] < 0.05 / sigma * np.max(np.abs(d))
    assert errs[1] < errs[0] / 50.0  # the error falls as 1/sigma
    wood, _ = oracle.marginalize_templates(nside, d, P["mask"], sigma=1e3)
    dense = np.linalg.solve(np.eye(d.size) + 1e3 * V @ V.T, d)
    np.testing.assert_allclose(wood, dense, atol=1e-12 * np.max(np.abs(d)))
