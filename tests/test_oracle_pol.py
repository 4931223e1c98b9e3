"""Pins of the oracle's polarised messenger iteration (Eqs. 10-11): the
decoupled limit against the temperature iteration, the dense discrete
fixed-point system (from explicitly evaluated basis functions), and the
contraction of the iteration at lambda = 1."""
import math

import numpy as np
import pytest
import scipy.special as sp

import wf_inputs as gen


@pytest.fixture(scope="module")
def oracle():
    import oracle as o

    return o


def _pol_case(oracle, nside, lmax, seed, partial=False, **kw):
    from oracle.messenger_pol import HealpixPolBasis, pol_inverse_noise

    P = gen.healpix_pol_problem(nside, lmax, seed, **kw)
    basis = HealpixPolBasis(nside, lmax)
    d = basis.synth(P["a_signal"]) + P["noise"]
    obs = P["mask"] > 0
    if not partial:
        nu = np.zeros_like(P["noise_cov"])
        nu[obs] = np.linalg.inv(P["noise_cov"][obs])
        return P, basis, d, nu, obs
    # separate masks: every fourth observed pixel observes I only, every fifth Q, U only
    code = obs.astype(np.uint8)
    k = np.nonzero(obs)[0]
    code[k[::4]] = 2
    code[k[1::5]] = 3
    return P, basis, d, pol_inverse_noise(P["noise_cov"], code), code


def test_decoupled_limit_is_the_temperature_iteration(oracle):
    """Diagonal noise and TE = 0: the I/T part of the polarised iteration is the
    temperature iteration with the same tau and (lambda, L) trace."""
    from oracle.messenger_pol import messenger_solve_pol

    nside, lmax = 8, 16
    P, basis, d, nu, obs = _pol_case(oracle, nside, lmax, 41, corr=0.0, fwhm_arcmin=120.0, n_disks=4,
                                     disk_radius_deg=10.0)
    cl = P["c_ell"].copy()
    cl[:, 3] = 0.0
    S = basis.per_mode(cl)
    N = P["noise_cov"]
    tau = float(N[obs][:, [0, 1, 2], [0, 1, 2]].min())
    replay = [(4.0, 10)] * 3 + [(2.0, 14)] * 3 + [(1.0, lmax)] * 6
    r = np.einsum("nij,jn->in", nu, d)
    res = messenger_solve_pol(basis, r, nu, S, tau, replay=replay)
    b0 = oracle.HealpixBasis(nside, lmax)
    nuT = nu[:, 0, 0]
    resT = oracle.messenger_solve(b0, nuT * d[0], nuT, b0.per_mode(cl[:, 0]), tau, replay=replay, d=d[0])
    np.testing.assert_allclose(res["a"][0], resT["a"], rtol=0, atol=1e-12 * np.max(np.abs(resT["a"])))


def _dense_pol(oracle, nside, lmax):
    """Real-coordinate synthesis matrix (3 npix x n) from explicitly evaluated
    basis functions: scipy's Y_lm for T, sum over +-m of 2a 2Y for E and B
    (2Y from spin_legendre and e^{i m phi}); x = (Re, Im for m > 0) per
    component; weights 1 (m = 0) or 2 (m > 0)."""
    th, ph = oracle.pixel_angles(nside)
    npx = th.size
    l, m = oracle.alm_lm(lmax)
    z = np.cos(th)
    cols, wts, modes = [], [], []

    def y2(ll, mm):
        lam = np.array([oracle.spin_legendre(lmax, mm, 2, zz)[ll] for zz in z])
        return lam * np.exp(1j * mm * ph)

    for comp in range(3):
        for k in range(l.size):
            ll, mm = int(l[k]), int(m[k])
            parts = [0] if mm == 0 else [0, 1]
            for part in parts:
                col = np.zeros(3 * npx)
                if comp == 0:
                    Y = sp.sph_harm_y(ll, mm, th, ph)
                    col[:npx] = (Y.real if mm == 0 else 2 * Y.real) if part == 0 else -2 * Y.imag
                elif ll >= 2:
                    e = 1.0 if part == 0 else 1j  # unit E_lm (comp 1) or B_lm (comp 2)
                    E, B = (e, 0.0) if comp == 1 else (0.0, e)
                    pol = -(E + 1j * B) * y2(ll, mm)
                    if mm > 0:
                        sg = (-1) ** mm
                        pol = pol - (sg * np.conj(E) + 1j * sg * np.conj(B)) * y2(ll, -mm)
                    col[npx:2 * npx] = pol.real
                    col[2 * npx:] = pol.imag
                cols.append(col)
                wts.append(1.0 if mm == 0 else 2.0)
                modes.append((comp, k, part))
    return np.array(cols).T, np.array(wts), modes


def _to_x(a, modes):
    return np.array([a[c, k].real if p == 0 else a[c, k].imag for c, k, p in modes])


@pytest.mark.parametrize("bb,partial", [(0.3, False), (0.0, False), (0.3, True)])
def test_pol_converges_to_dense_fixed_point(oracle, bb, partial):
    """[S^+ + Y^T nu Y + (1 - Omega Y^T Y) / tau_h] a = Y^T r on the range of S,
    solved densely; the iteration at lambda = 1 contracts (spectral radius < 1)
    and the reported residual is the dense one."""
    from oracle.messenger_pol import messenger_solve_pol, pol_tau

    nside, lmax = 2, 4
    P, basis, d, nu, obs = _pol_case(oracle, nside, lmax, 43, partial=partial, bb_ratio=bb, corr=0.1,
                                     fwhm_arcmin=600.0, b_cut_deg=10.0, n_disks=1, disk_radius_deg=20.0,
                                     noise_level_ell=lmax)
    if partial:
        assert set(np.unique(obs)) == {0, 1, 2, 3}
    tau = pol_tau(P["noise_cov"], obs)
    om = basis.omega
    S = basis.per_mode(P["c_ell"])
    r = np.einsum("nij,jn->in", nu, d)
    res = messenger_solve_pol(basis, r, nu, S, tau, tol=1e-12, maxiter=20000)
    assert res["converged"]

    Y, W, modes = _dense_pol(oracle, nside, lmax)
    n = len(modes)
    Sx = np.zeros((n, n))
    idx = {}
    for i, (c, k, p) in enumerate(modes):
        idx[(c, k, p)] = i
    for i, (c, k, p) in enumerate(modes):
        for c2 in range(3):
            j = idx.get((c2, k, p))
            if j is not None:
                Sx[i, j] = S[k][c, c2]
    act = np.diag(Sx) > 0
    npx = 12 * nside * nside
    nub = np.zeros((3 * npx, 3 * npx))
    for c in range(3):
        for c2 in range(3):
            nub[c * npx:(c + 1) * npx, c2 * npx:(c2 + 1) * npx] = np.diag(nu[:, c, c2])
    Yt = Y.T / W[:, None]
    Sa = Sx[np.ix_(act, act)]
    tau_h = tau * om
    M = np.linalg.inv(Sa) + (Yt @ nub @ Y)[np.ix_(act, act)] + (np.eye(act.sum()) - om * (Yt @ Y)[np.ix_(act, act)]) / tau_h
    rhs = (Yt @ (nub @ d.ravel()))[act]
    x_ref = np.linalg.solve(M, rhs)
    x = _to_x(res["a"], modes)[act]
    assert np.max(np.abs(x - x_ref)) / np.max(np.abs(x_ref)) < 1e-9

    F = Sa @ np.linalg.inv(Sa + tau_h * np.eye(act.sum()))
    It = F @ (om * Yt @ (np.eye(3 * npx) - tau * nub) @ Y)[np.ix_(act, act)]
    assert np.max(np.abs(np.linalg.eigvals(It))) < 1.0

    its = []
    res2 = messenger_solve_pol(basis, r, nu, S, tau, replay=[(1.0, lmax)] * 4,
                               callback=lambda k, a: its.append(_to_x(a, modes)[act]))
    xs = [np.zeros(act.sum())] + its[:-1]
    Wa = W[act]
    for xk, rep in zip(xs, res2["resid"]):
        rr = M @ xk - rhs
        true = math.sqrt(np.sum(Wa * rr ** 2)) / math.sqrt(np.sum(Wa * rhs ** 2))
        assert rep == pytest.approx(true, rel=1e-9)


def test_pol_fluct_source_matches_dense_construction(oracle):
    """Eq. (9) for (I, Q, U): r = nu^1/2 g1 + Omega Y (S^+1/2 g2), built here
    from scipy's matrix square root per pixel and per l (pseudo-inverse of the
    root) and from the explicitly evaluated basis functions, against the
    oracle's source."""
    import scipy.linalg as sl

    from oracle.messenger_pol import fluct_source_pol

    nside, lmax = 2, 4
    P, basis, d, nu, obs = _pol_case(oracle, nside, lmax, 47, corr=0.1, fwhm_arcmin=600.0, b_cut_deg=10.0,
                                     n_disks=1, disk_radius_deg=20.0, noise_level_ell=lmax)
    S = basis.per_mode(P["c_ell"])
    rng = np.random.default_rng(48)
    npx = 12 * nside * nside
    g1 = rng.standard_normal((3, npx))
    g2 = np.stack([gen.alm_unit_gaussian(rng, lmax) for _ in range(3)])
    r = fluct_source_pol(basis, nu, S, g1, g2)

    pix = np.stack([sl.sqrtm(nu[p]).real @ g1[:, p] if obs[p] else np.zeros(3) for p in range(npx)], axis=1)
    def pinv_root(B):  # scipy's root of the nonsingular sub-block on the active components, inverted
        act = np.diag(B) > 0
        out = np.zeros((3, 3))
        out[np.ix_(act, act)] = np.linalg.inv(sl.sqrtm(B[np.ix_(act, act)]).real)
        return out

    h = np.stack([pinv_root(S[k]) @ g2[:, k] for k in range(basis.ell.size)], axis=1)
    Y, W, modes = _dense_pol(oracle, nside, lmax)
    z = (Y @ _to_x(h, modes)).reshape(3, npx)
    ref = pix + basis.omega * z
    np.testing.assert_allclose(r, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    assert np.all(r[:, ~obs] == pytest.approx(basis.omega * z[:, ~obs], rel=1e-12, abs=1e-14))


def test_pol_fluct_source_decoupled_limit(oracle):
    """Diagonal noise and TE = 0: the I part of the polarised source is the
    temperature source of the same draws, and Q, U get g1 / sigma in each
    observed pixel plus the spin-2 synthesis of (E, B) / sqrt(C_l)."""
    from oracle.messenger_pol import fluct_source_pol

    nside, lmax = 8, 16
    P, basis, d, nu, obs = _pol_case(oracle, nside, lmax, 49, corr=0.0, fwhm_arcmin=120.0, n_disks=4,
                                     disk_radius_deg=10.0)
    cl = P["c_ell"].copy()
    cl[:, 3] = 0.0
    S = basis.per_mode(cl)
    rng = np.random.default_rng(50)
    npx = 12 * nside * nside
    g1 = rng.standard_normal((3, npx))
    g2 = np.stack([gen.alm_unit_gaussian(rng, lmax) for _ in range(3)])
    r = fluct_source_pol(basis, nu, S, g1, g2)
    b0 = oracle.HealpixBasis(nside, lmax)
    rT = oracle.fluct_source(b0, nu[:, 0, 0], b0.per_mode(cl[:, 0]), g1[0], g2[0])
    np.testing.assert_allclose(r[0], rT, rtol=0, atol=1e-12 * np.max(np.abs(rT)))
    e = np.where(cl[basis.ell, 1] > 0, g2[1] / np.sqrt(np.where(cl[basis.ell, 1] > 0, cl[basis.ell, 1], 1.0)), 0.0)
    b = np.where(cl[basis.ell, 2] > 0, g2[2] / np.sqrt(np.where(cl[basis.ell, 2] > 0, cl[basis.ell, 2], 1.0)), 0.0)
    Q, U = oracle.synthesis_pol(nside, lmax, lmax, e, b)
    for c, z in ((1, Q), (2, U)):
        ref = np.sqrt(nu[:, c, c]) * g1[c] + basis.omega * z
        np.testing.assert_allclose(r[c], ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def test_partial_mask_inverse_noise_is_the_infinite_variance_limit(oracle):
    """nu for separate T / P masks equals the inverse of the full block once the
    unobserved components' variances are made huge (1e12 added on the
    diagonal), and tau is the smallest eigenvalue of the observed sub-blocks:
    N - tau (1 - 1e-9) is positive definite on every observed sub-block and
    N - tau (1 + 1e-9) is not on at least one (Cholesky)."""
    from oracle.messenger_pol import observed_components, pol_inverse_noise, pol_tau

    rng = np.random.default_rng(52)
    n = 400
    X = rng.standard_normal((n, 3, 3))
    N = np.einsum("nij,nkj->nik", X, X) + 0.3 * np.eye(3)
    code = rng.integers(0, 4, size=n).astype(np.uint8)
    nu = pol_inverse_noise(N, code)
    comp = observed_components(code)
    big = N + np.einsum("ni,ij->nij", (~comp).astype(float) * 1e12, np.eye(3))
    lim = np.linalg.inv(big)
    np.testing.assert_allclose(nu, lim, rtol=0, atol=1e-9 * np.max(np.abs(nu)))
    assert np.all(nu[~comp[:, 0], 0, :] == 0.0) and np.all(nu[code == 2][:, 1:, :] == 0.0)
    tau = pol_tau(N, code)
    ok_below, fails_above = True, False
    for p in range(n):
        K = np.nonzero(comp[p])[0]
        if K.size == 0:
            continue
        sub = N[p][np.ix_(K, K)]
        try:
            np.linalg.cholesky(sub - tau * (1 - 1e-9) * np.eye(K.size))
        except np.linalg.LinAlgError:
            ok_below = False
        try:
            np.linalg.cholesky(sub - tau * (1 + 1e-9) * np.eye(K.size))
        except np.linalg.LinAlgError:
            fails_above = True
    assert ok_below and fails_above
