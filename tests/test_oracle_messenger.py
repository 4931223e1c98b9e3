"""Pins for the oracle's messenger iteration (Eqs. 2-9 of the paper).

Every dense reference here is built from explicit DFT matrices or scipy's
spherical harmonics, never from the oracle's own transforms."""
import math

import numpy as np
import pytest
from scipy import special as sp

import wf_inputs as gen

# ---------------------------------------------------------------------------
# dense flat-sky helpers (explicit unitary DFT matrices)
# ---------------------------------------------------------------------------


def _dft2(n):
    j = np.arange(n)
    f = np.exp(-2j * np.pi * np.outer(j, j) / n) / math.sqrt(n)
    return np.kron(f, f)  # acts on row-major flattened n x n maps


def _full_plane(S_half, n):
    """Half-plane (n, n/2+1) prior -> full n x n plane."""
    full = np.empty((n, n))
    h = n // 2 + 1
    full[:, :h] = S_half
    ky = (-np.arange(n)) % n
    for kx in range(h, n):
        full[:, kx] = S_half[ky, n - kx]
    return full


class DenseFlat:
    def __init__(self, P):
        n = P["ny"]
        self.n = n
        self.F = _dft2(n)
        Sf = _full_plane(P["S"], n).ravel()
        self.S = (self.F.conj().T @ np.diag(Sf) @ self.F).real
        self.Sinv = (self.F.conj().T @ np.diag(1.0 / Sf) @ self.F).real


def _problem(n=16, **kw):
    kw.setdefault("band_rows", (7, 9))
    kw.setdefault("n_disks", 2)
    kw.setdefault("disk_radius", 1.5)
    P = gen.flat_problem(n, seed=kw.pop("seed", 7), **kw)
    return P


def _setup(oracle, P):
    B = oracle.FlatBasis(P["ny"], P["nx"])
    d = B.synth(P["a_signal"]) + P["noise"]
    obs = P["mask"] > 0
    nu = np.where(obs, 1.0 / P["noise_var"], 0.0)
    tau = float(P["noise_var"][obs].min())
    return B, d, nu, tau


# ---------------------------------------------------------------------------
# flat sky
# ---------------------------------------------------------------------------


def test_flat_converges_to_dense_wiener_filter(oracle):
    """Eq. (2): (S^-1 + N^-1) s_WF = N^-1 d, masked pixels at N^-1 = 0."""
    P = _problem()
    B, d, nu, tau = _setup(oracle, P)
    D = DenseFlat(P)
    s_ref = np.linalg.solve(D.Sinv + np.diag(nu.ravel()), (nu * d).ravel())
    res = oracle.messenger_solve(B, nu * d, nu, P["S"], tau, tol=1e-12)
    assert res["converged"]
    err = np.max(np.abs(res["s"].ravel() - s_ref)) / np.max(np.abs(s_ref))
    assert err < 1e-9


def test_flat_one_step_exact_for_homogeneous_noise(oracle):
    """Sect. 2.2: with N proportional to 1 the system is solved in a single
    iteration (lam = 1): s = S (S + N)^-1 d."""
    P = _problem(homogeneous=True, masked=False)
    B, d, nu, tau = _setup(oracle, P)
    res = oracle.messenger_solve(B, nu * d, nu, P["S"], tau, replay=[(1.0, None)])
    expect = P["S"] / (P["S"] + tau) * np.fft.rfft2(d, norm="ortho")
    np.testing.assert_allclose(res["a"], expect, atol=1e-13 * np.max(np.abs(expect)))
    D = DenseFlat(P)
    s_dense = D.S @ np.linalg.solve(D.S + tau * np.eye(d.size), d.ravel())
    np.testing.assert_allclose(res["s"].ravel(), s_dense, atol=1e-12)


def _s_lambda(D, nu, tau, lam, d):
    """Dense s(lam) = S (S + N + (lam - 1) T)^-1 d, in information form so that
    masked pixels (N = infinity) are exact: (S^-1 + W) s = W d,
    W = diag(nu / (1 + (lam - 1) tau nu))."""
    W = (nu / (1.0 + (lam - 1.0) * tau * nu)).ravel()
    return np.linalg.solve(D.Sinv + np.diag(W), W * d.ravel()), W


@pytest.mark.parametrize("lam", [1.0, 3.0, 40.0])
def test_flat_error_contraction_bound(oracle, lam):
    """Eq. (5): eps_{i+1} = [S(S + lam T)^-1][Nbar(Nbar + lam T)^-1] eps_i, so
    |eps_{i+1}| <= rho1 rho2 |eps_i|."""
    P = _problem()
    B, d, nu, tau = _setup(oracle, P)
    D = DenseFlat(P)
    s_lam, _ = _s_lambda(D, nu, tau, lam, d)
    rho1 = float(np.max(P["S"] / (P["S"] + lam * tau)))
    Nbar = np.where(nu > 0, P["noise_var"] - tau, np.inf)
    rho2 = float(np.max(np.where(np.isinf(Nbar), 1.0, Nbar / (Nbar + lam * tau))))
    errs = []
    oracle.messenger_solve(B, nu * d, nu, P["S"], tau, replay=[(lam, None)] * 25,
                           callback=lambda k, a: errs.append(np.linalg.norm(B.synth(a).ravel() - s_lam)))
    errs = np.array(errs)
    assert np.all(errs[1:] <= rho1 * rho2 * errs[:-1] * (1 + 1e-10) + 1e-13)
    assert errs[-1] < errs[0]


@pytest.mark.parametrize("masked", [False, True])
def test_flat_fixed_lambda_limit_and_chi2_min(oracle, masked):
    """Sect. 2.2: at fixed lam the iterations converge to
    s(lam) = S (S + N + (lam - 1) T)^-1 d, where
    chi2_min(lam) = d^T (S + N + (lam - 1) T)^-1 d = d^T S^-1 s(lam)."""
    lam = 4.0
    P = _problem(masked=masked)
    B, d, nu, tau = _setup(oracle, P)
    D = DenseFlat(P)
    s_lam, W = _s_lambda(D, nu, tau, lam, d)
    res = oracle.messenger_solve(B, nu * d, nu, P["S"], tau, replay=[(lam, None)] * 3000)
    np.testing.assert_allclose(res["s"].ravel(), s_lam, atol=1e-10 * np.max(np.abs(s_lam)))
    x = res["s"].ravel()
    dv = d.ravel()
    chi2 = x @ D.Sinv @ x + np.sum(W * (dv - x) ** 2)
    obs = (nu > 0).ravel()
    Cn = D.S[np.ix_(obs, obs)] + np.diag(1.0 / W[obs])
    chi2_ref = dv[obs] @ np.linalg.solve(Cn, dv[obs])
    assert chi2 == pytest.approx(chi2_ref, rel=1e-9)
    if not masked:
        assert chi2 == pytest.approx(dv @ D.Sinv @ s_lam, rel=1e-9)


def test_flat_chi2_monotone_at_fixed_lambda(oracle):
    """The iterations minimise chi^2(x, lam) (Eq. 6): it never increases."""
    P = _problem()
    B, d, nu, tau = _setup(oracle, P)
    for lam in (1.0, 7.0):
        res = oracle.messenger_solve(B, nu * d, nu, P["S"], tau, replay=[(lam, None)] * 60)
        c = res["chi2"]
        assert np.all(np.diff(c) <= 1e-11 * np.abs(c[:-1]))


def test_flat_residual_formula_is_true_residual(oracle):
    """At lam = 1 the reported residual equals |(S^-1 + N^-1) s_k - N^-1 d| /
    |N^-1 d| evaluated densely."""
    P = _problem()
    B, d, nu, tau = _setup(oracle, P)
    D = DenseFlat(P)
    its = []
    res = oracle.messenger_solve(B, nu * d, nu, P["S"], tau, replay=[(1.0, None)] * 8,
                                 callback=lambda k, a: its.append(B.synth(a).ravel()))
    rhs = (nu * d).ravel()
    xs = [np.zeros(d.size)] + its[:-1]
    for x, rep in zip(xs, res["resid"]):
        true = np.linalg.norm((D.Sinv + np.diag(nu.ravel())) @ x - rhs) / np.linalg.norm(rhs)
        assert rep == pytest.approx(true, rel=1e-9)


def test_flat_schedule_is_cooling(oracle):
    P = _problem(n=32, seed=3)
    B, d, nu, tau = _setup(oracle, P)
    res = oracle.messenger_solve(B, nu * d, nu, P["S"], tau, tol=1e-8)
    lams = np.array([t[0] for t in res["trace"]])
    assert lams[0] == 100.0 and lams[-1] == 1.0
    assert np.all(lams >= 1.0) and np.all(np.diff(lams) <= 0)
    assert res["converged"] and res["resid"][-1] < 1e-8


# ---------------------------------------------------------------------------
# fluctuation maps (Sect. 2.3)
# ---------------------------------------------------------------------------


def test_fluct_source_masked_identity(oracle):
    """Eq. (9) literally: Nbar^-1 d -> Nbar^-1 N (N^-1/2 g1 + S^-1/2 g2) with
    Nbar^-1 N -> 1 in masked pixels, inserted in Eq. (3) and Eq. (4) for one
    step from s = 0, against the oracle's source-vector form."""
    P = _problem()
    B, d, nu, tau = _setup(oracle, P)
    lam = 2.5
    obs = nu > 0
    N = P["noise_var"]
    z = B.synth(np.where(P["S"] > 0, P["g2"] / np.sqrt(P["S"]), 0.0))  # S^-1/2 g2 in pixel basis
    Nbar = N - tau
    t = np.empty_like(N)
    # Eq. (3) with s = 0: (Nbar^-1 + (lam T)^-1) t = Nbar^-1 N (N^-1/2 g1 + z)
    with np.errstate(divide="ignore"):
        nb_inv = np.where(obs, 1.0 / Nbar, 0.0)
    src_obs = nb_inv * N * (P["g1"] / np.sqrt(N) + z)
    lim = obs & (Nbar == 0)  # the minimum-noise pixel: Nbar -> 0 limit
    t[obs & ~lim] = (src_obs / (nb_inv + 1.0 / (lam * tau)))[obs & ~lim]
    t[lim] = (N * (P["g1"] / np.sqrt(N) + z))[lim]
    t[~obs] = lam * tau * z[~obs]  # identity block: (1/(lam tau)) t = z
    expect = P["S"] / (P["S"] + lam * tau) * np.fft.rfft2(t, norm="ortho")
    r = oracle.fluct_source(B, nu, P["S"], P["g1"], P["g2"])
    res = oracle.messenger_solve(B, r, nu, P["S"], tau, replay=[(lam, None)])
    np.testing.assert_allclose(res["a"], expect, atol=1e-12 * np.max(np.abs(expect)))


def _mc_problem(n=8, seed=21):
    P = gen.flat_problem(n, seed=seed, masked=False, noise_decades=0.5)
    return P


def test_fluct_covariance_monte_carlo(oracle):
    """Eq. (8): <f f^T> = (S^-1 + N^-1)^-1, by 4000 draws on an 8 x 8 grid."""
    P = _mc_problem()
    n = P["ny"]
    B = oracle.FlatBasis(n, n)
    nu = 1.0 / P["noise_var"]
    tau = float(P["noise_var"].min())
    rng = np.random.default_rng(99)
    nd = 4000
    g1 = rng.standard_normal((nd, n, n))
    g2 = np.stack([gen.flat_unit_gaussian(rng, n, n) for _ in range(nd)])
    r = oracle.fluct_source(B, nu, P["S"], g1, g2)
    res = oracle.messenger_solve(B, r, nu, P["S"], tau, replay=[(1.0, None)] * 150)
    f = res["s"].reshape(nd, -1)
    C = f.T @ f / nd
    D = DenseFlat(P)
    Cref = np.linalg.inv(D.Sinv + np.diag(nu.ravel()))
    L = np.linalg.cholesky(Cref)
    Li = np.linalg.inv(L)
    ev = np.linalg.eigvalsh(Li @ C @ Li.T)
    assert abs(ev.mean() - 1.0) < 0.03
    assert ev.min() > 0.6 and ev.max() < 1.45


def test_wiener_covariance_and_chi2_statistics_monte_carlo(oracle):
    """Eq. (7): <s_WF s_WF^T> = S (S + N)^-1 S over data drawn from the model,
    and chi2_min(1) ~ chi^2(n_dof): mean n_dof (Sect. 2.2)."""
    P = _mc_problem(seed=22)
    n = P["ny"]
    B = oracle.FlatBasis(n, n)
    nu = 1.0 / P["noise_var"]
    tau = float(P["noise_var"].min())
    D = DenseFlat(P)
    rng = np.random.default_rng(5)
    nd = 4000
    sig = np.stack([B.synth(np.sqrt(P["S"]) * gen.flat_unit_gaussian(rng, n, n)) for _ in range(nd)])
    d = sig + np.sqrt(P["noise_var"]) * rng.standard_normal((nd, n, n))
    res = oracle.messenger_solve(B, nu * d, nu, P["S"], tau, replay=[(1.0, None)] * 150)
    s = res["s"].reshape(nd, -1)
    C = s.T @ s / nd
    Cref = D.S @ np.linalg.solve(D.S + np.diag(P["noise_var"].ravel()), D.S)
    L = np.linalg.cholesky(Cref)
    Li = np.linalg.inv(L)
    ev = np.linalg.eigvalsh(Li @ C @ Li.T)
    assert abs(ev.mean() - 1.0) < 0.03
    assert ev.min() > 0.6 and ev.max() < 1.45
    # chi^2_min(1) per draw: s^T S^-1 s + (d - s)^T N^-1 (d - s)
    dv = d.reshape(nd, -1)
    chi2 = np.einsum("bi,ij,bj->b", s, D.Sinv, s) + np.sum(nu.ravel() * (dv - s) ** 2, axis=1)
    ndof = n * n
    assert abs(chi2.mean() - ndof) < 4.0 * math.sqrt(2 * ndof / nd)


# ---------------------------------------------------------------------------
# HEALPix: dense discrete fixed-point system at nside 4
# ---------------------------------------------------------------------------


def _dense_healpix(oracle, nside, lmax):
    """Real-coordinate synthesis matrix from scipy's Y_lm at the pixel
    centres: x = (Re a_l0; Re a_lm, Im a_lm for m > 0)."""
    th, ph = oracle.pixel_angles(nside)
    l, m = oracle.alm_lm(lmax)
    cols, wts, modes = [], [], []
    for k in range(l.size):
        Y = sp.sph_harm_y(int(l[k]), int(m[k]), th, ph)
        if m[k] == 0:
            cols.append(Y.real)
            wts.append(1.0)
            modes.append((k, 0))
        else:
            cols.append(2 * Y.real)
            cols.append(-2 * Y.imag)
            wts += [2.0, 2.0]
            modes += [(k, 0), (k, 1)]
    return np.array(cols).T, np.array(wts), modes


def _to_x(a, modes):
    return np.array([a[k].real if p == 0 else a[k].imag for k, p in modes])


@pytest.mark.parametrize("nside,lmax", [(4, 8), (8, 12)])
def test_healpix_converges_to_dense_fixed_point(oracle, nside, lmax):
    """On HEALPix the analysis Omega Y^T is not the inverse of Y, so the
    iteration's fixed point is the discrete system
    [S^-1 + Y^T nu Y + (I - Omega Y^T Y) / (tau Omega)] a = Y^T r;
    solved densely from scipy's Y_lm, and the iteration matrix at lam = 1
    has spectral radius < 1."""
    P = gen.healpix_problem(nside, lmax, seed=31, fwhm_arcmin=60.0, b_cut_deg=20.0,
                            n_disks=2, disk_radius_deg=15.0, noise_level_ell=lmax)
    basis = oracle.HealpixBasis(nside, lmax)
    d = basis.synth(P["a_signal"]) + P["noise"]
    obs = P["mask"] > 0
    nu = np.where(obs, 1.0 / P["noise_var"], 0.0)
    tau = float(P["noise_var"][obs].min())
    om = basis.omega
    S = basis.per_mode(P["c_ell"])
    sched = oracle.messenger.HealpixSchedule(P["c_ell"], tau * om, lmax)
    res = oracle.messenger_solve(basis, nu * d, nu, S, tau, schedule=sched, tol=1e-12)
    assert res["converged"]

    Y, W, modes = _dense_healpix(oracle, nside, lmax)
    Sx = np.array([S[k] for k, _ in modes])
    act = Sx > 0
    Yt = (Y.T / W[:, None])  # weighted adjoint in x coordinates
    M = np.diag(1.0 / Sx[act]) + (Yt @ (nu[:, None] * Y))[np.ix_(act, act)] \
        + (np.eye(act.sum()) - om * (Yt @ Y)[np.ix_(act, act)]) / (tau * om)
    rhs = (Yt @ (nu * d))[act]
    x_ref = np.linalg.solve(M, rhs)
    x = _to_x(res["a"], modes)[act]
    assert np.max(np.abs(x - x_ref)) / np.max(np.abs(x_ref)) < 1e-9

    # iteration matrix at lam = 1: a' = diag(S/(S+tau Om)) Om Y^T diag(1 - tau nu) Y a
    It = np.diag(Sx[act] / (Sx[act] + tau * om)) @ (om * Yt @ ((1.0 - tau * nu)[:, None] * Y))[np.ix_(act, act)]
    assert np.max(np.abs(np.linalg.eigvals(It))) < 1.0

    # the reported residual is |M a_k - b| / |b| in the weighted norm
    its = []
    replay = [(1.0, lmax)] * 4
    r2 = oracle.messenger_solve(basis, nu * d, nu, S, tau, replay=replay,
                                callback=lambda k, a: its.append(_to_x(a, modes)[act]))
    xs = [np.zeros(act.sum())] + its[:-1]
    Wa = W[act]
    for xk, rep in zip(xs, r2["resid"]):
        rr = M @ xk - rhs
        true = math.sqrt(np.sum(Wa * rr ** 2)) / math.sqrt(np.sum(Wa * rhs ** 2))
        assert rep == pytest.approx(true, rel=1e-9)


def test_healpix_schedule_follows_paper(oracle):
    """Sect. 3: l_iter starts at 20 and doubles (increment <= 500), lam =
    max(1, S_l_iter / tau_h), band limit L = l_iter + 100 <= lmax."""
    c = gen.cmb_like_cl(4096, 5.0)
    tau_h = c[2048] * 0.1
    s = oracle.messenger.HealpixSchedule(c, tau_h, 4096)
    seen = [(s.ell_iter, s.lam, s.L)]
    while not s.final:
        s.advance()
        seen.append((s.ell_iter, s.lam, s.L))
    ells = [e for e, _, _ in seen]
    assert ells[:7] == [20, 40, 80, 160, 320, 640, 1140]
    assert all(b - a <= 500 for a, b in zip(ells, ells[1:]))
    for e, lam, L in seen[:-1]:
        assert lam == pytest.approx(max(1.0, c[e] / tau_h))
        assert L == min(4096, e + 100)
    assert seen[-1][1] == 1.0 and seen[-1][2] == 4096


# ---------------------------------------------------------------------------
# chi^2-bound cooling (Sect. 2.2)
# ---------------------------------------------------------------------------


def test_rigorous_schedule_keeps_the_chi2_bound(oracle):
    """Each lambda > 1 is chosen so that chi^2(lambda, x) = b for the current
    iterate (dense chi^2 of Eq. 6, including its x-independent part); b stays
    below chi2_min(1) = d^T (S + N)^-1 d and approaches it; the result is the
    Wiener filter of Eq. (2)."""
    from oracle.messenger import RigorousSchedule

    P = _problem()
    B, d, nu, tau = _setup(oracle, P)
    D = DenseFlat(P)
    obs = (nu > 0).ravel()
    dv = d.ravel()
    chi2_min1 = dv[obs] @ np.linalg.solve(D.S[np.ix_(obs, obs)] + np.diag(P["noise_var"].ravel()[obs]), dv[obs])
    sch = RigorousSchedule(int(obs.sum()))
    b0 = sch.b
    xs = [np.zeros(d.size)]
    res = oracle.messenger_solve(B, nu * d, nu, P["S"], tau, schedule=sch, tol=1e-11, d=d,
                                 callback=lambda k, a: xs.append(B.synth(a).ravel()))
    assert res["converged"]
    lams = np.array([t[0] for t in res["trace"]])
    assert lams[0] > 1.0 and np.all(np.diff(lams) <= 0) and lams[-1] == 1.0
    W = lambda lam: (nu / (1.0 + (lam - 1.0) * tau * nu)).ravel()
    checked = 0
    for k, (lam, bk) in enumerate(zip(lams, res["bound"])):
        if lam <= 1.0:
            break
        x = xs[k]
        chi2 = x @ D.Sinv @ x + np.sum(W(lam) * (dv - x) ** 2)
        assert chi2 == pytest.approx(bk, rel=1e-9)
        checked += 1
    assert checked > 5
    assert res["bound"].max() <= chi2_min1 * (1 + 1e-10)  # b approaches chi2_min(1) from below up to rounding
    assert b0 < res["bound"].max() and (chi2_min1 - res["bound"].max()) < 0.1 * (chi2_min1 - b0)
    s_ref = np.linalg.solve(D.Sinv + np.diag(nu.ravel()), (nu * d).ravel())
    assert np.max(np.abs(res["s"].ravel() - s_ref)) / np.max(np.abs(s_ref)) < 1e-8


def test_rigorous_initial_lambda(oracle):
    """The first lambda solves d^T (N + (lambda - 1) T)^-1 d = b (Sect. 2.2)."""
    from oracle.messenger import RigorousSchedule

    P = _problem(seed=9)
    B, d, nu, tau = _setup(oracle, P)
    obs = nu > 0
    sch = RigorousSchedule(int(obs.sum()))
    b = sch.b
    res = oracle.messenger_solve(B, nu * d, nu, P["S"], tau, schedule=sch, tol=1e-6, d=d, maxiter=1)
    lam = res["trace"][0][0]
    N = P["noise_var"][obs]
    assert np.sum(d[obs] ** 2 / (N + (lam - 1.0) * tau)) == pytest.approx(b, rel=1e-10)
