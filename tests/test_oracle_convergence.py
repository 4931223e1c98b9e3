"""Why the lambda = 1 tail of the messenger iteration is long on the nside-2048
workload, shown densely at small nside with the same recipe (noise variance
range 1e4 over the observed pixels, |b| < 15 deg cut plus small disks, 5'
beam, noise level at C_l of lmax / 2).

Sect. 2.2, Eq. (5): an error component is multiplied every iteration by
S (S + lam T)^-1 in harmonic space and by Nbar (Nbar + lam T)^-1 in pixel
space, so convergence is slowest "for modes with high prior variance in high
noise pixels".  With T = tau 1 and tau the smallest noise variance, the pixel
factor at lam = 1 is 1 - tau/N_i: 1 where masked and 1 - 1e-4 in the noisiest
observed pixels of a map whose noise spans four decades.

These tests build the lam = 1 iteration matrix of the HEALPix iteration
densely from scipy's Y_lm (independently of the oracle's transforms),
  It = diag(S / (S + tau Omega)) Omega Y^T diag(1 - tau nu) Y,
and check that
  * the oracle's residual trace is the one the eigen-decomposition of It
    predicts from the iterate at the start of the lam = 1 phase (so the
    iteration counts to 1e-4 .. 1e-6 are predicted, not just observed);
  * the slowest eigenvectors are large-scale modes with high S/tau_h living
    in the masked and high-noise pixels, as Eq. (5) says;
  * the slow rate is not an artefact of the HEALPix quadrature (Omega Y^T Y
    != I): with an exact inverse of the synthesis in place of Omega Y^T the
    slowest rate changes by a factor that shrinks towards 1 with nside;
  * the final decade of the oracle's run takes ln(10) / (1 - rho) iterations
    to within 25 %;
  * 1 - rho falls as nside grows with the recipe fixed (nside 8 -> 16), i.e.
    the tail lengthens at higher resolution.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import wf_inputs as gen

RECIPE = dict(fwhm_arcmin=5.0, b_cut_deg=15.0, n_disks=3000, disk_radius_deg=0.3, noise_range=1e4)


def _dense_real_basis(oracle, nside, lmax):
    """Real synthesis matrix from scipy's Y_lm at the pixel centres, columns
    x = (Re a_l0; Re a_lm, Im a_lm for m > 0), their weights (1 or 2) and l."""
    th, ph = oracle.pixel_angles(nside)
    l, m = oracle.alm_lm(lmax)
    cols, wts, modes, ells = [], [], [], []
    for k in range(l.size):
        Y = sp.sph_harm_y(int(l[k]), int(m[k]), th, ph)
        if m[k] == 0:
            cols.append(Y.real)
            wts.append(1.0)
            modes.append((k, 0))
            ells.append(l[k])
        else:
            cols += [2 * Y.real, -2 * Y.imag]
            wts += [2.0, 2.0]
            modes += [(k, 0), (k, 1)]
            ells += [l[k], l[k]]
    return np.array(cols).T, np.array(wts), modes, np.array(ells)


class Dense:
    """lam = 1 iteration of one problem in real coordinates, and its
    symmetrised eigen-decomposition: It = Z^2 K with Z = (D / W)^1/2 and K =
    Omega Y^T diag(1 - q) Y symmetric, so It = Z U diag(mu) U^T Z^-1."""

    def __init__(self, oracle, nside):
        self.nside, self.lmax = nside, 2 * nside
        P = gen.healpix_problem(nside, self.lmax, gen.seed_for(3, 0), **RECIPE)
        basis = oracle.HealpixBasis(nside, self.lmax)
        self.basis, self.P = basis, P
        self.d = basis.synth(P["a_signal"]) + P["noise"]
        obs = P["mask"] > 0
        self.obs = obs
        self.nu = np.where(obs, 1.0 / P["noise_var"], 0.0)
        self.tau = float(P["noise_var"][obs].min())
        self.q = self.tau * self.nu
        om = basis.omega
        self.tau_h = self.tau * om
        self.S = basis.per_mode(P["c_ell"])
        Y, W, modes, ells = _dense_real_basis(oracle, nside, self.lmax)
        Sx = np.array([self.S[k] for k, _ in modes])
        act = Sx > 0
        self.modes, self.act = modes, act
        self.Y, self.W, self.Sx, self.ells = Y[:, act], W[act], Sx[act], ells[act]
        self.D = self.Sx / (self.Sx + self.tau_h)
        K = om * (self.Y.T @ ((1.0 - self.q)[:, None] * self.Y))
        self.Z = np.sqrt(self.D / self.W)
        mu, U = np.linalg.eigh(self.Z[:, None] * K * self.Z[None, :])
        o = np.argsort(-mu)
        self.mu, self.U = mu[o], U[:, o]
        self.rhs = (self.Y.T @ (self.nu * self.d)) / self.W  # Y^T r in x coordinates (weighted adjoint)
        self.bnorm = math.sqrt(np.sum(self.W * self.rhs ** 2))
        self.rweight = 1.0 / self.Sx + 1.0 / self.tau_h

    def x(self, a):
        return np.array([a[k].real if p == 0 else a[k].imag for k, p in self.modes])[self.act]

    def predicted_residuals(self, x0, ks):
        """Relative residuals |(1/S + 1/tau_h)(x_k - x_{k+1})| / |b| of the
        iterates k steps after x0 (x_{k+1} = It x_k + c)."""
        c = self.D * self.basis.omega * (self.Y.T @ (self.tau * self.nu * self.d)) / self.W
        x1 = self.Z * (self.U @ (self.mu * (self.U.T @ (x0 / self.Z)))) + c
        diff0 = (x0 - x1) / self.Z  # x_k - x_{k+1} evolves with It as well
        coef = self.U.T @ diff0
        out = []
        for k in ks:
            dk = self.Z * (self.U @ (self.mu ** k * coef))
            out.append(math.sqrt(np.sum(self.W * (self.rweight * dk) ** 2)) / self.bnorm)
        return np.array(out)


@pytest.fixture(scope="module")
def dense8(oracle):
    return Dense(oracle, 8)


def _heuristic_run(oracle, D, tol=1e-6):
    xs = {}
    sched = oracle.messenger.HealpixSchedule(D.P["c_ell"], D.tau_h, D.lmax)
    res = oracle.messenger_solve(D.basis, D.nu * D.d, D.nu, D.S, D.tau, schedule=sched, tol=tol, maxiter=100000,
                                 callback=lambda k, a: xs.__setitem__(k, D.x(a)))
    return res, xs


def test_residual_tail_is_predicted_by_the_dense_iteration_matrix(oracle, dense8):
    D = dense8
    res, xs = _heuristic_run(oracle, D)
    assert res["converged"]
    lam = np.array([t[0] for t in res["trace"]])
    L = np.array([t[1] for t in res["trace"]])
    k0 = int(np.nonzero((lam == 1.0) & (L == D.lmax))[0][0])  # first lam = 1, full-band iteration
    x0 = xs[k0] if k0 > 0 else np.zeros(D.act.sum())
    r = res["resid"]
    for tol in (1e-4, 1e-5, 1e-6):
        k_or = int(np.nonzero(r < tol)[0][0])
        ks = np.arange(k_or - k0 - 3, min(k_or - k0 + 4, r.size - k0))
        pred = D.predicted_residuals(x0, ks)
        np.testing.assert_allclose(pred, r[k0 + ks], rtol=1e-6)
        # the predicted crossing is the oracle's
        assert k0 + ks[np.nonzero(pred < tol)[0][0]] == k_or


def test_slowest_modes_are_high_prior_modes_in_masked_and_noisy_pixels(dense8):
    """Eq. (5): slowest for high prior variance in high-noise pixels."""
    D = dense8
    assert 0.0 < D.mu[0] < 1.0
    for j in range(3):
        v = D.Z * D.U[:, j]
        f2 = (D.Y @ v) ** 2
        in_slow_pixels = f2[(~D.obs) | (D.q < 1e-2)].sum() / f2.sum()
        w = D.W * v ** 2
        mean_l = np.sum(w * D.ells) / w.sum()
        snr = np.sum(w * D.Sx / D.tau_h) / w.sum()
        assert in_slow_pixels > 0.95
        assert mean_l < 5.0
        assert snr > 100.0
        # the rate is the mode's own mix of tau_h / S and tau / N (first order in both)
        est = np.sum(w * D.tau_h / D.Sx) / w.sum() + float(np.sum(f2 * D.q) / f2.sum())
        assert 0.5 < est / (1.0 - D.mu[j]) < 2.0


def _exact_analysis_rate(D):
    """Slowest rate of the lam = 1 iteration with an exact inverse of the
    synthesis on the band-limited space (least squares, G^-1 Omega Y^T with
    G = Omega Y^T Y) in place of the analysis Omega Y^T: the iteration
    D G^-1 Omega Y^T diag(1 - q) Y, whose fixed point is the exact normal
    equations."""
    om = D.basis.omega
    Yt = (D.Y / D.W[None, :]).T  # weighted adjoint in x coordinates
    G = om * (Yt @ D.Y)
    Kp = om * (Yt @ ((1.0 - D.q)[:, None] * D.Y))
    mu = np.linalg.eigvals(D.D[:, None] * np.linalg.solve(G, Kp))
    assert float(np.max(np.abs(mu.imag))) < 1e-8
    g = np.linalg.eigvals(G).real
    return 1.0 - float(np.max(mu.real)), float(g.max() - g.min())


@pytest.fixture(scope="module")
def dense16(oracle):
    return Dense(oracle, 16)


def test_slow_rate_is_not_a_quadrature_effect(dense8, dense16):
    """The HEALPix quadrature (Omega Y^T Y != I at lmax = 2 nside) slows the
    slowest mode by a factor that shrinks towards 1 with resolution (1.4 at
    nside 8, 1.14 at nside 16): it does not cause the long tail."""
    ratios = []
    for D in (dense8, dense16):
        rate_exact, spread = _exact_analysis_rate(D)
        assert spread > 0.05  # the quadrature is visibly inexact ...
        ratios.append(rate_exact / (1.0 - D.mu[0]))
    assert 1.0 <= ratios[0] < 1.6 and 1.0 <= ratios[1] < 1.25 and ratios[1] < ratios[0]


def test_last_decade_takes_ln10_over_one_minus_rho(oracle, dense8):
    D = dense8
    res, _ = _heuristic_run(oracle, D)
    r = res["resid"]
    k5, k6 = int(np.nonzero(r < 1e-5)[0][0]), int(np.nonzero(r < 1e-6)[0][0])
    assert abs((k6 - k5) / (math.log(10.0) / (1.0 - D.mu[0])) - 1.0) < 0.25


def test_tail_lengthens_with_resolution(dense8, dense16):
    assert (1.0 - dense16.mu[0]) < 0.7 * (1.0 - dense8.mu[0])
