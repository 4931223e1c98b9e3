"""Polarised messenger iteration (Eqs. 10-11): the oracle's statement.

TEST INFRASTRUCTURE (see the package docstring).  Maps are (I, Q, U) per
pixel, harmonic coefficients (T, E, B) per mode; the noise is a symmetric
positive definite 3x3 block per pixel on its observed components (inverse
nu = N^-1 there, zero rows and columns for masked components, see
pol_inverse_noise), the prior a 3x3 block per l,

    S_l = [[TT, TE, 0], [TE, EE, 0], [0, 0, BB]],

applied with its pseudo-inverse where it is singular (l < 2, BB = 0).  With
T = tau 1 and tau the smallest eigenvalue of any observed N_p, one
iteration at cooling parameter lambda is

    t_p   = s_p + lambda tau (1 + (lambda - 1) tau nu_p)^-1 (r_p - nu_p s_p)    (Eq. 10)
    a_lm  = S_l (S_l + lambda tau_h 1)^-1 Omega Y^T t                           (Eq. 11)

(the 3x3 form of Eqs. 3-4 solved for t, with r = nu d), tau_h = tau Omega.
chi^2 (Eq. 6, x-independent part dropped) and the residual at lambda = 1,
|(S^+ + 1/tau_h)(a_k - a_{k+1})| / |P Y^T r| (P the projector on the range of
S), follow the temperature case; the cooling uses the largest eigenvalue of
S_l in place of C_l.
"""
import numpy as np

from . import adjoint_pol, adjoint_synthesis, alm_lm, npix, synthesis, synthesis_pol
from .messenger import HealpixSchedule


class HealpixPolBasis:
    """(I, Q, U) maps on the HEALPix RING grid, (T, E, B) harmonic vectors of
    shape (3, n_alm); m = 0 counts once in norms, m > 0 twice."""

    kind = "healpix_pol"

    def __init__(self, nside: int, lmax: int):
        self.nside, self.lmax = nside, lmax
        self.omega = 4.0 * np.pi / npix(nside)
        self.ell, self.m = alm_lm(lmax)
        self.w = np.where(self.m == 0, 1.0, 2.0)

    def synth(self, a, L=None):
        L = self.lmax if L is None else L
        I = synthesis(self.nside, self.lmax, L, a[0])
        Q, U = synthesis_pol(self.nside, self.lmax, L, a[1], a[2])
        return np.stack([I, Q, U])

    def adjoint(self, t, L=None):
        L = self.lmax if L is None else L
        T = adjoint_synthesis(self.nside, self.lmax, L, t[0])
        E, B = adjoint_pol(self.nside, self.lmax, L, t[1], t[2])
        return np.stack([T, E, B])

    def band(self, L):
        return self.ell <= L

    def per_mode(self, cl):
        """(n_alm, 3, 3) prior blocks from C_l columns (TT, EE, BB, TE)."""
        cl = np.asarray(cl, dtype=np.float64)
        S = np.zeros((self.ell.size, 3, 3))
        S[:, 0, 0] = cl[self.ell, 0]
        S[:, 1, 1] = cl[self.ell, 1]
        S[:, 2, 2] = cl[self.ell, 2]
        S[:, 0, 1] = S[:, 1, 0] = cl[self.ell, 3]
        return S


def _apply(Mb, v):
    """Per-mode / per-pixel 3x3 blocks (n, 3, 3) times vectors (3, n)."""
    return np.einsum("nij,jn->in", Mb, v)


def sym_pinv(S):
    """Pseudo-inverse of symmetric PSD blocks (n, 3, 3) and the projector on their range."""
    w, V = np.linalg.eigh(S)
    big = w > 1e-300 * np.maximum(1.0, np.max(np.abs(w), axis=1, keepdims=True))
    inv = np.where(big, 1.0 / np.where(big, w, 1.0), 0.0)
    Sp = np.einsum("nij,nj,nkj->nik", V, inv, V)
    P = np.einsum("nij,nj,nkj->nik", V, big.astype(float), V)
    return Sp, P


def sym_sqrt(M, inverse=False):
    """Square root (or pseudo-inverse square root) of symmetric PSD blocks."""
    w, V = np.linalg.eigh(M)
    w = np.maximum(w, 0.0)
    if inverse:
        big = w > 0
        f = np.where(big, 1.0 / np.sqrt(np.where(big, w, 1.0)), 0.0)
    else:
        f = np.sqrt(w)
    return np.einsum("nij,nj,nkj->nik", V, f, V)


def observed_components(mask):
    """(npix, 3) booleans: which of I, Q, U each pixel observes.  ``mask`` is
    either booleans (all three or none) or the codes 0 (none), 1 (I, Q, U),
    2 (I only: polarisation masked) and 3 (Q, U only: temperature masked)."""
    m = np.asarray(mask)
    if m.dtype == bool:
        return np.repeat(m[:, None], 3, axis=1)
    out = np.zeros((m.size, 3), dtype=bool)
    out[m == 1] = True
    out[m == 2, 0] = True
    out[m == 3, 1:] = True
    return out


def _patterns(comp):
    for pattern in np.unique(comp, axis=0):
        K = np.nonzero(pattern)[0]
        if K.size:
            yield np.all(comp == pattern, axis=1), K


def pol_inverse_noise(N, mask):
    """nu per pixel: the inverse of the noise block restricted to the observed
    components, zero in the rows and columns of the others -- the limit of
    N^-1 as the variance of an unobserved component goes to infinity (the
    masked pixels of Sect. 2.1, N^-1 = 0, component by component)."""
    comp = observed_components(mask)
    nu = np.zeros_like(N)
    for sel, K in _patterns(comp):
        idx = np.nonzero(sel)[0]
        sub = N[np.ix_(idx, K, K)]
        nu[np.ix_(idx, K, K)] = np.linalg.inv(sub)
    return nu


def pol_tau(N, obs):
    """tau = smallest eigenvalue of the noise blocks over the observed
    components (the observed sub-block of each pixel), so that N - tau stays
    positive semi-definite where there is data."""
    comp = observed_components(obs)
    return float(min(np.linalg.eigvalsh(N[np.ix_(np.nonzero(sel)[0], K, K)]).min() for sel, K in _patterns(comp)))


def fluct_source_pol(basis, nu, S, g1, g2):
    """Source of Eq. (9) for polarisation: r = nu^1/2 g1 + Omega Y (S^+1/2 g2)."""
    z = basis.omega * basis.synth(_apply(sym_sqrt(S, inverse=True), g2))
    return _apply(sym_sqrt(nu), g1) + z


def messenger_solve_pol(basis, r, nu, S, tau, *, tol=1e-6, maxiter=20000, replay=None, eta=1e-2, level_cap=200,
                        callback=None):
    """Polarised messenger iteration from a = 0 (heuristic cooling of Sect. 3
    on the largest eigenvalue of S_l, or a replay of (lam, L) pairs).

    r (3, npix), nu (npix, 3, 3), S (n_alm, 3, 3).  Returns a dict like
    messenger_solve: a (3, n_alm), s (3, npix), trace, chi2, resid, iters,
    converged, n_dof, bnorm.
    """
    lmax = basis.lmax
    omega = basis.omega
    tau_h = tau * omega
    Sp, Pr = sym_pinv(S)
    w = basis.w
    b = basis.adjoint(r, lmax)
    bnorm = float(np.sqrt(np.sum(w * np.sum(np.abs(_apply(Pr, b)) ** 2, axis=0))))
    n_dof = int(np.count_nonzero(np.diagonal(nu, axis1=1, axis2=2) > 0.0))  # observed components
    sigma = float(np.sqrt(2.0 * n_dof))
    schedule = None
    if replay is None:
        lam_ell = np.zeros(lmax + 1)
        for l in range(lmax + 1):
            k = np.nonzero(basis.ell == l)[0][0]
            lam_ell[l] = np.linalg.eigvalsh(S[k]).max()
        schedule = HealpixSchedule(lam_ell, tau_h, lmax)
    a = np.zeros((3, basis.ell.size), dtype=np.complex128)
    eye = np.eye(3)
    trace, chi2s, resids = [], [], []
    converged = False
    prev = None
    level_iters = 0
    k = 0
    while True:
        if replay is not None:
            if k >= len(replay):
                break
            lam, L = replay[k]
            L = int(L)
        else:
            if k >= maxiter:
                break
            lam, L = schedule.lam, schedule.L
        full = L == lmax
        s = basis.synth(a, L)
        # Eq. (10), per pixel: t = s + lam tau (1 + (lam-1) tau nu)^-1 (r - nu s)
        Minv = np.linalg.inv(eye[None] + (lam - 1.0) * tau * nu)  # (npix, 3, 3)
        t = s + lam * tau * _apply(Minv, r - _apply(nu, s))
        # Eq. (11), per mode: a = S (S + lam tau_h)^-1 Omega Y^T t
        that = omega * basis.adjoint(t, L)
        F = S @ np.linalg.inv(S + lam * tau_h * eye[None])
        a_new = np.where(basis.band(L)[None, :], _apply(F, that), 0.0)
        # chi^2 of the iterate (Eq. 6, x-independent part dropped)
        Mnu = Minv @ nu
        chi2 = float(np.sum(w * np.einsum("in,nij,jn->n", np.conj(a), Sp, a).real)
                     + np.sum(np.einsum("in,nij,jn->n", s, Mnu, s) - 2.0 * np.einsum("in,nij,jn->n", r, Minv, s)))
        resid = np.nan
        if lam == 1.0 and full:
            dv = _apply(Sp + eye[None] / tau_h, a - a_new)
            resid = float(np.sqrt(np.sum(w * np.sum(np.abs(dv) ** 2, axis=0)))) / bnorm
        trace.append((float(lam), int(L)))
        chi2s.append(chi2)
        resids.append(resid)
        a = a_new
        k += 1
        if callback is not None:
            callback(k, a)
        if replay is not None:
            if lam == 1.0 and full and resid < tol:
                converged = True
            continue
        if schedule.final:
            if resid < tol:
                converged = True
                break
        else:
            level_iters += 1
            plateau = prev is not None and abs(chi2 - prev) < eta * sigma
            if plateau or level_iters >= level_cap:
                schedule.advance()
                prev = None
                level_iters = 0
                continue
        prev = chi2
    return {"a": a, "s": basis.synth(a, lmax), "trace": trace, "chi2": np.array(chi2s), "resid": np.array(resids),
            "iters": k, "converged": converged, "n_dof": n_dof, "bnorm": bnorm}
