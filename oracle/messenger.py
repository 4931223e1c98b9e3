"""Messenger-field iteration, cooling schedules and fluctuation source.

TEST INFRASTRUCTURE (part of the oracle; see ``oracle/__init__.py``).

Paper passages followed, in order of use:

* Eq. (3), pixel-space blend: (Nbar^-1 + (lam T)^-1) t = Nbar^-1 d + (lam T)^-1 s
  with T = tau 1, tau = min diag(N), Nbar = N - T (Sect. 2.1).  Written per
  pixel with nu = N^-1 (0 where masked) and the source r = nu d:
      t = s + lam tau (r - nu s) / (1 + (lam - 1) tau nu).
  This is Eq. (3) solved for t, multiplied through by Nbar; it has no
  division by zero for lam >= 1 and gives t = s in masked pixels.
* Eq. (4), harmonic-space blend: (S^-1 + (lam T)^-1) s = (lam T)^-1 t, i.e.
  a = S / (S + lam tau_h) * (Omega Y^T t), tau_h = tau Omega being T seen
  per harmonic mode (Omega = 1 on the flat grid, 4 pi / n_pix on HEALPix).
* Eq. (6), chi^2(x, lam) = x^T S^-1 x + (d - x)^T [N + (lam - 1) T]^-1 (d - x);
  evaluated here without its x-independent part, as
      sum_modes w |a|^2 / S + sum_pix (nu s^2 - 2 r s) / (1 + (lam - 1) tau nu),
  which is what the iteration minimises for any source r.
* Stopping residual at lam = 1 (derived from Eqs. (3)-(4)): with b = Y^T r,
      ||(1/S + 1/tau_h)(a_k - a_{k+1})|| / ||b||
  equals ||M a_k - b|| / ||b|| for the fixed-point operator M of the
  iteration.  On the flat grid M = S^-1 + N^-1 in harmonic coordinates, so
  this is the relative residual of Eq. (2).
* Cooling schedule, Sect. 3: lam from the ratio of S at l_iter = 20 to T
  (read as S_l / tau_h, since lam >= 1 and cooling starts high), l_iter
  doubled on a chi^2 plateau with the increment capped at 500, lam >= 1,
  and the transforms band-limited to L = l_iter + 100 <= lmax.
* Fluctuation source, Eq. (9): Nbar^-1 d -> Nbar^-1 N (N^-1/2 g1 + S^-1/2 g2),
  identity in masked pixels; in the r form above this is
  r = nu^1/2 g1 + Omega Y (S^-1/2 g2).

Readings where the paper is silent: the
plateau test |chi2_k - chi2_{k-1}| < eta sigma_chi2 with eta = 1e-2 and
sigma_chi2 = sqrt(2 n_dof); a cap of ``level_cap`` iterations per level; on
the flat grid the levels are k_iter = 1, 2, 4, ... with
lam = clip(S(k_iter) / tau, 1, lam_max) and the first level at lam_max.
"""
import numpy as np


def wnorm(w, v, sel):
    """Weighted Euclidean norm sqrt(sum w |v|^2) over the modes in ``sel``."""
    return float(np.sqrt(np.sum(np.where(sel, w * np.abs(v) ** 2, 0.0))))


class HealpixSchedule:
    """Heuristic cooling of Sect. 3 on the sphere."""

    def __init__(self, c_ell, tau_h, lmax, ell0=20, max_increment=500, margin=100):
        self.c = np.asarray(c_ell, dtype=np.float64)
        self.tau_h = float(tau_h)
        self.lmax = int(lmax)
        self.ell_iter = min(int(ell0), self.lmax)
        self.max_increment = max_increment
        self.margin = margin
        self.lam, self.L = self._level()

    def _level(self):
        if self.ell_iter >= self.lmax:
            return 1.0, self.lmax
        lam = max(1.0, self.c[self.ell_iter] / self.tau_h)
        return lam, min(self.lmax, self.ell_iter + self.margin)

    @property
    def final(self):
        return self.lam == 1.0 and self.L == self.lmax

    def advance(self):
        lam0, L0 = self.lam, self.L
        while True:
            self.ell_iter = min(2 * self.ell_iter, self.ell_iter + self.max_increment)
            self.lam, self.L = self._level()
            if (self.lam, self.L) != (lam0, L0) or self.final:
                return


class FlatSchedule:
    """Cooling on the flat grid: k_iter = 1, 2, 4, ...; lam from the prior
    variance at |k| = k_iter (largest over the modes on that radius) over tau,
    clipped to [1, lam_max]; the first level sits at lam_max."""

    def __init__(self, S, kabs, tau, lam_max=100.0):
        self.S = np.asarray(S)
        self.kr = np.rint(np.asarray(kabs)).astype(np.int64)
        self.tau = float(tau)
        self.lam_max = float(lam_max)
        self.k_iter = 1
        self.lam = self.lam_max
        self.L = None

    def _lam(self, k):
        sel = self.kr == k
        if not np.any(sel):
            return 1.0
        return float(np.clip(self.S[sel].max() / self.tau, 1.0, self.lam_max))

    @property
    def final(self):
        return self.lam == 1.0

    def advance(self):
        lam0 = self.lam
        while True:
            self.k_iter *= 2
            self.lam = self._lam(self.k_iter) if self.k_iter <= self.kr.max() else 1.0
            if self.lam != lam0 or self.final:
                return


class RigorousSchedule:
    """Cooling that keeps the chi^2 bound (Sect. 2.2): with b = n_dof -
    m sigma_chi2, lambda starts where chi^2(lambda, 0) = d^T (N + (lambda-1)
    T)^-1 d = b; after every iteration lambda is lowered until chi^2(lambda,
    x) = b again; when lambda stops falling (x has converged to s(lambda) at
    lambda > 1) b is raised to b' = chi2_min(lambda) + (lambda - 1) tau x^T
    S^-2 x, the first-order estimate of chi2_min(1) from below; lambda = 1
    is taken once lambda - 1 < lam_floor.  Written with u = (lambda - 1) tau:
    chi^2(u, x) = x^T S^-1 x + sum (d - x)^2 / (N + u) over observed pixels.
    Readings (the paper gives none): m = 5, "stops falling" = relative change
    of lambda - 1 below stall_tol over one iteration."""

    def __init__(self, n_dof, m_sigma=5.0, stall_tol=1e-7, lam_floor=1e-9):
        self.b = n_dof - m_sigma * np.sqrt(2.0 * n_dof)
        self.stall_tol = stall_tol
        self.lam_floor = lam_floor
        self.u = None
        self.b_updates = 0

    @staticmethod
    def _root(f, hi):
        """Largest-accuracy root of the decreasing function f on [0, hi]
        (returns 0 when f(0) <= 0)."""
        from scipy.optimize import brentq

        if f(0.0) <= 0.0:
            return 0.0
        if f(hi) >= 0.0:
            return hi
        return brentq(f, 0.0, hi, xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)

    def lam(self, tau):
        return 1.0 + self.u / tau


def fluct_source(basis, nu, S, g1, g2):
    """Pixel source of Eq. (9): r = nu^1/2 g1 + Omega Y (S^-1/2 g2); modes
    with S = 0 get no draw (pseudo-inverse)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        isq = np.where(S > 0, 1.0 / np.sqrt(np.where(S > 0, S, 1.0)), 0.0)
    z = basis.omega * basis.synth(isq * g2, basis.lmax)
    return np.sqrt(nu) * g1 + z


def messenger_solve(basis, r, nu, S, tau, *, tol=1e-6, maxiter=20000,
                    replay=None, schedule=None, eta=1e-2, level_cap=200, d=None,
                    callback=None, a0=None):
    """Run the messenger iteration (Eqs. 3-4) from a = 0.

    basis   FlatBasis or HealpixBasis
    r, nu   pixel source (nu d for the Wiener filter) and inverse noise
            variance (0 where masked)
    S       prior variance per stored harmonic mode (0: mode held at zero)
    tau     min noise variance over unmasked pixels
    replay  optional list of (lam, L) pairs: run exactly these iterations
    schedule  FlatSchedule / HealpixSchedule (built from S if omitted)
    callback  optional f(k, a_new) called after every iteration
    a0        optional starting harmonic vector (default: zeros, as in Sect. 2.1)
    Leading batch axes on r / nu are allowed on the flat grid (norms and
    chi^2 are then summed over the batch).

    Returns a dict with the final harmonic vector ``a``, its map ``s``, the
    (lam, L) trace, chi^2 and residual per iteration, and whether the
    residual fell below ``tol`` at lam = 1 on the full band.
    """
    full_L = basis.lmax
    omega = basis.omega
    tau_h = tau * omega
    active = S > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        inv_S = np.where(active, 1.0 / np.where(active, S, 1.0), 0.0)
    b = basis.adjoint(r, full_L)
    bnorm = wnorm(basis.w, b, active)
    n_dof = int(np.count_nonzero(nu > 0))
    sigma = float(np.sqrt(2.0 * n_dof))

    rigorous = isinstance(schedule, RigorousSchedule)
    if rigorous and d is None:
        raise ValueError("the chi^2-bound schedule needs the data d")
    if replay is None and schedule is None:
        if basis.kind == "flat":
            schedule = FlatSchedule(S, basis.kabs(), tau)
        else:
            raise ValueError("a HealpixSchedule (built from C_ell) is required")

    a = np.zeros(b.shape, dtype=np.complex128) if a0 is None else np.array(a0, dtype=np.complex128)
    trace, chi2s, resids, bounds = [], [], [], []
    converged = False
    prev_chi2 = None
    level_iters = 0
    k = 0
    while True:
        if replay is not None:
            if k >= len(replay):
                break
            lam, L = replay[k]
            L = None if L is None or basis.kind == "flat" else int(L)
        elif rigorous:
            if k >= maxiter:
                break
            L = full_L
            s = basis.synth(a, full_L)
            obs = nu > 0
            e2 = np.where(obs, (d - s) ** 2, 0.0)
            N = np.where(obs, 1.0 / np.where(obs, nu, 1.0), 1.0)
            h = float(np.sum(basis.w * np.abs(a) ** 2 * inv_S))

            def g(u):
                return h + float(np.sum(np.where(obs, e2 / (N + u), 0.0))) - schedule.b

            if schedule.u is None:  # initial lambda: chi^2(lambda, 0) = b
                hi = 1.0
                while g(hi) > 0.0 and hi < 1e300:
                    hi *= 4.0
                schedule.u = schedule._root(g, hi)
            else:
                u_prev = schedule.u
                u_new = schedule._root(g, u_prev) if u_prev > 0.0 else 0.0
                if u_new > 0.0 and (u_prev - u_new) <= schedule.stall_tol * u_new:
                    # converged at lambda > 1: raise b towards chi2_min(1)
                    q = float(np.sum(basis.w * np.abs(a) ** 2 * inv_S ** 2))
                    schedule.b = (h + float(np.sum(np.where(obs, e2 / (N + u_new), 0.0)))) + u_new * omega * q
                    schedule.b_updates += 1
                    u_new = schedule._root(g, u_prev)
                schedule.u = u_new
            if schedule.u / tau < schedule.lam_floor:
                schedule.u = 0.0
            lam = schedule.lam(tau)
        else:
            if k >= maxiter:
                break
            lam, L = schedule.lam, schedule.L
        full = basis.kind == "flat" or L == full_L
        Lb = full_L if L is None else L

        # Eq. (3): pixel blend
        if not rigorous or replay is not None:
            s = basis.synth(a, Lb)
        den = 1.0 + (lam - 1.0) * tau * nu
        t = s + lam * tau * (r - nu * s) / den
        # Eq. (4): harmonic blend
        that = omega * basis.adjoint(t, Lb)
        filt = np.where(active & basis.band(Lb), S / (S + lam * tau_h), 0.0)
        a_new = filt * that
        # Eq. (6) at x = s (= Y a), x-independent part dropped
        chi2 = float(np.sum(basis.w * np.abs(a) ** 2 * inv_S) + np.sum((nu * s * s - 2.0 * r * s) / den))
        resid = np.nan
        if lam == 1.0 and full:
            resid = wnorm(basis.w, (inv_S + 1.0 / tau_h) * (a - a_new), active) / bnorm
        trace.append((float(lam), None if basis.kind == "flat" else int(Lb)))
        if rigorous and replay is None:
            bounds.append(schedule.b)
        chi2s.append(chi2)
        resids.append(resid)
        a = a_new
        k += 1
        if callback is not None:
            callback(k, a)

        if replay is None and rigorous:
            if lam == 1.0 and resid < tol:
                converged = True
                break
            continue
        if replay is None:
            if schedule.final:
                if resid < tol:
                    converged = True
                    break
            else:
                level_iters += 1
                plateau = prev_chi2 is not None and abs(chi2 - prev_chi2) < eta * sigma
                if plateau or level_iters >= level_cap:
                    schedule.advance()
                    prev_chi2 = None
                    level_iters = 0
                    continue
            prev_chi2 = chi2
        elif lam == 1.0 and full and resid < tol:
            converged = True

    out = {
        "a": a,
        "s": basis.synth(a, full_L),
        "trace": trace,
        "chi2": np.array(chi2s),
        "resid": np.array(resids),
        "iters": k,
        "converged": converged,
        "n_dof": n_dof,
        "bnorm": bnorm,
        "bound": np.array(bounds),
    }
    if d is not None:
        s = out["s"]
        out["chi2_final"] = float(np.sum(basis.w * np.abs(a) ** 2 * inv_S) + np.sum(nu * (d - s) ** 2))
    return out
