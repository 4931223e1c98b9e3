"""The lambda = 1 system behind the messenger iteration is symmetric positive
definite, so a Krylov method can take the place of its long tail (on the
oracle, CPU; the workload recipe of the nside-2048 map at nside 8 and 16).

At lambda = 1 the iteration is a <- G(a) = B a + c with B = F K, where
F = diag(S / (S + tau_h)) and K = Omega Y^T diag(1 - tau nu) Y is self-adjoint
in the quadrature inner product <u, v> = sum_modes w Re(conj(u) v).  Its fixed
point solves M a = F^-1 c with M = F^-1 (I - B) = F^-1 - K, self-adjoint and
positive definite, and the messenger iteration is Richardson's iteration on
that system preconditioned by F (a <- a + F (F^-1 c - M a) = G(a)).  Conjugate
gradients with the same preconditioner use the same one application of B per
step; here they reach the residuals of the paper's criterion in a small
fraction of the messenger iteration's steps.  Not part of the paper's method:
this pins the reading behind the next step listed for the solver."""
import math

import numpy as np
import pytest

import wf_inputs as gen
from oracle.messenger import wnorm

def recipe(nside):
    # the nside-2048 map's beam and disks scaled to the pixel size; noise range 1e4, |b| < 15 deg
    return dict(fwhm_arcmin=5.0 * 2048 / nside, b_cut_deg=15.0, n_disks=30, disk_radius_deg=0.3 * 2048 / nside / 4,
                noise_range=1e4)


def _make_system(oracle, NSIDE):
    LMAX = 2 * NSIDE
    P = gen.healpix_problem(NSIDE, LMAX, gen.seed_for(3, 5), **recipe(NSIDE))
    basis = oracle.HealpixBasis(NSIDE, LMAX)
    d = basis.synth(P["a_signal"]) + P["noise"]
    obs = P["mask"] > 0
    nu = np.where(obs, 1.0 / P["noise_var"], 0.0)
    tau = float(P["noise_var"][obs].min())
    S = basis.per_mode(P["c_ell"])
    r = nu * d

    def G(a):
        return oracle.messenger_solve(basis, r, nu, S, tau, replay=[(1.0, LMAX)], a0=a)["a"]

    active = S > 0
    tau_h = tau * basis.omega
    F = np.where(active, S / (S + tau_h), 0.0)
    Finv = np.where(active, (S + tau_h) / np.where(active, S, 1.0), 0.0)
    inv_S = np.where(active, 1.0 / np.where(active, S, 1.0), 0.0)
    bnorm = wnorm(basis.w, basis.adjoint(r, LMAX), active)
    c = G(np.zeros(S.shape, dtype=np.complex128))

    def M(a):
        return Finv * (a - (G(a) - c))

    def dot(u, v):
        return float(np.sum(basis.w * (np.conj(u) * v).real * active))

    def resid(a):
        # the relative residual the solver reports at lambda = 1 (one step from a)
        return wnorm(basis.w, (inv_S + 1.0 / tau_h) * (a - G(a)), active) / bnorm

    return dict(G=G, M=M, F=F, Finv=Finv, c=c, dot=dot, resid=resid, active=active, shape=S.shape, nside=NSIDE)


@pytest.fixture(scope="module", params=[8, 16])
def system(oracle, request):
    return _make_system(oracle, request.param)


@pytest.fixture(scope="module")
def system8(oracle):
    return _make_system(oracle, 8)


def _pcg(M, F, dot, rhs, steps, stop=None):
    """Conjugate gradients on M y = rhs preconditioned by F, from y = 0; stop(y, r)
    ends them early.  Returns y and the steps taken."""
    y = np.zeros_like(rhs)
    rv = rhs.copy()
    z = F * rv
    p = z.copy()
    rz = dot(rv, z)
    for k in range(1, steps + 1):
        Ap = M(p)
        alpha = rz / dot(p, Ap)
        y = y + alpha * p
        rv = rv - alpha * Ap
        z = F * rv
        rz_new = dot(rv, z)
        if stop is not None and stop(y, rz_new):
            return y, k
        p = z + (rz_new / rz) * p
        rz = rz_new
    return y, steps


def _random_alm(rng, shape, active):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * active


def test_the_lambda_one_system_is_self_adjoint_and_positive(system):
    M, dot, act = system["M"], system["dot"], system["active"]
    rng = np.random.default_rng(7)
    for _ in range(3):
        u, v = _random_alm(rng, system["shape"], act), _random_alm(rng, system["shape"], act)
        muv, mvu = dot(u, M(v)), dot(M(u), v)
        assert abs(muv - mvu) <= 1e-10 * math.sqrt(dot(u, M(u)) * dot(v, M(v)))
        assert dot(u, M(u)) > 0.0


def test_messenger_iteration_is_preconditioned_richardson(system):
    G, M, F, Finv, c = system["G"], system["M"], system["F"], system["Finv"], system["c"]
    rng = np.random.default_rng(8)
    a = _random_alm(rng, system["shape"], system["active"])
    rich = a + F * (Finv * c - M(a))
    assert np.abs(rich - G(a)).max() <= 1e-12 * np.abs(G(a)).max()


def test_conjugate_gradients_on_the_same_system_cut_the_tail(system):
    """From a = 0, preconditioned CG reaches the 1e-6 residual in far fewer
    steps than the messenger iteration needs for one decade of its tail, and
    lands on the messenger iteration's fixed point."""
    G, M, F, Finv, c, dot, resid = (system[k] for k in ("G", "M", "F", "Finv", "c", "dot", "resid"))
    b = Finv * c
    x = np.zeros(system["shape"], dtype=np.complex128)
    rv = b.copy()
    z = F * rv
    p = z.copy()
    rz = dot(rv, z)
    k_cg = None
    for k in range(1, 2001):
        Ap = M(p)
        alpha = rz / dot(p, Ap)
        x = x + alpha * p
        rv = rv - alpha * Ap
        if resid(x) < 1e-6:
            k_cg = k
            break
        z = F * rv
        rz_new = dot(rv, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    assert k_cg is not None
    # the messenger iteration from the same start: its residual after as many steps, and
    # the contraction of its last steps
    a = np.zeros(system["shape"], dtype=np.complex128)
    for _ in range(4 * k_cg):
        a = G(a)
    r_msg = resid(a)
    print("nside %d: CG reaches 1e-6 in %d steps; the messenger iteration is at %.2e after %d"
          % (system["nside"], k_cg, r_msg, 4 * k_cg))
    assert r_msg > 1e-4  # four times CG's steps leave the messenger iteration two decades short or more
    # the same fixed point: a few more messenger steps from CG's result keep it there
    y = x.copy()
    for _ in range(5):
        y = G(y)
    assert np.abs(y - x).max() <= 1e-5 * np.abs(x).max()


def test_cg_with_a_rounded_operator_needs_fp64_residuals(system8):
    """With each application of B perturbed by 1e-6 of its operand's RMS (the
    FP32 kernels' rounding, modelled), CG stalls far above 1e-6; restarted on
    the residual of the FP64 operator (iterative refinement: the correction
    form's idea applied to CG), it goes on to 1e-8 in a few restarts."""
    S8 = system8
    G, M, F, Finv, c, dot, resid, act = (S8[k] for k in ("G", "M", "F", "Finv", "c", "dot", "resid", "active"))
    G0 = c
    rng = np.random.default_rng(12104931)

    def M_rounded(v):
        Bv = G(v) - G0
        rms = np.sqrt(np.mean(np.abs(v[act]) ** 2))
        Bv = Bv + 1e-6 * rms * (rng.standard_normal(v.shape) + 1j * rng.standard_normal(v.shape)) * act
        return Finv * (v - Bv)

    b = Finv * c
    best = [1.0]

    def track(y, _):
        best[0] = min(best[0], resid(y))
        return False

    _pcg(M_rounded, F, dot, b, 400, stop=track)
    print("CG with the rounded operator: best residual %.2e in 400 steps" % best[0])
    assert best[0] > 1e-5
    x = np.zeros_like(b)
    restarts, total = 0, 0
    while resid(x) > 1e-8 and restarts < 6:
        restarts += 1
        r64 = b - M(x)  # the residual of the FP64 operator
        n0 = math.sqrt(dot(r64, F * r64))
        y, k = _pcg(M_rounded, F, dot, r64, 1000, stop=lambda y, rz: math.sqrt(rz) < 1e-3 * n0)
        x = x + y
        total += k
    print("refined CG: %d restarts, %d steps, residual %.2e" % (restarts, total, resid(x)))
    assert resid(x) <= 1e-8 and restarts <= 4
