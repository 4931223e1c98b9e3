"""The algebra behind the correction form of the mixed iteration, on the
oracle (FP64, small HEALPix maps; no GPU).

At lambda = 1 on the full band the messenger step (Eqs. 3-4) is affine,
G(a) = B a + c: the pixel blend of Eq. (3) and the harmonic blend of Eq. (4)
are linear in a, and the source enters additively.  Iterating
delta <- d0 + B delta from delta_0 = d0 = G(x0) - x0 therefore reproduces the
plain iterates, a_{j+1} = x0 + delta_j, with the same steps.  When every
application of the step carries a rounding error relative to its operand (a
model of the FP32 kernels), the residual the correction form computes is off
by an amount that scales with |delta| instead of |a|."""
import numpy as np
import pytest

import oracle
import wf_inputs as gen
from oracle.messenger import wnorm

NSIDE, LMAX = 8, 16


@pytest.fixture(scope="module")
def case():
    P = gen.healpix_problem(NSIDE, LMAX, gen.seed_for(3, 90), fwhm_arcmin=4 * 3438.0 / LMAX, n_disks=4,
                            disk_radius_deg=8.0)
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
    inv_S = np.where(active, 1.0 / np.where(active, S, 1.0), 0.0)
    bnorm = wnorm(basis.w, basis.adjoint(r, LMAX), active)

    def resid(v):
        # the lambda = 1 residual of a step a -> a - v (Eq. 2 at the fixed point)
        return wnorm(basis.w, (inv_S + 1.0 / (tau * basis.omega)) * v, active) / bnorm

    a = np.zeros(S.shape, dtype=np.complex128)
    for _ in range(30):
        a = G(a)
    return G, resid, active, a


def test_the_lambda_one_step_is_affine(case):
    """G(alpha x + (1 - alpha) y) = alpha G(x) + (1 - alpha) G(y), inside and
    outside [0, 1]: what lets B delta = G(delta) - G(0) stand for the step
    with its source set to zero."""
    G, _, _, x0 = case
    x1 = x0.copy()
    for _ in range(20):
        x1 = G(x1)
    for alpha in (0.5, 3.0, -2.0):
        lhs = G(alpha * x1 + (1.0 - alpha) * x0)
        rhs = alpha * G(x1) + (1.0 - alpha) * G(x0)
        assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(lhs).max(), alpha


def test_correction_iterates_are_the_plain_iterates(case):
    """delta_0 = d0 = G(x0) - x0, delta_{j+1} = d0 + B delta_j gives
    x0 + delta_j = a_{j+1} and delta_j - delta_{j+1} = a_{j+1} - a_{j+2}: the
    same iterates and the same residuals."""
    G, resid, _, x0 = case
    G0 = G(np.zeros_like(x0))

    def B(v):
        return G(v) - G0

    plain = [x0]
    for _ in range(12):
        plain.append(G(plain[-1]))
    d0 = G(x0) - x0
    delta = [d0]
    for _ in range(10):
        delta.append(d0 + B(delta[-1]))
    scale = np.abs(x0).max()
    for j in range(10):
        assert np.abs(x0 + delta[j] - plain[j + 1]).max() <= 1e-12 * scale, j
        step_c = delta[j] - delta[j + 1]
        step_p = plain[j + 1] - plain[j + 2]
        assert resid(step_c) == pytest.approx(resid(step_p), rel=1e-8), j


def test_rounding_of_the_correction_scales_with_delta(case):
    """Each application perturbed by 1e-6 of its operand's RMS (a model of
    FP32 rounding): the residual computed from the plain noisy iterates is
    off by far more than the one the correction form computes, whose
    operand delta is a few percent of a."""
    G, resid, active, x0 = case
    G0 = G(np.zeros_like(x0))
    rng = np.random.default_rng(12104931)

    def noisy(f, v):
        out = f(v)
        rms = np.sqrt(np.mean(np.abs(v[active]) ** 2))
        return out + 1e-6 * rms * (rng.standard_normal(out.shape) + 1j * rng.standard_normal(out.shape)) * active

    err_plain, err_corr = [], []
    a = x0.copy()
    for _ in range(40):
        a_new = noisy(G, a)
        err_plain.append(abs(resid(a - a_new) - resid(a - G(a))) / resid(a - G(a)))
        a = a_new
    d0 = G(x0) - x0
    delta = d0.copy()
    ratio = []
    for _ in range(40):
        delta_new = d0 + noisy(lambda v: G(v) - G0, delta)
        x = x0 + delta
        err_corr.append(abs(resid(delta - delta_new) - resid(x - G(x))) / resid(x - G(x)))
        ratio.append(np.sqrt(np.mean(np.abs(delta[active]) ** 2) / np.mean(np.abs(x[active]) ** 2)))
        delta = delta_new
    print("median relative error of the residual: plain %.2e, correction %.2e, |delta|/|a| %.3f"
          % (np.median(err_plain), np.median(err_corr), ratio[-1]))
    assert max(ratio) < 0.2
    assert np.median(err_corr) < 0.1 * np.median(err_plain)
