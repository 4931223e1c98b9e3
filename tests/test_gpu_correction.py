"""Correction form of the mixed iteration (wf_options.mixed_correction).

The messenger iteration (Eqs. 3-4) is affine, a_{k+1} = B a_k + c.  After one
FP64 iteration from the iterate x0 the FP32 kernels iterate on delta = a - x0
(delta <- d0 + B delta, d0 = B x0 + c - x0), so their rounding scales with
|delta| instead of |a| and the residual they report is the FP64 operator's.
Checked against the oracle's FP64 operator: one lambda = 1 step of the oracle
from the returned a_lm."""
import numpy as np
import pytest

import oracle
import wf_inputs as gen
from gpu_util import T, healpix_case, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    import torch

    import paper_1210_4931_gb300 as w

    w.load()
    torch.cuda.set_device(0)
    return w


def _solve(wf, prec, nside, lmax, seed, tol, **opts):
    import torch

    P, basis, d, nu, tau = healpix_case(nside, lmax, seed)
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=prec)
    wf.wf_set_options(plan, **opts)
    s = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
    alm = torch.empty(plan.nalm, dtype=torch.complex128, device="cuda")
    rep = wf.wf_solve(plan, T(d), T(P["noise_var"]), T(P["mask"]), T(P["c_ell"]), tol, s, alm, trace_cap=20000)
    plan.close()
    a = alm.cpu().numpy()
    S = basis.per_mode(P["c_ell"])
    r1 = oracle.messenger_solve(basis, nu * d, nu, S, tau, replay=[(1.0, lmax)], a0=a)["resid"][0]
    return rep, a, s.cpu().numpy(), r1


@pytest.mark.parametrize("prec", ["mixed", "tf32"])
def test_correction_form_reports_the_fp64_operator_residual(wf, prec):
    """No FP64 sweeps at all: the residual the correction form reports at the
    end is the FP64 operator's, to the rounding of the correction.  One oracle
    FP64 step from the returned a_lm gives a residual within 3 % of the
    reported one (here the switch comes at the first full-band lambda = 1
    iteration, so delta carries the whole lambda = 1 phase, about 1500
    iterations; 3xTF32 transforms measured a ratio of 1.010, FP32 within 1.01).  The
    trace holds the switch's FP64 step at lambda = 1 on the full band, with
    chi^2 NaN from there on (the kernels see delta, not the iterate)."""
    nside, lmax, tol = 32, 64, 1e-5
    # a switch factor this large switches at the first full-band lambda = 1 iteration
    rep, a, s, r1 = _solve(wf, prec, nside, lmax, gen.seed_for(3, 54), tol, refine_sweeps=0,
                           mixed_correction=1e6)
    assert rep["converged"] and rep["final_residual"] < tol
    chi2 = rep["chi2_trace"]
    nan = np.flatnonzero(np.isnan(chi2))
    assert len(nan) > 0
    k0 = int(nan[0])
    assert np.all(np.isnan(chi2[k0:])) and np.all(np.isfinite(chi2[:k0]))
    assert rep["lambda_trace"][k0] == 1.0 and rep["L_trace"][k0] == lmax
    assert k0 == 0 or rep["lambda_trace"][k0 - 1] == 1.0  # the switch follows a full-band lambda = 1 iteration
    print(prec, "switch at", k0, "of", rep["iters"], "reported", rep["final_residual"], "fp64 operator", r1)
    assert r1 <= rep["final_residual"] * 1.03
    # the output map is the plan's (FP32) synthesis of the returned a_lm
    assert rel(s, oracle.synthesis(nside, lmax, lmax, a)) < 2e-5


@pytest.mark.parametrize("prec", ["mixed", "tf32"])
def test_correction_form_with_a_verifying_sweep(wf, prec):
    """The correction form followed by FP64 sweeps (their verdict is the
    report's): the FP32 phase may stop close to tol, and one sweep confirms it;
    the returned a_lm meets tol under the oracle's FP64 operator and its map is
    the FP64 synthesis (1e-10 of the oracle's)."""
    nside, lmax, tol = 32, 64, 1e-5
    rep, a, s, r1 = _solve(wf, prec, nside, lmax, gen.seed_for(3, 55), tol, refine_sweeps=4,
                           mixed_tol_factor=0.98, mixed_correction=100.0)
    assert rep["converged"] and rep["final_residual"] < tol
    assert 1 <= rep["refine_sweeps"] <= 4
    print(prec, "iters", rep["iters"], "sweeps", rep["refine_sweeps"], "fp64 operator", r1)
    assert r1 < tol
    assert rel(s, oracle.synthesis(nside, lmax, lmax, a)) < 1e-10


def test_correction_form_leaves_fp64_plans_and_batches_alone(wf):
    """The option acts on single mixed solves only: an FP64 plan's solve with
    the option set reproduces the one without it, and a mixed solve inside
    wf_solve_batch keeps a finite chi^2 trace (no switch)."""
    import torch

    nside, lmax, tol = 16, 32, 1e-6
    r_off, a_off, _, _ = _solve(wf, "fp64", nside, lmax, gen.seed_for(3, 56), tol)
    r_on, a_on, _, _ = _solve(wf, "fp64", nside, lmax, gen.seed_for(3, 56), tol, mixed_correction=100.0)
    assert r_on["iters"] == r_off["iters"]
    assert rel(a_on, a_off) < 1e-12
    P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(3, 57))
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="mixed")
    wf.wf_set_options(plan, mixed_correction=100.0)
    s = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
    item = {"d": T(d), "noise_var": T(P["noise_var"]), "mask": T(P["mask"]),
            "C_ell": T(P["c_ell"]), "tol": 1e-4, "s_out": s}
    rep = wf.wf_solve_batch([plan], [item], trace_cap=20000)[0]
    assert rep["converged"]
    assert np.all(np.isfinite(rep["chi2_trace"]))
    plan.close()
