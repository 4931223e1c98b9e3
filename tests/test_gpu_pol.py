"""Polarised (I, Q, U) path on the GPU against the oracle: the spin-2 basis
change (synthesis and its adjoint) to 1e-12, and the polarised messenger
solve of Eqs. 10-11 and its fluctuation variant (Eq. 9), FP64, to 1e-10
against the oracle replaying the GPU's own (lambda, L) trace."""
import numpy as np
import pytest

import oracle
import wf_inputs as gen
from gpu_util import T, healpix_pol_case, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    import torch

    import paper_1210_4931_gb300 as w

    w.load()
    torch.cuda.set_device(0)
    return w


def _rand_teb(rng, lmax):
    l, m = oracle.alm_lm(lmax)
    a = np.stack([gen.alm_unit_gaussian(rng, lmax) for _ in range(3)])
    a[1:, l < 2] = 0.0
    return a


@pytest.mark.parametrize("nside,lmax", [(2, 4), (4, 8), (8, 16), (16, 32), (32, 64), (64, 100)])
def test_pol_basis_change_matches_oracle(wf, nside, lmax):
    import torch

    rng = np.random.default_rng(500 + nside)
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64", ncomp=3)
    npx = 12 * nside * nside
    a = _rand_teb(rng, lmax)
    m = torch.empty(3 * npx, dtype=torch.float64, device="cuda")
    for L in (lmax, lmax // 2 + 1):
        wf.wf_alm2map(plan, T(a.ravel()), L, m)
        got = m.cpu().numpy().reshape(3, npx)
        I = oracle.synthesis(nside, lmax, L, a[0])
        Q, U = oracle.synthesis_pol(nside, lmax, L, a[1], a[2])
        ref = np.stack([I, Q, U])
        assert rel(got, ref) < 1e-12, (L, rel(got[0], I), rel(got[1], Q), rel(got[2], U))
    f = rng.standard_normal((3, npx))
    out = torch.empty(3 * plan.nalm, dtype=torch.complex128, device="cuda")
    for L in (lmax, lmax // 2 + 1):
        wf.wf_map2alm_adjoint(plan, T(f.ravel()), L, out)
        got = out.cpu().numpy().reshape(3, plan.nalm)
        Tt = oracle.adjoint_synthesis(nside, lmax, L, f[0])
        Et, Bt = oracle.adjoint_pol(nside, lmax, L, f[1], f[2])
        assert rel(got, np.stack([Tt, Et, Bt])) < 1e-12, (L, rel(got[1], Et), rel(got[2], Bt))
    plan.close()


def _pol_case(nside, lmax, seed, corr=0.1):
    return healpix_pol_case(nside, lmax, seed, corr=corr)


@pytest.mark.parametrize("nside,lmax", [(8, 16), (16, 32)])
def test_pol_solve_fp64_matches_oracle_replay(wf, nside, lmax):
    import torch

    from oracle.messenger_pol import messenger_solve_pol, pol_tau

    P, basis, d, nu, obs, N6, C4 = _pol_case(nside, lmax, gen.seed_for(4, nside))
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64", ncomp=3)
    npx = 12 * nside * nside
    s = torch.empty(3 * npx, dtype=torch.float64, device="cuda")
    alm = torch.empty(3 * plan.nalm, dtype=torch.complex128, device="cuda")
    rep = wf.wf_solve(plan, T(d.ravel()), T(N6.ravel()), T(P["mask"]), T(C4.ravel()), 1e-7, s, alm, trace_cap=20000)
    assert rep["converged"] and rep["final_residual"] < 1e-7
    tau = pol_tau(P["noise_cov"], obs)
    assert rep["tau"] == pytest.approx(tau, rel=1e-12)
    lam = rep["lambda_trace"]
    assert lam[-1] == 1.0 and np.all(np.diff(lam) <= 0)
    S = basis.per_mode(P["c_ell"])
    r = np.einsum("nij,jn->in", nu, d)
    ref = messenger_solve_pol(basis, r, nu, S, tau, replay=list(zip(lam, rep["L_trace"])))
    assert rel(alm.cpu().numpy().reshape(3, -1), ref["a"]) < 1e-10
    assert rel(s.cpu().numpy().reshape(3, npx), ref["s"]) < 1e-10
    np.testing.assert_allclose(rep["chi2_trace"], ref["chi2"], rtol=1e-10, atol=1e-10 * np.max(np.abs(ref["chi2"])))
    fin = ~np.isnan(ref["resid"])
    np.testing.assert_allclose(rep["resid_trace"][fin], ref["resid"][fin], rtol=1e-7)
    assert rep["n_dof"] == ref["n_dof"]
    plan.close()


def test_pol_rejections(wf):
    import torch

    nside, lmax = 8, 16
    P, basis, d, nu, obs, N6, C4 = _pol_case(nside, lmax, gen.seed_for(4, 99))
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64", ncomp=3)
    npx = 12 * nside * nside
    s = torch.empty(3 * npx, dtype=torch.float64, device="cuda")
    bad = N6.copy()
    k = np.nonzero(P["mask"])[0][5]
    bad[3, k] = 2.0 * np.sqrt(bad[0, k] * bad[1, k])  # |rho_IQ| > 1: not positive definite
    with pytest.raises(wf.WfError) as e:
        wf.wf_solve(plan, T(d.ravel()), T(bad.ravel()), T(P["mask"]), T(C4.ravel()), 1e-6, s)
    assert e.value.status == wf.WF_EINVAL
    badC = C4.copy()
    badC[3, 10] = 2.0 * np.sqrt(badC[0, 10] * badC[1, 10])
    with pytest.raises(wf.WfError) as e:
        wf.wf_solve(plan, T(d.ravel()), T(N6.ravel()), T(P["mask"]), T(badC.ravel()), 1e-6, s)
    assert e.value.status == wf.WF_EINVAL
    badC = C4.copy()
    badC[3, 12] = 1.0000001 * np.sqrt(badC[0, 12] * badC[1, 12])  # |rho_TE| just above 1
    g1 = T(np.zeros(3 * npx))
    g2 = T(np.zeros(3 * plan.nalm, dtype=np.complex128))
    with pytest.raises(wf.WfError) as e:
        wf.wf_fluct(plan, T(N6.ravel()), T(P["mask"]), T(badC.ravel()), g1, g2, 1e-6, s)
    assert e.value.status == wf.WF_EINVAL
    # mask codes: 4 is not one; a code-2 pixel (I only) needs N_II > 0 but nothing of Q, U;
    # a code-3 pixel (Q, U only) needs its 2x2 block positive definite; all masked is rejected
    m4 = P["mask"].copy()
    m4[3] = 4
    with pytest.raises(wf.WfError) as e:
        wf.wf_solve(plan, T(d.ravel()), T(N6.ravel()), T(m4), T(C4.ravel()), 1e-6, s)
    assert e.value.status == wf.WF_EINVAL
    k = np.nonzero(P["mask"])[0][7]
    m2, bad2 = P["mask"].copy(), N6.copy()
    m2[k] = 2
    bad2[1, k] = -1.0  # QQ < 0 is not observed at a code-2 pixel: accepted
    rep = wf.wf_solve(plan, T(d.ravel()), T(bad2.ravel()), T(m2), T(C4.ravel()), 1e-4, s)
    assert rep["status"] in (wf.WF_OK, wf.WF_ENOCONV)
    bad2[0, k] = 0.0  # N_II = 0 at an I-only pixel: rejected
    with pytest.raises(wf.WfError) as e:
        wf.wf_solve(plan, T(d.ravel()), T(bad2.ravel()), T(m2), T(C4.ravel()), 1e-6, s)
    assert e.value.status == wf.WF_EINVAL
    m3, bad3 = P["mask"].copy(), N6.copy()
    m3[k] = 3
    bad3[5, k] = 2.0 * np.sqrt(bad3[1, k] * bad3[2, k])  # |rho_QU| > 1
    with pytest.raises(wf.WfError) as e:
        wf.wf_solve(plan, T(d.ravel()), T(bad3.ravel()), T(m3), T(C4.ravel()), 1e-6, s)
    assert e.value.status == wf.WF_EINVAL
    with pytest.raises(wf.WfError) as e:
        wf.wf_solve(plan, T(d.ravel()), T(N6.ravel()), T(np.zeros_like(P["mask"])), T(C4.ravel()), 1e-6, s)
    assert e.value.status == wf.WF_EINVAL
    wf.wf_set_options(plan, schedule=1)
    with pytest.raises(wf.WfError) as e:
        wf.wf_solve(plan, T(d.ravel()), T(N6.ravel()), T(P["mask"]), T(C4.ravel()), 1e-6, s)
    assert e.value.status == wf.WF_EUNSUPPORTED
    plan.close()


@pytest.mark.parametrize("nside,lmax,corr", [(8, 16, 0.1), (16, 32, 0.1), (8, 16, 0.0)])
def test_pol_fluct_fp64_matches_oracle_replay(wf, nside, lmax, corr):
    """Fluctuation solve of Eq. (9) on (I, Q, U): the source nu^1/2 g1 +
    Omega Y (S^+1/2 g2) and the iteration against the oracle replaying the
    GPU's trace; corr = 0 gives noise blocks with equal Q and U variances
    (a repeated eigenvalue in the square root)."""
    import torch

    from oracle.messenger_pol import fluct_source_pol, messenger_solve_pol, pol_tau

    P, basis, d, nu, obs, N6, C4 = _pol_case(nside, lmax, gen.seed_for(4, 200 + nside), corr=corr)
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64", ncomp=3)
    npx = 12 * nside * nside
    rng = np.random.default_rng(700 + nside)
    g1 = rng.standard_normal((3, npx))
    g2 = np.stack([gen.alm_unit_gaussian(rng, lmax) for _ in range(3)])
    f = torch.empty(3 * npx, dtype=torch.float64, device="cuda")
    alm = torch.empty(3 * plan.nalm, dtype=torch.complex128, device="cuda")
    rep = wf.wf_fluct(plan, T(N6.ravel()), T(P["mask"]), T(C4.ravel()), T(g1.ravel()), T(g2.ravel()), 1e-7, f, alm,
                      trace_cap=20000)
    assert rep["converged"] and rep["final_residual"] < 1e-7
    assert np.isnan(rep["chi2_over_ndof"])
    tau = pol_tau(P["noise_cov"], obs)
    S = basis.per_mode(P["c_ell"])
    r = fluct_source_pol(basis, nu, S, g1, g2)
    ref = messenger_solve_pol(basis, r, nu, S, tau, replay=list(zip(rep["lambda_trace"], rep["L_trace"])))
    assert rel(alm.cpu().numpy().reshape(3, -1), ref["a"]) < 1e-10
    assert rel(f.cpu().numpy().reshape(3, npx), ref["s"]) < 1e-10
    np.testing.assert_allclose(rep["chi2_trace"], ref["chi2"], rtol=1e-10, atol=1e-10 * np.max(np.abs(ref["chi2"])))
    # the host entry point gives the same map
    fh = np.empty(3 * npx)
    rep_h = wf.wf_fluct_host(plan, np.ascontiguousarray(N6.ravel()), np.ascontiguousarray(P["mask"]),
                             np.ascontiguousarray(C4.ravel()), np.ascontiguousarray(g1.ravel()),
                             np.ascontiguousarray(g2.ravel()), 1e-7, fh)
    assert rep_h["iters"] == rep["iters"]
    assert rel(fh, f.cpu().numpy()) < 1e-12
    plan.close()


def test_pol_solve_with_b_modes_matches_oracle_replay(wf):
    """A prior with BB > 0 (B modes filtered too) and a TE block of full rank:
    the FP64 polarised solve against the oracle replaying its trace."""
    import torch

    from oracle.messenger_pol import messenger_solve_pol, pol_tau

    nside, lmax = 8, 16
    P, basis, d, nu, obs, N6, C4 = healpix_pol_case(nside, lmax, gen.seed_for(4, 77), bb_ratio=0.3)
    assert np.all(C4[2, 2:] > 0)
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64", ncomp=3)
    npx = 12 * nside * nside
    s = torch.empty(3 * npx, dtype=torch.float64, device="cuda")
    alm = torch.empty(3 * plan.nalm, dtype=torch.complex128, device="cuda")
    rep = wf.wf_solve(plan, T(d.ravel()), T(N6.ravel()), T(P["mask"]), T(C4.ravel()), 1e-8, s, alm, trace_cap=20000)
    assert rep["converged"]
    S = basis.per_mode(P["c_ell"])
    tau = pol_tau(P["noise_cov"], obs)
    r = np.einsum("nij,jn->in", nu, d)
    ref = messenger_solve_pol(basis, r, nu, S, tau, replay=list(zip(rep["lambda_trace"], rep["L_trace"])))
    got = alm.cpu().numpy().reshape(3, -1)
    assert np.max(np.abs(got[2])) > 1e-3 * np.max(np.abs(got[1]))  # B is not held at zero
    assert rel(got, ref["a"]) < 1e-10
    assert rel(s.cpu().numpy().reshape(3, npx), ref["s"]) < 1e-10
    plan.close()


@pytest.mark.parametrize("nside,lmax,L", [(16, 32, 17), (32, 64, 40)])
def test_pol_mixed_band_limited_transforms(wf, nside, lmax, L):
    """Mixed-precision (I, Q, U) transforms restricted to l <= L < lmax (the
    band limits of the cooling schedule) against the oracle."""
    import torch

    rng = np.random.default_rng(600 + L)
    a = _rand_teb(rng, lmax)
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="mixed", ncomp=3)
    npx = 12 * nside * nside
    m = torch.empty(3 * npx, dtype=torch.float64, device="cuda")
    wf.wf_alm2map(plan, T(a.ravel()), L, m)
    got = m.cpu().numpy().reshape(3, npx)
    I = oracle.synthesis(nside, lmax, L, a[0])
    Q, U = oracle.synthesis_pol(nside, lmax, L, a[1], a[2])
    for c, ref in enumerate((I, Q, U)):
        assert rel(got[c], ref) < 5e-5, (c, rel(got[c], ref))
    f = rng.standard_normal((3, npx))
    out = torch.empty(3 * plan.nalm, dtype=torch.complex128, device="cuda")
    wf.wf_map2alm_adjoint(plan, T(f.ravel()), L, out)
    got = out.cpu().numpy().reshape(3, plan.nalm)
    Tt = oracle.adjoint_synthesis(nside, lmax, L, f[0])
    Et, Bt = oracle.adjoint_pol(nside, lmax, L, f[1], f[2])
    for c, ref in enumerate((Tt, Et, Bt)):
        assert rel(got[c], ref) < 5e-5, (c, rel(got[c], ref))
    plan.close()


def _partial_case(nside, lmax, seed, **kw):
    """Separate masks: a temperature cut, a wider polarisation-only cut (code
    2) and, by hand, a few pixels that observe Q, U only (code 3); NaN in d
    on every unobserved component."""
    from oracle.messenger_pol import observed_components, pol_inverse_noise

    P, basis, d, nu, obs, N6, C4 = healpix_pol_case(nside, lmax, seed, p_b_cut_deg=25.0, **kw)
    code = P["mask"].copy()
    zero = np.nonzero(code == 0)[0]
    code[zero[::3]] = 3
    comp = observed_components(code)
    d = d.copy()
    d[~comp.T] = np.nan
    nu = pol_inverse_noise(P["noise_cov"], code)
    return P, basis, d, nu, code, N6, C4


@pytest.mark.parametrize("kind", ["wf", "fluct"])
def test_pol_separate_masks_match_oracle_replay(wf, kind):
    import torch

    from oracle.messenger_pol import fluct_source_pol, messenger_solve_pol, pol_tau

    nside, lmax = 16, 32
    P, basis, d, nu, code, N6, C4 = _partial_case(nside, lmax, gen.seed_for(4, 88))
    assert set(np.unique(code)) == {0, 1, 2, 3}
    npx = 12 * nside * nside
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64", ncomp=3)
    s = torch.empty(3 * npx, dtype=torch.float64, device="cuda")
    alm = torch.empty(3 * plan.nalm, dtype=torch.complex128, device="cuda")
    rng = np.random.default_rng(89)
    g1 = rng.standard_normal((3, npx))
    g2 = np.stack([gen.alm_unit_gaussian(rng, lmax) for _ in range(3)])
    if kind == "wf":
        rep = wf.wf_solve(plan, T(d.ravel()), T(N6.ravel()), T(code), T(C4.ravel()), 1e-8, s, alm, trace_cap=20000)
    else:
        rep = wf.wf_fluct(plan, T(N6.ravel()), T(code), T(C4.ravel()), T(g1.ravel()), T(g2.ravel()), 1e-8, s, alm,
                          trace_cap=20000)
    assert rep["converged"]
    tau = pol_tau(P["noise_cov"], code)
    assert rep["tau"] == pytest.approx(tau, rel=1e-12)
    S = basis.per_mode(P["c_ell"])
    if kind == "wf":
        r = np.einsum("nij,jn->in", nu, np.nan_to_num(d))
        assert np.isfinite(rep["chi2_over_ndof"])
    else:
        r = fluct_source_pol(basis, nu, S, g1, g2)
    ref = messenger_solve_pol(basis, r, nu, S, tau, replay=list(zip(rep["lambda_trace"], rep["L_trace"])))
    assert rep["n_dof"] == ref["n_dof"] == int(3 * np.sum(code == 1) + np.sum(code == 2) + 2 * np.sum(code == 3))
    assert rel(alm.cpu().numpy().reshape(3, -1), ref["a"]) < 1e-10
    assert rel(s.cpu().numpy().reshape(3, npx), ref["s"]) < 1e-10
    np.testing.assert_allclose(rep["chi2_trace"], ref["chi2"], rtol=1e-10, atol=1e-10 * np.max(np.abs(ref["chi2"])))
    plan.close()


def test_e_modes_in_the_polarisation_mask_follow_te(wf):
    """Quality experiment on synthetic data: inside a polarisation-only cut
    (I observed, Q and U masked), the Wiener filter's E modes come from the
    temperature through the TE correlation; with TE set to zero in the prior
    only what the polarisation data outside the cut constrain remains.  The
    filtered E-mode (Q, U) maps in the cut correlate with the true E-mode
    signal there far better with TE than without, on scales l >= 16 that the
    polarisation data outside a 60-degree-wide cut cannot reach (the lowest
    multipoles are constrained from outside the cut either way)."""
    import torch

    nside, lmax = 32, 64
    P, basis, d, nu, obs, N6, C4 = healpix_pol_case(nside, lmax, gen.seed_for(4, 90), p_b_cut_deg=30.0,
                                                    b_cut_deg=5.0, n_disks=4, pol_noise_factor=2.0)
    code = P["mask"]
    cut = code == 2
    assert cut.mean() > 0.3
    npx = 12 * nside * nside
    high = gen.alm_ell(lmax) >= 16
    Qt, Ut = oracle.synthesis_pol(nside, lmax, lmax, P["a_signal"][1] * high, np.zeros_like(P["a_signal"][2]))
    corr = {}
    for te in (True, False):
        C = C4.copy()
        if not te:
            C[3] = 0.0
        plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64", ncomp=3)
        s = torch.empty(3 * npx, dtype=torch.float64, device="cuda")
        alm = torch.empty(3 * plan.nalm, dtype=torch.complex128, device="cuda")
        rep = wf.wf_solve(plan, T(d.ravel()), T(N6.ravel()), T(code), T(C.ravel()), 1e-7, s, alm)
        assert rep["converged"]
        a = alm.cpu().numpy().reshape(3, -1)
        Qw, Uw = oracle.synthesis_pol(nside, lmax, lmax, a[1] * high, np.zeros_like(a[2]))
        num = np.sum(Qw[cut] * Qt[cut] + Uw[cut] * Ut[cut])
        den = np.sqrt(np.sum(Qw[cut] ** 2 + Uw[cut] ** 2) * np.sum(Qt[cut] ** 2 + Ut[cut] ** 2))
        corr[te] = num / den
        plan.close()
    assert corr[True] > 0.3 and corr[True] > corr[False] + 0.15, corr
