"""GPU path vs the oracle, element by element, through the C ABI.

FP64 mode must match within 1e-10 relative (schedule replay: the oracle
re-runs the GPU's own lambda/L trace).  Sizes span all three ring-DFT
engines (direct, power-of-two FFT, Bluestein) and several Legendre tiles."""
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


def _random_alm(lmax, rng, cl=None):
    g = gen.alm_unit_gaussian(rng, lmax)
    if cl is not None:
        g = g * np.sqrt(cl[gen.alm_ell(lmax)])
    return g


@pytest.mark.parametrize("nside,lmax", [(2, 4), (4, 8), (8, 16), (16, 32), (32, 64), (64, 128), (64, 100)])
def test_basis_change_matches_oracle(wf, nside, lmax):
    import torch

    rng = np.random.default_rng(nside * 1000 + lmax)
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64")
    a = _random_alm(lmax, rng)
    m = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
    for L in (lmax, lmax // 2 + 1):
        wf.wf_alm2map(plan, T(a), L, m)
        assert rel(m.cpu().numpy(), oracle.synthesis(nside, lmax, L, a)) < 1e-12
    f = rng.standard_normal(plan.npix)
    out = torch.empty(plan.nalm, dtype=torch.complex128, device="cuda")
    for L in (lmax, lmax // 2 + 1):
        wf.wf_map2alm_adjoint(plan, T(f), L, out)
        assert rel(out.cpu().numpy(), oracle.adjoint_synthesis(nside, lmax, L, f)) < 1e-12
    plan.close()


@pytest.mark.parametrize("nside,lmax", [(8, 16), (16, 32), (32, 64)])
def test_healpix_solve_fp64_matches_oracle_replay(wf, nside, lmax):
    import torch

    P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(2, 100 + nside))
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64")
    s = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
    alm = torch.empty(plan.nalm, dtype=torch.complex128, device="cuda")
    rep = wf.wf_solve(plan, T(d), T(P["noise_var"]), T(P["mask"]), T(P["c_ell"]), 1e-7, s, alm, trace_cap=20000)
    assert rep["converged"] and rep["final_residual"] < 1e-7
    lam = rep["lambda_trace"]
    assert lam[0] >= 1.0 and lam[-1] == 1.0 and np.all(np.diff(lam) <= 0)
    if nside >= 32:
        assert lam[0] > 1.0  # the prior at l_iter = 20 is above T: cooling starts high
    replay = list(zip(lam, rep["L_trace"]))
    ref = oracle.messenger_solve(basis, nu * d, nu, basis.per_mode(P["c_ell"]), tau, replay=replay, d=d)
    assert rel(alm.cpu().numpy(), ref["a"]) < 1e-10
    assert rel(s.cpu().numpy(), ref["s"]) < 1e-10
    np.testing.assert_allclose(rep["chi2_trace"], ref["chi2"], rtol=1e-10, atol=1e-10 * np.max(np.abs(ref["chi2"])))
    fin = ~np.isnan(ref["resid"])
    np.testing.assert_allclose(rep["resid_trace"][fin], ref["resid"][fin], rtol=1e-7)
    assert rep["chi2_over_ndof"] == pytest.approx(ref["chi2_final"] / ref["n_dof"], rel=1e-10)
    assert rep["tau"] == tau
    plan.close()


@pytest.mark.parametrize("n", [16, 32, 128])
def test_flat_solve_fp64_matches_oracle_replay(wf, n):
    import torch

    P = gen.flat_problem(n, seed=gen.seed_for(1, n)) if n == 128 else gen.flat_problem(
        n, seed=gen.seed_for(1, n), band_rows=(n // 2 - 2, n // 2 + 2), n_disks=3, disk_radius=2.0)
    B = oracle.FlatBasis(n, n)
    d = B.synth(P["a_signal"]) + P["noise"]
    obs = P["mask"] > 0
    nu = np.where(obs, 1.0 / P["noise_var"], 0.0)
    tau = float(P["noise_var"][obs].min())
    plan = wf.wf_plan_create("flat", n=n, precision="fp64")
    s = torch.empty(n * n, dtype=torch.float64, device="cuda")
    alm = torch.empty(plan.nalm, dtype=torch.complex128, device="cuda")
    rep = wf.wf_solve(plan, T(d.ravel()), T(P["noise_var"].ravel()), T(P["mask"].ravel()), T(P["S"].ravel()), 1e-6,
                      s, alm, trace_cap=20000)
    assert rep["converged"] and rep["final_residual"] < 1e-6
    lam = rep["lambda_trace"]
    assert lam[0] == 100.0 and lam[-1] == 1.0
    ref = oracle.messenger_solve(B, nu * d, nu, P["S"], tau, replay=[(l, None) for l in lam], d=d)
    assert rel(s.cpu().numpy().reshape(n, n), ref["s"]) < 1e-10
    assert rel(alm.cpu().numpy().reshape(n, n // 2 + 1), ref["a"]) < 1e-10
    fin = ~np.isnan(ref["resid"])
    np.testing.assert_allclose(rep["resid_trace"][fin], ref["resid"][fin], rtol=1e-7)
    assert rep["chi2_over_ndof"] == pytest.approx(ref["chi2_final"] / ref["n_dof"], rel=1e-10)
    plan.close()


def test_flat_fluct_matches_oracle(wf):
    import torch

    n = 32
    P = gen.flat_problem(n, seed=gen.seed_for(1, 7), band_rows=(14, 18), n_disks=3, disk_radius=2.0)
    B = oracle.FlatBasis(n, n)
    obs = P["mask"] > 0
    nu = np.where(obs, 1.0 / P["noise_var"], 0.0)
    tau = float(P["noise_var"][obs].min())
    plan = wf.wf_plan_create("flat", n=n)
    f = torch.empty(n * n, dtype=torch.float64, device="cuda")
    rep = wf.wf_fluct(plan, T(P["noise_var"].ravel()), T(P["mask"].ravel()), T(P["S"].ravel()),
                      T(P["g1"].ravel()), T(P["g2"].ravel()), 1e-6, f, trace_cap=20000)
    assert rep["converged"]
    r = oracle.fluct_source(B, nu, P["S"], P["g1"], P["g2"])
    ref = oracle.messenger_solve(B, r, nu, P["S"], tau, replay=[(l, None) for l in rep["lambda_trace"]])
    assert rel(f.cpu().numpy().reshape(n, n), ref["s"]) < 1e-10
    plan.close()


def test_healpix_fluct_matches_oracle(wf):
    import torch

    nside, lmax = 16, 32
    P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(2, 300))
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax)
    f = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
    rep = wf.wf_fluct(plan, T(P["noise_var"]), T(P["mask"]), T(P["c_ell"]), T(P["g1"]), T(P["g2"]), 1e-7, f,
                      trace_cap=20000)
    assert rep["converged"]
    S = basis.per_mode(P["c_ell"])
    r = oracle.fluct_source(basis, nu, S, P["g1"], P["g2"])
    ref = oracle.messenger_solve(basis, r, nu, S, tau, replay=list(zip(rep["lambda_trace"], rep["L_trace"])))
    assert rel(f.cpu().numpy(), ref["s"]) < 1e-10
    plan.close()


def test_invalid_inputs_are_rejected(wf):
    import torch

    nside, lmax = 8, 16
    P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(2, 5))
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax)
    s = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
    bad = P["noise_var"].copy()
    bad[np.nonzero(P["mask"])[0][3]] = np.nan
    with pytest.raises(wf.WfError) as e:
        wf.wf_solve(plan, T(d), T(bad), T(P["mask"]), T(P["c_ell"]), 1e-6, s)
    assert e.value.status == wf.WF_EINVAL
    bad = P["noise_var"].copy()
    bad[np.nonzero(P["mask"])[0][0]] = -1.0
    with pytest.raises(wf.WfError):
        wf.wf_solve(plan, T(d), T(bad), T(P["mask"]), T(P["c_ell"]), 1e-6, s)
    with pytest.raises(wf.WfError):
        wf.wf_solve(plan, T(d), T(P["noise_var"]), T(np.zeros_like(P["mask"])), T(P["c_ell"]), 1e-6, s)
    # masked pixels may hold anything, including NaN noise
    nv = P["noise_var"].copy()
    nv[P["mask"] == 0] = np.nan
    rep = wf.wf_solve(plan, T(d), T(nv), T(P["mask"]), T(P["c_ell"]), 1e-6, s)
    assert rep["converged"]
    with pytest.raises(wf.WfError):
        wf.wf_plan_create("healpix", nside=8, lmax=17)
    # the prior must be finite and >= 0 (C_0 = C_1 = 0 is allowed)
    for bad_c in (-1e-3, np.nan, np.inf):
        cl = P["c_ell"].copy()
        cl[5] = bad_c
        with pytest.raises(wf.WfError) as e:
            wf.wf_solve(plan, T(d), T(P["noise_var"]), T(P["mask"]), T(cl), 1e-6, s)
        assert e.value.status == wf.WF_EINVAL
    plan.close()
    pm = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="mixed")
    cl = P["c_ell"].copy()
    cl[7] = -cl[7]
    with pytest.raises(wf.WfError) as e:
        wf.wf_solve(pm, T(d), T(P["noise_var"]), T(P["mask"]), T(cl), 1e-6, s)
    assert e.value.status == wf.WF_EINVAL
    pm.close()
    # flat grid: S per mode
    n = 32
    F = gen.flat_problem(n, seed=gen.seed_for(1, 5))
    pf = wf.wf_plan_create("flat", n=n)
    sf = torch.empty(n * n, dtype=torch.float64, device="cuda")
    for bad_s in (-1.0, np.nan):
        S = F["S"].copy()
        S[1, 1] = bad_s
        with pytest.raises(wf.WfError) as e:
            wf.wf_solve(pf, T(F["noise"].ravel()), T(F["noise_var"].ravel()), T(F["mask"].ravel()),
                        T(S.ravel()), 1e-6, sf)
        assert e.value.status == wf.WF_EINVAL
    pf.close()


def test_no_mask_pointer_means_all_observed(wf):
    import torch

    nside, lmax = 8, 16
    P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(2, 6), masked=False)
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax)
    s1 = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
    s2 = torch.empty_like(s1)
    r1 = wf.wf_solve(plan, T(d), T(P["noise_var"]), None, T(P["c_ell"]), 1e-8, s1)
    r2 = wf.wf_solve(plan, T(d), T(P["noise_var"]), T(P["mask"]), T(P["c_ell"]), 1e-8, s2)
    assert r1["iters"] == r2["iters"]
    assert rel(s1.cpu().numpy(), s2.cpu().numpy()) < 1e-14
    plan.close()


def test_host_entry_point_matches_device(wf):
    import torch

    nside, lmax = 16, 32
    P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(2, 8))
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax)
    s = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
    wf.wf_solve(plan, T(d), T(P["noise_var"]), T(P["mask"]), T(P["c_ell"]), 1e-7, s)
    sh = np.empty(plan.npix)
    ah = np.empty(plan.nalm, dtype=np.complex128)
    rep = wf.wf_solve_host(plan, d, P["noise_var"], P["mask"], P["c_ell"], 1e-7, sh, ah)
    assert rep["converged"]
    assert rel(sh, s.cpu().numpy()) < 1e-13
    plan.close()


def test_flat_plans_of_different_sizes_coexist(wf):
    """A small flat plan created after a large one must not break the large
    one (per-function launch attributes are shared by all plans)."""
    import torch

    big = wf.wf_plan_create("flat", n=128)
    small = wf.wf_plan_create("flat", n=16)
    P = gen.flat_problem(128, seed=gen.seed_for(1, 55))
    d = oracle.FlatBasis(128, 128).synth(P["a_signal"]) + P["noise"]
    s = torch.empty(128 * 128, dtype=torch.float64, device="cuda")
    rep = wf.wf_solve(big, T(d.ravel()), T(P["noise_var"].ravel()), T(P["mask"].ravel()), T(P["S"].ravel()), 1e-6, s)
    assert rep["converged"]
    small.close()
    big.close()


@pytest.mark.parametrize("nside", [8, 64])
def test_template_marginalisation_matches_oracle(wf, nside):
    import torch

    P, basis, d, nu, tau = healpix_case(nside, 2 * nside, gen.seed_for(2, 400 + nside))
    th, ph = oracle.pixel_angles(nside)
    d_raw = d + 5.0 + 0.7 * np.sin(th) * np.cos(ph) - 1.3 * np.cos(th)  # residual monopole + dipole
    ref, cref = oracle.marginalize_templates(nside, d_raw, P["mask"])
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=2 * nside, precision="fp64")
    out = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
    c = wf.wf_remove_templates(plan, T(d_raw), T(P["mask"]), out)
    assert rel(out.cpu().numpy(), ref) < 1e-10
    np.testing.assert_allclose(c, cref, rtol=1e-9, atol=1e-9)
    plan.close()


@pytest.mark.parametrize("nside", [8, 16])
def test_chi2_bound_schedule_matches_oracle(wf, nside):
    """Cooling of Sect. 2.2 on the GPU: lambda solves chi^2(lambda, x_k) = b
    for every iterate; the result matches the oracle replaying the GPU's
    lambda trace, the reported chi^2 is the full chi^2 (J-form of the oracle
    plus its x-independent term), and the lambda decisions match the oracle
    running the same schedule on its own."""
    import torch

    from oracle.messenger import RigorousSchedule

    lmax = 2 * nside
    P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(2, 700 + nside))
    S = basis.per_mode(P["c_ell"])
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64")
    wf.wf_set_options(plan, schedule=1)
    s = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
    alm = torch.empty(plan.nalm, dtype=torch.complex128, device="cuda")
    rep = wf.wf_solve(plan, T(d), T(P["noise_var"]), T(P["mask"]), T(P["c_ell"]), 1e-7, s, alm, trace_cap=20000)
    assert rep["converged"] and rep["final_residual"] < 1e-7
    lam, chi2 = rep["lambda_trace"], rep["chi2_trace"]
    assert lam[0] > 1.0 and np.all(np.diff(lam) <= 0) and lam[-1] == 1.0
    assert np.all(rep["L_trace"] == lmax)

    ref = oracle.messenger_solve(basis, nu * d, nu, S, tau, replay=[(x, lmax) for x in lam], d=d)
    assert rel(alm.cpu().numpy(), ref["a"]) < 1e-10
    assert rel(s.cpu().numpy(), ref["s"]) < 1e-10
    const = np.array([np.sum(nu * d * d / (1.0 + (x - 1.0) * tau * nu)) for x in lam])
    np.testing.assert_allclose(chi2, ref["chi2"] + const, rtol=1e-9, atol=1e-11 * const.max())

    n_dof = int(np.count_nonzero(nu > 0))
    b0 = n_dof - 5.0 * np.sqrt(2.0 * n_dof)
    assert chi2[0] == pytest.approx(b0, rel=1e-12)
    hot = lam > 1.0
    assert np.all(np.diff(chi2[hot]) >= -1e-9 * b0)  # b only rises

    sch = RigorousSchedule(n_dof)
    ind = oracle.messenger_solve(basis, nu * d, nu, S, tau, schedule=sch, tol=1e-7, d=d, maxiter=20000)
    lam_o = np.array([t[0] for t in ind["trace"]])
    k = min(50, lam_o.size, lam.size)
    np.testing.assert_allclose(lam[:k] - 1.0, lam_o[:k] - 1.0, rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(chi2[:k][hot[:k]], ind["bound"][:k][hot[:k]], rtol=1e-10)
    assert abs(ind["iters"] - rep["iters"]) <= 0.02 * ind["iters"] + 2
    plan.close()


def test_chi2_bound_schedule_rejections(wf):
    import torch

    nside, lmax = 8, 16
    P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(2, 9))
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64")
    wf.wf_set_options(plan, schedule=1)
    f = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
    g1 = T(np.zeros(plan.npix))
    g2 = T(np.zeros(plan.nalm, dtype=np.complex128))
    with pytest.raises(wf.WfError) as e:
        wf.wf_fluct(plan, T(P["noise_var"]), T(P["mask"]), T(P["c_ell"]), g1, g2, 1e-6, f)
    assert e.value.status == wf.WF_EUNSUPPORTED
    with pytest.raises(wf.WfError) as e:
        wf.wf_set_options(plan, schedule=2)
    assert e.value.status == wf.WF_EINVAL
    plan.close()
    flat = wf.wf_plan_create("flat", n=16)
    wf.wf_set_options(flat, schedule=1)
    Pf = gen.flat_problem(16, seed=gen.seed_for(1, 9))
    sf = torch.empty(256, dtype=torch.float64, device="cuda")
    with pytest.raises(wf.WfError) as e:
        wf.wf_solve(flat, T(Pf["noise"].ravel()), T(Pf["noise_var"].ravel()), T(Pf["mask"].ravel()),
                    T(Pf["S"].ravel()), 1e-6, sf)
    assert e.value.status == wf.WF_EUNSUPPORTED
    flat.close()


@pytest.mark.parametrize("ncomp", [1, 3])
def test_checkpoint_resume_repeats_the_uninterrupted_run(wf, ncomp):
    """A replayed run stopped after k iterations and resumed from its alm_out
    with the rest of the trace (wf_set_start + wf_set_schedule) ends where the
    uninterrupted run ends (FP64, to the reduction order of the atomics)."""
    import torch

    from gpu_util import healpix_pol_case

    nside, lmax = 16, 32
    if ncomp == 1:
        P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(2, 77))
        args = (T(d), T(P["noise_var"]), T(P["mask"]), T(P["c_ell"]))
    else:
        P, basis, d, nu, obs, N6, C4 = healpix_pol_case(nside, lmax, gen.seed_for(4, 78))
        args = (T(d.ravel()), T(N6.ravel()), T(P["mask"]), T(C4.ravel()))
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64", ncomp=ncomp)
    n = ncomp * plan.npix
    s_full = torch.empty(n, dtype=torch.float64, device="cuda")
    a_full = torch.empty(ncomp * plan.nalm, dtype=torch.complex128, device="cuda")
    wf.wf_set_options(plan, maxiter=240)
    rep = wf.wf_solve(plan, *args, 1e-30, s_full, a_full, trace_cap=400)  # tol below reach: 240 iterations
    lam, Ls = rep["lambda_trace"], rep["L_trace"]
    assert rep["iters"] == len(lam) == 240
    k = len(lam) // 3
    wf.wf_set_schedule(plan, lam[:k], Ls[:k])
    s1 = torch.empty_like(s_full)
    a1 = torch.empty_like(a_full)
    wf.wf_solve(plan, *args, 1e-30, s1, a1)
    wf.wf_set_start(plan, a1)
    wf.wf_set_schedule(plan, lam[k:], Ls[k:])
    s2 = torch.empty_like(s_full)
    rep2 = wf.wf_solve(plan, *args, 1e-30, s2, trace_cap=400)
    assert rep2["iters"] == len(lam) - k
    assert rel(s2.cpu().numpy(), s_full.cpu().numpy()) < 1e-12
    wf.wf_set_start(plan, None)
    wf.wf_set_schedule(plan, [], [])
    plan.close()
