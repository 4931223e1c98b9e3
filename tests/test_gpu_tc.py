"""Tensor-core (tcgen05) Legendre synthesis of WF_PREC_MIXED_TF32 and
WF_PREC_MIXED_SPLITBF16 plans against the oracle (Sect. 2.1 basis change) and
against the FP32 plans.

Both splits keep FP32-grade accuracy (3xTF32: dropped terms below 2^-20 of a
product; three BF16 pieces with six products: below 2^-23), so the
tolerances are the FP32 path's: 2e-5 relative (max norm) against the oracle."""
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


def _cmb_alm(lmax, seed):
    rng = np.random.default_rng(seed)
    cl = gen.cmb_like_cl(lmax, 4 * 3438.0 / lmax)
    return gen.alm_unit_gaussian(rng, lmax) * np.sqrt(cl[gen.alm_ell(lmax)])


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("nside,lmax", [(4, 8), (16, 32), (64, 100), (64, 128), (128, 256), (200, 400)])
def test_tc_synthesis_matches_oracle(wf, nside, lmax, prec):
    """Sizes span one and several 256-pair CTAs (ragged last one), chunks of
    32 l with a ragged last chunk, and both recurrence forms."""
    import torch

    a = _cmb_alm(lmax, 100 + nside)
    ref = oracle.synthesis(nside, lmax, lmax, a)
    out = {}
    for pr in (prec, "mixed"):
        plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=pr)
        m = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
        wf.wf_alm2map(plan, T(a), lmax, m)
        out[pr] = m.cpu().numpy()
        plan.close()
    assert rel(out[prec], ref) < 2e-5
    assert rel(out[prec], out["mixed"]) < 2e-5


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("L", [0, 1, 33, 64, 95])
def test_tc_synthesis_band_limit(wf, L, prec):
    import torch

    nside, lmax = 48, 96
    a = gen.alm_unit_gaussian(np.random.default_rng(7), lmax)  # power at every l, l < 2 included
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=prec)
    m = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
    wf.wf_alm2map(plan, T(a), L, m)
    ref = oracle.synthesis(nside, lmax, L, a)
    assert rel(m.cpu().numpy(), ref) < 2e-5
    plan.close()


def test_tc_plan_rejections(wf):
    for prec in ("tf32", "bf16"):
        with pytest.raises(wf.WfError) as e:
            wf.wf_plan_create("flat", n=32, precision=prec)
        assert e.value.status == wf.WF_EUNSUPPORTED


def _cmb_teb(lmax, seed):
    """CMB-like (T, E, B) with EE = 0.05 TT and BB = 0.005 TT, so that E and B both reach
    the spin-2 synthesis, and no E, B power below l = 2."""
    rng = np.random.default_rng(seed)
    ell = gen.alm_ell(lmax)
    tt = gen.cmb_like_cl(lmax, 4 * 3438.0 / lmax)
    a = np.stack([gen.alm_unit_gaussian(rng, lmax) * np.sqrt(tt[ell] * f) for f in (1.0, 0.05, 0.005)])
    a[1:, ell < 2] = 0.0
    return a


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("nside,lmax", [(4, 8), (16, 32), (64, 100), (128, 256), (200, 400)])
def test_tc_pol_synthesis_matches_oracle(wf, nside, lmax, prec):
    """(I, Q, U) synthesis of a polarised tensor-core plan: T through the temperature
    tensor-core kernel, E and B through the spin-2 one (the Re and Im of E + iB and E - iB
    against the spin +2 and -2 recurrences, even and odd l - m in separate accumulators).
    Each component within 5e-5 of the oracle (relative to its largest value, as the FP32
    polarised kernels) and of the FP32 plan."""
    import torch

    a = _cmb_teb(lmax, 300 + nside)
    I = oracle.synthesis(nside, lmax, lmax, a[0])
    Q, U = oracle.synthesis_pol(nside, lmax, lmax, a[1], a[2])
    out = {}
    for pr in (prec, "mixed"):
        plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=pr, ncomp=3)
        m = torch.empty(3 * plan.npix, dtype=torch.float64, device="cuda")
        wf.wf_alm2map(plan, T(a.ravel()), lmax, m)
        out[pr] = m.cpu().numpy().reshape(3, plan.npix)
        plan.close()
    for c, ref in enumerate((I, Q, U)):
        assert rel(out[prec][c], ref) < 5e-5, (c, rel(out[prec][c], ref))
        assert rel(out[prec][c], out["mixed"][c]) < 5e-5, (c, rel(out[prec][c], out["mixed"][c]))


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("L", [0, 2, 33, 95])
def test_tc_pol_synthesis_band_limit(wf, L, prec):
    import torch

    nside, lmax = 48, 96
    rng = np.random.default_rng(17)
    a = np.stack([gen.alm_unit_gaussian(rng, lmax) for _ in range(3)])
    a[1:, gen.alm_ell(lmax) < 2] = 0.0
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=prec, ncomp=3)
    m = torch.empty(3 * plan.npix, dtype=torch.float64, device="cuda")
    wf.wf_alm2map(plan, T(a.ravel()), L, m)
    got = m.cpu().numpy().reshape(3, plan.npix)
    plan.close()
    I = oracle.synthesis(nside, lmax, L, a[0])
    Q, U = oracle.synthesis_pol(nside, lmax, L, a[1], a[2])
    for c, ref in enumerate((I, Q, U)):
        if np.max(np.abs(ref)) == 0.0:
            assert np.max(np.abs(got[c])) == 0.0
        else:
            assert rel(got[c], ref) < 5e-5, (c, rel(got[c], ref))


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_tc_solve_matches_mixed_and_reaches_tol(wf, prec):
    """A whole mixed solve with the tensor-core synthesis: same iteration as
    the FP32 plan within the mixed tolerance, residual below tol."""
    import torch

    nside, lmax = 32, 64
    P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(2, 77))
    res = {}
    for pr in (prec, "mixed"):
        plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=pr)
        s = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
        rep = wf.wf_solve(plan, T(d), T(P["noise_var"]), T(P["mask"]), T(P["c_ell"]), 1e-5, s, trace_cap=20000)
        assert rep["converged"] and rep["final_residual"] < 1e-5
        res[pr] = s.cpu().numpy()
        plan.close()
    assert rel(res[prec], res["mixed"]) < 1e-4


def _pair_items(nside, lmax, nmaps, seed):
    """nmaps maps of one noise model, each a Wiener filter plus a
    fluctuation solve (Sect. 2.3): 2 nmaps items of one geometry."""
    import torch

    P, basis, d0, nu, tau = healpix_case(nside, lmax, seed)
    items = []
    for j in range(nmaps):
        rng = np.random.default_rng(seed + 31 * j)
        d = basis.synth(gen.alm_unit_gaussian(rng, lmax) * np.sqrt(P["c_ell"][gen.alm_ell(lmax)])) + \
            np.sqrt(P["noise_var"]) * rng.standard_normal(P["noise_var"].size)
        common = {"noise_var": T(P["noise_var"]), "mask": T(P["mask"]), "C_ell": T(P["c_ell"]), "tol": 1e-5}
        items.append(dict(common, kind="wf", d=T(d),
                          s_out=torch.full((d.size,), float("nan"), dtype=torch.float64, device="cuda")))
        items.append(dict(common, kind="fluct", g1=T(rng.standard_normal(d.size)),
                          g2=T(np.ascontiguousarray(gen.alm_unit_gaussian(rng, lmax), dtype=np.complex128)),
                          s_out=torch.full((d.size,), float("nan"), dtype=torch.float64, device="cuda")))
    return items


def _alone(w, nside, lmax, prec, it):
    import torch

    plan = w.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=prec)
    s = torch.empty_like(it["s_out"])
    if it["kind"] == "wf":
        rep = w.wf_solve(plan, it["d"], it["noise_var"], it["mask"], it["C_ell"], it["tol"], s, trace_cap=20000)
    else:
        rep = w.wf_fluct(plan, it["noise_var"], it["mask"], it["C_ell"], it["g1"], it["g2"], it["tol"], s,
                         trace_cap=20000)
    plan.close()
    return s.cpu().numpy(), rep


@pytest.mark.parametrize("prec,nmaps", [("tf32", 1), ("tf32", 3), ("tf32", 9), ("bf16", 3)])
def test_tc_batch_columns(wf, prec, nmaps):
    """Wiener-filter + fluctuation pairs of one geometry in wf_solve_batch:
    the tensor-core synthesis of every item runs in one launch per step (the
    items are the columns of one contraction; 9 maps = 18 columns span two
    launches of at most 16), and each item's result equals the same solve
    run alone (the columns do not interact: same iterations, same lambda
    trace, maps equal to 1e-12)."""
    nside, lmax = 32, 64
    items = _pair_items(nside, lmax, nmaps, gen.seed_for(4, 40 + nmaps))
    alone = [_alone(wf, nside, lmax, prec, it) for it in items]
    plans = [wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=prec) for _ in items]
    reps = wf.wf_solve_batch(plans, items, trace_cap=20000)
    for it, rep, (s_alone, rep_alone) in zip(items, reps, alone):
        assert rep["status"] == wf.WF_OK and rep["converged"]
        assert rep["iters"] == rep_alone["iters"]
        np.testing.assert_array_equal(rep["lambda_trace"], rep_alone["lambda_trace"])
        assert rel(it["s_out"].cpu().numpy(), s_alone) < 1e-12
    # launches: one group synthesis per step for up to 16 columns, counted on the group's first item
    ls = [r["kernel_launches"]["leg_syn"] for r in reps]
    ls_alone = [r["kernel_launches"]["leg_syn"] for _, r in alone]
    assert sum(ls) < sum(ls_alone) or len(items) == 1
    for p in plans:
        p.close()


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_tc_fluct_matches_mixed(wf, prec):
    """The fluctuation solve (Eq. 9) with the tensor-core synthesis: its source
    z = Omega Y (S^-1/2 g2) goes through the same synthesis.  Both plans reach
    the residual tolerance; the maps agree to the accuracy a 1e-6 residual
    gives."""
    import torch

    nside, lmax = 32, 64
    P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(2, 79))
    rng = np.random.default_rng(5)
    g1 = rng.standard_normal(d.size)
    g2 = np.ascontiguousarray(gen.alm_unit_gaussian(rng, lmax), dtype=np.complex128)
    res = {}
    for pr in (prec, "mixed"):
        plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=pr)
        f = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
        rep = wf.wf_fluct(plan, T(P["noise_var"]), T(P["mask"]), T(P["c_ell"]), T(g1), T(g2), 1e-6, f,
                          trace_cap=20000)
        assert rep["converged"] and rep["final_residual"] < 1e-6
        res[pr] = f.cpu().numpy()
        plan.close()
    print("fluct rel diff", prec, rel(res[prec], res["mixed"]))
    assert rel(res[prec], res["mixed"]) < 1e-3


@pytest.mark.parametrize("prec,nmaps", [("tf32", 3), ("tf32", 5), ("bf16", 2)])
def test_tc_pol_batch_columns(wf, prec, nmaps):
    """Polarised Wiener-filter + fluctuation pairs of one geometry and noise model in
    wf_solve_batch: every step runs one temperature and one spin-2 tensor-core synthesis
    for up to 8 items (5 maps = 10 items span two groups), and each item's result equals
    the same solve run alone (same iterations and lambda trace, maps to 1e-12)."""
    import torch

    from gpu_util import healpix_pol_case

    nside, lmax = 32, 64
    P, basis, d, nu, obs, N6, C4 = healpix_pol_case(nside, lmax, gen.seed_for(4, 600 + nmaps))
    npx = 12 * nside * nside
    rng = np.random.default_rng(6000 + nmaps)
    items = []
    for k in range(nmaps):
        dk = d + 0.1 * np.std(d) * rng.standard_normal(d.shape)
        g1 = rng.standard_normal((3, npx))
        g2 = np.stack([gen.alm_unit_gaussian(rng, lmax) for _ in range(3)])
        common = {"noise_var": T(N6.ravel()), "mask": T(P["mask"]), "C_ell": T(C4.ravel()), "tol": 1e-4}
        items.append(dict(common, kind="wf", d=T(dk.ravel()),
                          s_out=torch.full((3 * npx,), float("nan"), dtype=torch.float64, device="cuda")))
        items.append(dict(common, kind="fluct", g1=T(g1.ravel()), g2=T(g2.ravel()),
                          s_out=torch.full((3 * npx,), float("nan"), dtype=torch.float64, device="cuda")))
    alone = []
    for it in items:
        pl = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=prec, ncomp=3)
        s = torch.empty_like(it["s_out"])
        if it["kind"] == "wf":
            rep = wf.wf_solve(pl, it["d"], it["noise_var"], it["mask"], it["C_ell"], it["tol"], s, trace_cap=20000)
        else:
            rep = wf.wf_fluct(pl, it["noise_var"], it["mask"], it["C_ell"], it["g1"], it["g2"], it["tol"], s,
                              trace_cap=20000)
        pl.close()
        alone.append((s.cpu().numpy(), rep))
    plans = [wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=prec, ncomp=3) for _ in items]
    reps = wf.wf_solve_batch(plans, items, trace_cap=20000)
    for i, (it, rep, (s_alone, rep_alone)) in enumerate(zip(items, reps, alone)):
        assert rep["status"] == wf.WF_OK and rep["converged"], (i, rep["status"], rep["final_residual"])
        assert rep["iters"] == rep_alone["iters"], (i, rep["iters"], rep_alone["iters"])
        np.testing.assert_array_equal(rep["lambda_trace"], rep_alone["lambda_trace"])
        assert rel(it["s_out"].cpu().numpy(), s_alone) < 1e-12, (i, rel(it["s_out"].cpu().numpy(), s_alone))
    ls = [r["kernel_launches"]["leg_syn"] for r in reps]
    ls_alone = [r["kernel_launches"]["leg_syn"] for _, r in alone]
    assert sum(ls) < sum(ls_alone)
    for p in plans:
        p.close()
