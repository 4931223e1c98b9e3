"""Batched solves (wf_solve_batch): solves of uneven size advanced together,
one CUDA graph per step.  Each item must give the result of the same solve
run alone (wf_solve / wf_fluct on a fresh plan of the same geometry): FP64
to 1e-10 relative with the same iteration count and kernel-launch count,
mixed precision within the solve tolerance."""
import numpy as np
import pytest

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


CASES = [  # nside, lmax, precision, kind, tol
    (16, 32, "fp64", "wf", 1e-8),
    (32, 64, "mixed", "wf", 1e-5),
    (16, 32, "mixed", "fluct", 1e-5),
    (32, 64, "fp64", "fluct", 1e-7),
    (64, 128, "mixed", "wf", 1e-5),
    (8, 16, "fp64", "wf", 1e-9),
]


def _item(i, nside, lmax, kind, tol):
    import torch

    P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(6, i))
    rng = np.random.default_rng(2000 + i)
    it = {"kind": kind, "noise_var": T(P["noise_var"]), "mask": T(P["mask"]), "C_ell": T(P["c_ell"]), "tol": tol,
          "s_out": torch.full((d.size,), float("nan"), dtype=torch.float64, device="cuda"),
          "alm_out": torch.empty(basis.ell.size, dtype=torch.complex128, device="cuda")}
    if kind == "wf":
        it["d"] = T(d)
    else:
        it["g1"] = T(rng.standard_normal(d.size))
        it["g2"] = T(np.ascontiguousarray(gen.alm_unit_gaussian(rng, lmax), dtype=np.complex128))
    return it


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


def test_batch_equals_solves_run_alone(wf):
    items = [_item(i, n, l, k, t) for i, (n, l, p, k, t) in enumerate(CASES)]
    alone = [_alone(wf, n, l, p, it) for (n, l, p, k, t), it in zip(CASES, items)]
    plans = [wf.wf_plan_create("healpix", nside=n, lmax=l, precision=p) for n, l, p, k, t in CASES]
    reps = wf.wf_solve_batch(plans, items, trace_cap=20000)
    for (n, l, p, k, t), it, rep, (s_alone, rep_alone) in zip(CASES, items, reps, alone):
        assert rep["status"] == wf.WF_OK, (n, p, k, rep["status"])
        s = it["s_out"].cpu().numpy()
        if p == "fp64":
            assert rel(s, s_alone) < 1e-10, (n, k, rel(s, s_alone))
            assert rep["iters"] == rep_alone["iters"]
            np.testing.assert_array_equal(rep["lambda_trace"], rep_alone["lambda_trace"])
            assert rep["launches"] == rep_alone["launches"] > 0
        else:
            assert rep["final_residual"] < t and rep_alone["final_residual"] < t
            assert rel(s, s_alone) < 1e-3, (n, k, rel(s, s_alone))
            # the batched mixed item's a_lm under the oracle's FP64 operator: the FP32 iteration
            # stops on its own operator's residual, which the FP64 one matches to the FP32
            # operator error (well below tol here)
            import oracle as orc

            P, basis, d, nu, tau = healpix_case(n, l, gen.seed_for(6, CASES.index((n, l, p, k, t))))
            r_src = nu * d if k == "wf" else orc.fluct_source(basis, nu, basis.per_mode(P["c_ell"]),
                                                                it["g1"].cpu().numpy(), it["g2"].cpu().numpy())
            r1 = orc.messenger_solve(basis, r_src, nu, basis.per_mode(P["c_ell"]), tau, replay=[(1.0, l)],
                                     a0=it["alm_out"].cpu().numpy())
            print("batch item", n, k, "fp64-operator residual", r1["resid"][0], "reported", rep["final_residual"])
            assert r1["resid"][0] < 1.5 * t
    for pl in plans:
        pl.close()


def test_batch_of_one_and_reuse_of_plans(wf):
    """A batch of one, and the same plans used for a second batch, give the
    same FP64 results (the graph and streams are per call)."""
    n, l, p, k, t = CASES[0]
    it = _item(0, n, l, k, t)
    plan = wf.wf_plan_create("healpix", nside=n, lmax=l, precision=p)
    r1 = wf.wf_solve_batch([plan], [it])
    s1 = it["s_out"].cpu().numpy()
    r2 = wf.wf_solve_batch([plan], [it])
    assert r1[0]["status"] == r2[0]["status"] == wf.WF_OK and r1[0]["iters"] == r2[0]["iters"]
    assert rel(it["s_out"].cpu().numpy(), s1) < 1e-12
    plan.close()


def test_batch_rejections(wf):
    n, l, p, k, t = CASES[0]
    it = _item(0, n, l, k, t)
    plan = wf.wf_plan_create("healpix", nside=n, lmax=l, precision=p)
    with pytest.raises(wf.WfError) as e:
        wf.wf_solve_batch([plan, plan], [it, it])
    assert e.value.status == wf.WF_EINVAL
    wf.wf_set_options(plan, schedule=1)
    with pytest.raises(wf.WfError) as e:
        wf.wf_solve_batch([plan], [it])
    assert e.value.status == wf.WF_EUNSUPPORTED
    plan.close()


def test_autotuned_tiles_keep_the_results(wf):
    """The autotuner picks one of the tile variants (2, 4 or 8 ring pairs) and
    the solve on the tuned plan matches the default-tile solve within the
    mixed-precision tolerance; FP64 plans are left alone."""
    import torch

    n, l, p, k, t = 64, 128, "mixed", "wf", 1e-5
    it = _item(40, n, l, k, t)
    ref, rep_ref = _alone(wf, n, l, p, it)
    plan = wf.wf_plan_create("healpix", nside=n, lmax=l, precision=p)
    assert wf.wf_plan_tiles(plan) == (4, 8)
    tiles = wf.wf_plan_autotune(plan, reps=2)
    assert tiles[0] in (2, 4, 8) and tiles[1] in (2, 4, 8)
    s = torch.empty_like(it["s_out"])
    rep = wf.wf_solve(plan, it["d"], it["noise_var"], it["mask"], it["C_ell"], t, s)
    assert rep["final_residual"] < t
    assert rel(s.cpu().numpy(), ref) < 1e-3
    plan.close()
    p64 = wf.wf_plan_create("healpix", nside=16, lmax=32, precision="fp64")
    assert wf.wf_plan_autotune(p64) == (4, 8)
    p64.close()


def test_batch_of_polarised_constrained_realisations(wf):
    """(I, Q, U) Wiener-filter and fluctuation solves of mixed nside, paired
    per map (a constrained realisation is s_WF + f), in one batch beside a
    temperature solve: each item equals the same solve run alone (FP64, to
    1e-10, same iterations and launch count)."""
    import torch

    from gpu_util import healpix_pol_case

    geoms = [(8, 16), (16, 32), (32, 64)]
    plans, items, alone = [], [], []
    for j, (nside, lmax) in enumerate(geoms):
        P, basis, d, nu, obs, N6, C4 = healpix_pol_case(nside, lmax, gen.seed_for(4, 300 + j))
        rng = np.random.default_rng(3000 + j)
        npx = 12 * nside * nside
        g1 = rng.standard_normal((3, npx))
        g2 = np.stack([gen.alm_unit_gaussian(rng, lmax) for _ in range(3)])
        for kind in ("wf", "fluct"):
            it = {"kind": kind, "noise_var": T(N6.ravel()), "mask": T(P["mask"]), "C_ell": T(C4.ravel()), "tol": 1e-7,
                  "s_out": torch.full((3 * npx,), float("nan"), dtype=torch.float64, device="cuda")}
            if kind == "wf":
                it["d"] = T(d.ravel())
            else:
                it["g1"] = T(g1.ravel())
                it["g2"] = T(g2.ravel())
            pl = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64", ncomp=3)
            s = torch.empty_like(it["s_out"])
            if kind == "wf":
                rep = wf.wf_solve(pl, it["d"], it["noise_var"], it["mask"], it["C_ell"], 1e-7, s, trace_cap=20000)
            else:
                rep = wf.wf_fluct(pl, it["noise_var"], it["mask"], it["C_ell"], it["g1"], it["g2"], 1e-7, s,
                                  trace_cap=20000)
            pl.close()
            alone.append((s.cpu().numpy(), rep))
            plans.append(wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision="fp64", ncomp=3))
            items.append(it)
    n, l, p, k, t = CASES[0]
    it = _item(0, n, l, k, t)
    alone.append(_alone(wf, n, l, p, it))
    plans.append(wf.wf_plan_create("healpix", nside=n, lmax=l, precision=p))
    items.append(it)
    reps = wf.wf_solve_batch(plans, items, trace_cap=20000)
    for i, (it, rep, (s_alone, rep_alone)) in enumerate(zip(items, reps, alone)):
        assert rep["status"] == wf.WF_OK, (i, rep["status"])
        assert rel(it["s_out"].cpu().numpy(), s_alone) < 1e-10, (i, rel(it["s_out"].cpu().numpy(), s_alone))
        assert rep["iters"] == rep_alone["iters"]
        np.testing.assert_array_equal(rep["lambda_trace"], rep_alone["lambda_trace"])
        assert rep["launches"] == rep_alone["launches"] > 0
    for pl in plans:
        pl.close()
