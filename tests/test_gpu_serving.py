"""Request loop (wf_server_*): many Wiener-filter, fluctuation and
constrained-realization requests of mixed size, admitted by device memory and
run concurrently.  Each result must equal the same request run alone through
the direct host entry points (wf_solve_host / wf_fluct_host) on a fresh plan:
to 1e-10 relative in FP64 (the analysis sums use atomics, so runs may differ
in the last bits), and for mixed precision to within the solve tolerance
(relative map difference below 1e-3 with both residuals below tol)."""
import numpy as np
import pytest

import wf_inputs as gen
from gpu_util import healpix_case, rel

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
    (32, 64, "fp64", "cr", 1e-7),
    (64, 128, "mixed", "wf", 1e-5),
    (16, 32, "fp64", "fluct", 1e-8),
    (32, 64, "mixed", "cr", 1e-5),
    (64, 128, "fp64", "wf", 1e-7),
]


def _request(i, nside, lmax, kind):
    P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(5, i))
    rng = np.random.default_rng(1000 + i)
    g1 = rng.standard_normal(d.size)
    g2 = np.ascontiguousarray(gen.alm_unit_gaussian(rng, lmax), dtype=np.complex128)
    return dict(d=np.ascontiguousarray(d), noise_var=np.ascontiguousarray(P["noise_var"]),
                mask=np.ascontiguousarray(P["mask"]), C_ell=np.ascontiguousarray(P["c_ell"]), g1=g1, g2=g2)


def _alone(w, nside, lmax, prec, kind, tol, R):
    plan = w.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=prec)
    s = np.empty(R["d"].size)
    if kind in ("wf", "cr"):
        rep = w.wf_solve_host(plan, R["d"], R["noise_var"], R["mask"], R["C_ell"], tol, s)
    if kind in ("fluct", "cr"):
        f = np.empty(R["d"].size)
        rep = w.wf_fluct_host(plan, R["noise_var"], R["mask"], R["C_ell"], R["g1"], R["g2"], tol, f)
        s = f if kind == "fluct" else s + f
    plan.close()
    return s, rep


def test_results_in_the_mix_equal_results_alone(wf):
    reqs = [_request(i, n, l, k) for i, (n, l, p, k, t) in enumerate(CASES)]
    alone = [_alone(wf, n, l, p, k, t, R) for (n, l, p, k, t), R in zip(CASES, reqs)]
    srv = wf.Server(mem_budget=4 << 30, slots=4)
    outs = {}
    for rep_round in range(2):  # twice: the second round reuses the pooled plans
        for i, ((n, l, p, k, t), R) in enumerate(zip(CASES, reqs)):
            out = np.full(R["d"].size, np.nan)
            tag = 100 * rep_round + i
            outs[tag] = out
            srv.submit(k, nside=n, lmax=l, precision=p, tol=t, s_out=out, tag=tag,
                       **{key: R[key] for key in ("d", "noise_var", "mask", "C_ell", "g1", "g2")})
    results = {}
    while len(results) < 2 * len(CASES):
        for r in srv.wait(timeout=60.0):
            results[r["tag"]] = r
    st = srv.stats()
    srv.close()
    assert st["completed"] == 2 * len(CASES) and st["rejected"] == 0
    assert st["plans_created"] <= len({(n, l, p) for n, l, p, k, t in CASES}) * 4
    for tag, r in results.items():
        i = tag % 100
        n, l, p, k, t = CASES[i]
        assert r["status"] == wf.WF_OK, (tag, r)
        s_alone, rep = alone[i]
        if p == "fp64":
            assert rel(outs[tag], s_alone) < 1e-10, (tag, rel(outs[tag], s_alone))
        else:
            assert r["final_residual"] < t and rep["final_residual"] < t
            assert rel(outs[tag], s_alone) < 1e-3, (tag, rel(outs[tag], s_alone))
        assert r["t_submit"] <= r["t_start"] <= r["t_done"]
    assert any(r["plan_reused"] for r in results.values())


def test_plan_size_estimate_bounds_the_measured_size(wf):
    for nside, prec in ((16, "fp64"), (64, "mixed"), (128, "mixed"), (128, "fp64")):
        lmax = 2 * nside
        R = _request(50 + nside, nside, lmax, "wf")
        plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=prec)
        s = np.empty(R["d"].size)
        wf.wf_solve_host(plan, R["d"], R["noise_var"], R["mask"], R["C_ell"], 1e-5, s)
        f = np.empty(R["d"].size)
        wf.wf_fluct_host(plan, R["noise_var"], R["mask"], R["C_ell"], R["g1"], R["g2"], 1e-5, f)
        actual = plan.device_bytes
        est = wf.wf_plan_estimate_bytes("healpix", nside=nside, lmax=lmax, precision=prec)
        plan.close()
        assert actual <= est <= 1.6 * actual + (4 << 20), (nside, prec, actual, est)


def test_admission_keeps_the_memory_budget(wf):
    # two keys of nearly equal size and a budget that holds one plan: every
    # change of key must evict the idle plan of the other
    geoms = [(64, 128), (64, 126)] * 3
    budget = max(wf.wf_plan_estimate_bytes("healpix", nside=n, lmax=l, precision="mixed") for n, l in geoms[:2])
    budget += 1 << 20
    srv = wf.Server(mem_budget=budget, slots=3)
    reqs = [_request(60 + i, n, l, "wf") for i, (n, l) in enumerate(geoms)]
    outs = []
    for i, ((n, l), R) in enumerate(zip(geoms, reqs)):
        out = np.empty(R["d"].size)
        outs.append(out)
        srv.submit("wf", nside=n, lmax=l, precision="mixed", tol=1e-4, s_out=out, tag=i, d=R["d"],
                   noise_var=R["noise_var"], mask=R["mask"], C_ell=R["C_ell"])
    got = []
    while len(got) < len(geoms):
        got += srv.wait(timeout=60.0)
    st = srv.stats()
    srv.close()
    assert all(r["status"] == wf.WF_OK for r in got), got
    assert st["peak_bytes"] <= budget
    assert st["plans_evicted"] >= 1 and st["max_active"] == 1


def test_requests_overlap_on_the_device(wf):
    srv = wf.Server(mem_budget=4 << 30, slots=4)
    reqs = [_request(70 + i, 64, 128, "wf") for i in range(8)]
    outs = []
    for i, R in enumerate(reqs):
        out = np.empty(R["d"].size)
        outs.append(out)
        srv.submit("wf", nside=64, lmax=128, precision="mixed", tol=1e-5, s_out=out, tag=i, d=R["d"],
                   noise_var=R["noise_var"], mask=R["mask"], C_ell=R["C_ell"])
    got = []
    while len(got) < len(reqs):
        got += srv.wait(timeout=60.0)
    st = srv.stats()
    srv.close()
    assert all(r["status"] == wf.WF_OK for r in got)
    assert st["max_active"] >= 2
    spans = sorted((r["t_start"], r["t_done"]) for r in got)
    assert any(b[0] < a[1] for a, b in zip(spans, spans[1:]))  # some solves ran at the same time


def test_invalid_and_oversized_requests_are_rejected(wf):
    srv = wf.Server(mem_budget=64 << 20, slots=2)
    R = _request(80, 16, 32, "wf")
    out = np.empty(R["d"].size)
    srv.submit("wf", nside=16, lmax=40, precision="fp64", tol=1e-6, s_out=out, tag=1, d=R["d"],
               noise_var=R["noise_var"], C_ell=R["C_ell"])
    big = np.empty(12 * 1024 * 1024)
    srv.submit("wf", nside=1024, lmax=2048, precision="mixed", tol=1e-6, s_out=big, tag=2, d=big,
               noise_var=big, C_ell=np.ones(2049))
    got = {}
    while len(got) < 2:
        for r in srv.wait(timeout=10.0):
            got[r["tag"]] = r
    st = srv.stats()
    srv.close()
    assert got[1]["status"] == wf.WF_EINVAL and got[2]["status"] == wf.WF_ENOMEM
    assert st["rejected"] == 2 and st["plans_created"] == 0


def _pol_request(i, nside, lmax):
    from gpu_util import healpix_pol_case

    P, basis, d, nu, obs, N6, C4 = healpix_pol_case(nside, lmax, gen.seed_for(5, 200 + i))
    rng = np.random.default_rng(3000 + i)
    npx = 12 * nside * nside
    g1 = rng.standard_normal((3, npx))
    g2 = np.stack([gen.alm_unit_gaussian(rng, lmax) for _ in range(3)])
    return dict(d=np.ascontiguousarray(d.ravel()), noise_var=np.ascontiguousarray(N6.ravel()),
                mask=np.ascontiguousarray(P["mask"]), C_ell=np.ascontiguousarray(C4.ravel()),
                g1=np.ascontiguousarray(g1.ravel()), g2=np.ascontiguousarray(g2.ravel()))


POL_CASES = [  # nside, lmax, precision, kind, tol
    (8, 16, "fp64", "wf", 1e-8),
    (16, 32, "fp64", "cr", 1e-7),
    (16, 32, "mixed", "fluct", 1e-5),
    (32, 64, "mixed", "cr", 1e-5),
]


def test_polarised_requests_in_the_mix(wf):
    """(I, Q, U) Wiener-filter, fluctuation and constrained-realization
    requests (ncomp = 3) beside temperature ones: each result equals the same
    request run alone through the direct host entry points on a fresh plan."""
    reqs = [_pol_request(i, n, l) for i, (n, l, p, k, t) in enumerate(POL_CASES)]
    alone = []
    for (n, l, p, k, t), R in zip(POL_CASES, reqs):
        plan = wf.wf_plan_create("healpix", nside=n, lmax=l, precision=p, ncomp=3)
        s = np.empty(R["d"].size)
        if k in ("wf", "cr"):
            rep = wf.wf_solve_host(plan, R["d"], R["noise_var"], R["mask"], R["C_ell"], t, s)
        if k in ("fluct", "cr"):
            f = np.empty(R["d"].size)
            rep = wf.wf_fluct_host(plan, R["noise_var"], R["mask"], R["C_ell"], R["g1"], R["g2"], t, f)
            s = f if k == "fluct" else s + f
        plan.close()
        alone.append((s, rep))
    T_req = _request(90, 32, 64, "wf")
    srv = wf.Server(mem_budget=4 << 30, slots=3)
    outs = {}
    for i, ((n, l, p, k, t), R) in enumerate(zip(POL_CASES, reqs)):
        outs[i] = np.full(R["d"].size, np.nan)
        srv.submit(k, nside=n, lmax=l, precision=p, tol=t, s_out=outs[i], tag=i, ncomp=3,
                   **{key: R[key] for key in ("d", "noise_var", "mask", "C_ell", "g1", "g2")})
    outT = np.full(T_req["d"].size, np.nan)
    srv.submit("wf", nside=32, lmax=64, precision="mixed", tol=1e-5, s_out=outT, tag=99, d=T_req["d"],
               noise_var=T_req["noise_var"], mask=T_req["mask"], C_ell=T_req["C_ell"])
    got = {}
    while len(got) < len(POL_CASES) + 1:
        for r in srv.wait(timeout=60.0):
            got[r["tag"]] = r
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(POL_CASES) + 1 and st["rejected"] == 0
    assert got[99]["status"] == wf.WF_OK
    for i, (n, l, p, k, t) in enumerate(POL_CASES):
        r = got[i]
        assert r["status"] == wf.WF_OK, (i, r)
        s_alone, rep = alone[i]
        if p == "fp64":
            assert rel(outs[i], s_alone) < 1e-10, (i, rel(outs[i], s_alone))
        else:
            assert r["final_residual"] < t and rep["final_residual"] < t
            assert rel(outs[i], s_alone) < 1e-3, (i, rel(outs[i], s_alone))


def test_polarised_plan_size_estimate(wf):
    """The estimate bounds the measured size of polarised plans after a Wiener
    filter and a fluctuation solve through the host entry points."""
    for nside, prec in ((16, "fp64"), (64, "mixed"), (64, "fp64")):
        lmax = 2 * nside
        R = _pol_request(300 + nside, nside, lmax)
        plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax, precision=prec, ncomp=3)
        s = np.empty(R["d"].size)
        wf.wf_solve_host(plan, R["d"], R["noise_var"], R["mask"], R["C_ell"], 1e-4, s)
        f = np.empty(R["d"].size)
        wf.wf_fluct_host(plan, R["noise_var"], R["mask"], R["C_ell"], R["g1"], R["g2"], 1e-4, f)
        actual = plan.device_bytes
        est = wf.wf_plan_estimate_bytes("healpix", nside=nside, lmax=lmax, precision=prec, ncomp=3)
        plan.close()
        assert actual <= est <= 1.6 * actual + (4 << 20), (nside, prec, actual, est)


@pytest.mark.parametrize("prec,tol,bound", [("fp64", 1e-11, 1e-8), ("mixed", 1e-5, 1e-3), ("tf32", 1e-5, 1e-3)])
def test_served_request_matches_oracle(wf, prec, tol, bound):
    """A Wiener-filter request served by the request loop against the oracle's
    own solve of the same data (its heuristic schedule, run to a tighter tol):
    both converge to the same discrete fixed point, so the maps agree to the
    tolerance's accuracy."""
    import oracle

    nside, lmax = 16, 32
    P, basis, d, nu, tau = healpix_case(nside, lmax, gen.seed_for(5, 90))
    srv = wf.Server(device=0, mem_budget=1 << 30, slots=2)
    out = np.empty(d.size)
    srv.submit("wf", nside=nside, lmax=lmax, precision=prec, tol=tol, s_out=out, tag=1, d=np.ascontiguousarray(d),
               noise_var=np.ascontiguousarray(P["noise_var"]), mask=np.ascontiguousarray(P["mask"]),
               C_ell=np.ascontiguousarray(P["c_ell"]))
    res = []
    while not res:
        res = srv.wait(timeout=5.0)
    srv.close()
    assert res[0]["status"] == wf.WF_OK and res[0]["converged"]
    sched = oracle.messenger.HealpixSchedule(P["c_ell"], tau * basis.omega, lmax)
    ref = oracle.messenger_solve(basis, nu * d, nu, basis.per_mode(P["c_ell"]), tau, schedule=sched, tol=1e-12)
    assert ref["converged"]
    assert rel(out, ref["s"]) < bound
