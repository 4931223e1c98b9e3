"""Several data sets of one signal (the outlook of Sect. 4) through the C ABI:
the device combination equals the oracle's per pixel, and the messenger solve
on it matches the oracle's solve of the same combined data (schedule replay,
FP64, 1e-10); the oracle's combination is itself pinned against dense solves
of the stacked system (tests/test_oracle_datasets.py)."""
import numpy as np
import pytest

import oracle
import wf_inputs as gen
from gpu_util import T, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf():
    import torch

    import paper_1210_4931_gb300 as w

    w.load()
    torch.cuda.set_device(0)
    return w


def _datasets(nside, lmax, k, seed):
    P = gen.healpix_problem(nside, lmax, seed, fwhm_arcmin=4 * 3438.0 / lmax, n_disks=8, disk_radius_deg=6.0)
    basis = oracle.HealpixBasis(nside, lmax)
    sig = basis.synth(P["a_signal"])
    rng = np.random.default_rng(seed + 5)
    npix = sig.size
    ds, ns, ms = [], [], []
    for j in range(k):
        nv = P["noise_var"] * (1.0 + j) * rng.uniform(0.5, 2.0, size=npix)
        mk = P["mask"].copy() if j == 0 else (rng.uniform(size=npix) > 0.2 + 0.1 * j).astype(np.uint8)
        d = sig + np.sqrt(nv) * rng.standard_normal(npix)
        nv[mk == 0] = np.nan  # masked pixels may hold anything
        ds.append(d)
        ns.append(nv)
        ms.append(mk)
    return P, basis, ds, ns, ms


def test_combination_matches_oracle_and_solve_matches_oracle_replay(wf):
    import torch

    nside, lmax, k = 16, 32, 3
    P, basis, ds, ns, ms = _datasets(nside, lmax, k, gen.seed_for(2, 321))
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax)
    npix = plan.npix
    d_out = torch.empty(npix, dtype=torch.float64, device="cuda")
    n_out = torch.empty(npix, dtype=torch.float64, device="cuda")
    m_out = torch.empty(npix, dtype=torch.uint8, device="cuda")
    wf.wf_combine_datasets(plan, [T(x) for x in ds], [T(x) for x in ns], [T(x) for x in ms], d_out, n_out, m_out)
    d_ref, n_ref, m_ref = oracle.combine_datasets(ds, ns, ms)
    assert np.array_equal(m_out.cpu().numpy(), m_ref)
    assert rel(d_out.cpu().numpy(), d_ref) < 1e-14 and rel(n_out.cpu().numpy(), n_ref) < 1e-14
    s = torch.empty(npix, dtype=torch.float64, device="cuda")
    rep = wf.wf_solve(plan, d_out, n_out, m_out, T(P["c_ell"]), 1e-8, s, trace_cap=20000)
    assert rep["converged"]
    obs = m_ref > 0
    nu = np.where(obs, 1.0 / n_ref, 0.0)
    tau = float(n_ref[obs].min())
    ref = oracle.messenger_solve(basis, nu * d_ref, nu, basis.per_mode(P["c_ell"]), tau,
                                 replay=list(zip(rep["lambda_trace"], rep["L_trace"])))
    assert rel(s.cpu().numpy(), ref["s"]) < 1e-10
    plan.close()


def test_combination_rejections_and_single_dataset(wf):
    import torch

    nside, lmax = 8, 16
    P, basis, ds, ns, ms = _datasets(nside, lmax, 2, gen.seed_for(2, 322))
    plan = wf.wf_plan_create("healpix", nside=nside, lmax=lmax)
    npix = plan.npix
    d_out = torch.empty(npix, dtype=torch.float64, device="cuda")
    n_out = torch.empty(npix, dtype=torch.float64, device="cuda")
    m_out = torch.empty(npix, dtype=torch.uint8, device="cuda")
    # one data set, no mask: unchanged
    nv0 = np.abs(ns[0])
    nv0[~np.isfinite(nv0)] = 1.0
    wf.wf_combine_datasets(plan, [T(ds[0])], [T(nv0)], None, d_out, n_out, m_out)
    assert rel(d_out.cpu().numpy(), ds[0]) < 1e-15 and rel(n_out.cpu().numpy(), nv0) < 1e-15
    assert bool(torch.all(m_out == 1))
    bad = ns[1].copy()
    bad[np.nonzero(ms[1])[0][2]] = -1.0
    with pytest.raises(wf.WfError) as e:
        wf.wf_combine_datasets(plan, [T(x) for x in ds], [T(ns[0]), T(bad)], [T(x) for x in ms], d_out, n_out,
                               m_out)
    assert e.value.status == wf.WF_EINVAL
    with pytest.raises(wf.WfError) as e:
        wf.wf_combine_datasets(plan, [T(ds[0])] * 17, [T(nv0)] * 17, None, d_out, n_out, m_out)
    assert e.value.status == wf.WF_EINVAL
    plan.close()
