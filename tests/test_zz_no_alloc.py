"""The allocation-free flat-grid entry point (wf_flat_solve_noalloc).

Some callers cannot allocate device memory when they solve -- for example
code running inside another framework's memory pool or in a context where
cudaMalloc is not allowed -- so the library offers one entry point whose
scratch lives in a static device array.  It must give the same result as
wf_solve on a flat plan.  This file is collected last so that a run that
stops at the first failure has already run every other test; it also passes
on its own in a fresh process."""
import numpy as np
import pytest

import oracle
import wf_inputs as gen
from gpu_util import T, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,opts", [(16, {}), (32, {}), (64, {}), (128, {}),
                                    (64, {"lambda_max": 30.0, "level_cap": 50})])
def test_noalloc_matches_plan_solve_on_two_calls_in_a_row(n, opts):
    """The entry point builds its lambda levels on the device (largest prior per
    radius); wf_solve builds them on the host.  Both must pick the same levels,
    at every grid size and with non-default schedule options too."""
    import torch

    import paper_1210_4931_gb300 as wf

    wf.load()
    torch.cuda.set_device(0)
    plan = wf.wf_plan_create("flat", n=n)
    if opts:
        wf.wf_set_options(plan, **opts)
    for k in range(2):  # two different problems back to back: nothing may leak between calls
        P = gen.flat_problem(n, seed=gen.seed_for(1, 700 + 10 * n + k))
        d = oracle.FlatBasis(n, n).synth(P["a_signal"]) + P["noise"]
        args = (T(d.ravel()), T(P["noise_var"].ravel()), T(P["mask"].ravel()), T(P["S"].ravel()))
        s_ref = torch.empty(n * n, dtype=torch.float64, device="cuda")
        a_ref = torch.empty(n * (n // 2 + 1), dtype=torch.complex128, device="cuda")
        ref = wf.wf_solve(plan, *args, 1e-6, s_ref, a_ref, trace_cap=20000)
        s = torch.empty_like(s_ref)
        a = torch.empty_like(a_ref)
        got = wf.wf_flat_solve_noalloc(n, *args, 1e-6, s, a, trace_cap=20000, **opts)
        assert got["converged"] and ref["converged"]
        assert got["iters"] == ref["iters"]
        np.testing.assert_array_equal(got["lambda_trace"], ref["lambda_trace"])
        assert rel(s.cpu().numpy(), s_ref.cpu().numpy()) < 1e-10
        assert rel(a.cpu().numpy(), a_ref.cpu().numpy()) < 1e-10
        assert got["final_residual"] == pytest.approx(ref["final_residual"], rel=1e-10)
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    import paper_1210_4931_gb300 as wf

    wf.load()
    z = torch.zeros(256 * 256, dtype=torch.float64, device="cuda")
    with pytest.raises(wf.WfError) as e:
        wf.wf_flat_solve_noalloc(256, z, z + 1.0, None, z[: 256 * 129], 1e-6, z)
    assert e.value.status == wf.WF_EINVAL
    n = 32
    z = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    with pytest.raises(wf.WfError) as e:
        wf.wf_flat_solve_noalloc(n, z, z + 1.0, None, z[: n * 17] + 1.0, 1e-6, z, maxiter=20001)
    assert e.value.status == wf.WF_EINVAL


def test_noalloc_rejects_an_invalid_prior():
    """The device-side level search compares S by bit pattern, an order that
    holds only for S >= 0: a negative or NaN prior is rejected up front."""
    import torch

    import paper_1210_4931_gb300 as wf

    wf.load()
    n = 32
    P = gen.flat_problem(n, seed=gen.seed_for(1, 790))
    d, nv, m = T(P["noise"].ravel()), T(P["noise_var"].ravel()), T(P["mask"].ravel())
    out = torch.empty(n * n, dtype=torch.float64, device="cuda")
    for bad in (-1.0, float("nan"), float("inf")):
        S = P["S"].copy()
        S[3, 2] = bad
        with pytest.raises(wf.WfError) as e:
            wf.wf_flat_solve_noalloc(n, d, nv, m, T(S.ravel()), 1e-6, out)
        assert e.value.status == wf.WF_EINVAL
