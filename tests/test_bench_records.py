"""The benchmark's derived records, on hand-made traces (no GPU): the time to
each residual, and the paper's own stopping point (Sect. 3: the first lambda =
1, full-band iteration whose chi^2 moved by less than 1e-4 sigma_chi2), which
must ignore the iterations of the correction form, whose chi^2 is NaN."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rep(chi2, lam, L, resid, ms, n_dof=20000):
    return {"chi2_trace": np.array(chi2, dtype=float), "lambda_trace": np.array(lam, dtype=float),
            "L_trace": np.array(L), "resid_trace": np.array(resid, dtype=float),
            "iter_ms_trace": np.array(ms, dtype=float), "n_dof": n_dof}


def test_time_to_residual_takes_the_first_crossing():
    rep = _rep([1.0] * 5, [1.0] * 5, [8] * 5, [2e-2, 5e-3, 2e-4, 9e-5, 5e-5], [10.0, 10.0, np.nan, 10.0, 10.0])
    out = bench.time_to_residual(rep)
    assert out["0.01"] == {"s": 0.02, "iters": 2}
    assert out["0.0001"] == {"s": 0.03, "iters": 4}  # a NaN time (profiling off) counts as 0
    assert out["1e-05"] is None and out["1e-06"] is None


def test_paper_stop_uses_consecutive_full_band_lambda_one_chi2():
    sig = math.sqrt(2.0 * 20000)
    small, big = 0.5e-4 * sig, 10.0 * sig
    lmax = 8
    # iteration 1 -> 2 moves little but iteration 1 is band-limited; 3 -> 4 is the first valid stop
    chi2 = [100.0, 100.0 + big, 100.0 + big + small, 200.0, 200.0 + small, 200.0 + 2 * small]
    lam = [4.0, 1.0, 1.0, 1.0, 1.0, 1.0]
    L = [4, 4, lmax, lmax, lmax, lmax]
    rep = _rep(chi2, lam, L, [np.nan] * 2 + [1e-3] * 4, [1.0] * 6)
    out = bench.time_to_dchi2(rep, lmax)
    assert out["iters"] == 5 and out["s"] == 0.005 and out["residual"] == 1e-3


def test_paper_stop_ignores_the_correction_form_iterations():
    sig = math.sqrt(2.0 * 20000)
    lmax = 8
    # chi^2 keeps moving until the switch; from there the trace holds NaN (no chi^2 of delta)
    chi2 = [0.0, 10.0 * sig, 20.0 * sig, np.nan, np.nan, np.nan]
    rep = _rep(chi2, [1.0] * 6, [lmax] * 6, [1e-2, 5e-3, 2e-3, 1e-3, 5e-4, 2e-4], [1.0] * 6)
    assert bench.time_to_dchi2(rep, lmax) is None
