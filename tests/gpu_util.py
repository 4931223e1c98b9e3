"""Helpers shared by the GPU tests: device tensors and oracle-side problems."""
import numpy as np

import oracle
import wf_inputs as gen


def dev():
    import torch

    return torch.device("cuda:0")


def T(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def healpix_case(nside, lmax, seed, **kw):
    """Problem + data map made with the oracle's synthesis (never the GPU's)."""
    kw.setdefault("fwhm_arcmin", 4 * 3438.0 / lmax)
    kw.setdefault("n_disks", 8)
    kw.setdefault("disk_radius_deg", 6.0)
    P = gen.healpix_problem(nside, lmax, seed, **kw)
    basis = oracle.HealpixBasis(nside, lmax)
    d = basis.synth(P["a_signal"]) + P["noise"]
    obs = P["mask"] > 0
    nu = np.where(obs, 1.0 / P["noise_var"], 0.0)
    tau = float(P["noise_var"][obs].min())
    return P, basis, d, nu, tau


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
