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


def healpix_pol_case(nside, lmax, seed, corr=0.1, **kw):
    """Polarised problem + (I, Q, U) data made with the oracle's synthesis, the
    inverse noise blocks, and the device layouts: N6 (6 x npix: II, QQ, UU,
    IQ, IU, QU) and C4 (4 x (lmax + 1): TT, EE, BB, TE)."""
    from oracle.messenger_pol import HealpixPolBasis

    kw.setdefault("fwhm_arcmin", 4 * 3438.0 / lmax)
    kw.setdefault("n_disks", 6)
    kw.setdefault("disk_radius_deg", 6.0)
    P = gen.healpix_pol_problem(nside, lmax, seed, corr=corr, **kw)
    basis = HealpixPolBasis(nside, lmax)
    d = basis.synth(P["a_signal"]) + P["noise"]
    obs = P["mask"] > 0
    nu = np.zeros_like(P["noise_cov"])
    nu[obs] = np.linalg.inv(P["noise_cov"][obs])
    Nc = P["noise_cov"]
    N6 = np.stack([Nc[:, 0, 0], Nc[:, 1, 1], Nc[:, 2, 2], Nc[:, 0, 1], Nc[:, 0, 2], Nc[:, 1, 2]])
    C4 = np.ascontiguousarray(P["c_ell"].T)
    return P, basis, d, nu, obs, N6, C4


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
