"""Pins for the multi-dataset reduction (outlook of Sect. 4): the messenger
iteration on the combined data set equals a dense solve of the STACKED
Wiener-filter system, built from explicit DFT matrices (flat 16 x 16) or
scipy's Y_lm (HEALPix nside 4), never from the combination itself."""
import math

import numpy as np
import pytest
from scipy import special as sp

import wf_inputs as gen


def _dft2(n):
    j = np.arange(n)
    f = np.exp(-2j * np.pi * np.outer(j, j) / n) / math.sqrt(n)
    return np.kron(f, f)


def _full_plane(S_half, n):
    full = np.empty((n, n))
    h = n // 2 + 1
    full[:, :h] = S_half
    ky = (-np.arange(n)) % n
    for kx in range(h, n):
        full[:, kx] = S_half[ky, n - kx]
    return full


def _three_datasets(n, seed):
    """Three data sets of one signal: own noise levels and masks (each leaves
    different pixels unobserved; a few pixels are seen by none)."""
    P = gen.flat_problem(n, seed=seed, band_rows=(7, 9), n_disks=2, disk_radius=1.5)
    rng = np.random.default_rng(seed + 1)
    sig = np.fft.irfft2(P["a_signal"], s=(n, n), norm="ortho")
    ds, ns, ms = [], [], []
    for k in range(3):
        nv = 10.0 ** rng.uniform(-2.0 + 0.5 * k, 0.0, size=(n, n))
        mk = np.ones((n, n), dtype=np.uint8)
        mk[rng.uniform(size=(n, n)) < 0.25] = 0
        ds.append(sig + np.sqrt(nv) * rng.standard_normal((n, n)))
        ns.append(nv)
        ms.append(mk)
    ms[0][3, 3] = ms[1][3, 3] = ms[2][3, 3] = 0  # a pixel no data set observes
    return P, ds, ns, ms


def test_combination_per_pixel_definition(oracle):
    P, ds, ns, ms = _three_datasets(8, 41)
    d, nv, mk = oracle.combine_datasets([x.ravel() for x in ds], [x.ravel() for x in ns],
                                        [x.ravel() for x in ms])
    i = 5 * 8 + 2
    obs = [k for k in range(3) if ms[k].ravel()[i]]
    w = sum(1.0 / ns[k].ravel()[i] for k in obs)
    assert nv[i] == pytest.approx(1.0 / w, rel=1e-15)
    assert d[i] == pytest.approx(sum(ds[k].ravel()[i] / ns[k].ravel()[i] for k in obs) / w, rel=1e-14)
    assert mk[3 * 8 + 3] == 0 and d[3 * 8 + 3] == 0.0
    # one data set: unchanged where observed
    d1, n1, m1 = oracle.combine_datasets([ds[0].ravel()], [ns[0].ravel()], [ms[0].ravel()])
    o = ms[0].ravel() > 0
    assert np.array_equal(m1, ms[0].ravel()) and np.allclose(d1[o], ds[0].ravel()[o], rtol=1e-15)


def test_flat_messenger_on_combined_data_solves_the_stacked_system(oracle):
    n = 16
    P, ds, ns, ms = _three_datasets(n, 42)
    d, nv, mk = oracle.combine_datasets([x.ravel() for x in ds], [x.ravel() for x in ns],
                                        [x.ravel() for x in ms])
    obs = mk > 0
    nu = np.where(obs, 1.0 / nv, 0.0)
    tau = float(nv[obs].min())
    B = oracle.FlatBasis(n, n)
    res = oracle.messenger_solve(B, (nu * d).reshape(n, n), nu.reshape(n, n), P["S"], tau, tol=1e-12)
    assert res["converged"]
    # dense stacked system: (S^-1 + sum_k M_k N_k^-1 M_k) s = sum_k M_k N_k^-1 d_k
    F = _dft2(n)
    Sf = _full_plane(P["S"], n).ravel()
    Sinv = (F.conj().T @ np.diag(1.0 / Sf) @ F).real
    A = Sinv.copy()
    rhs = np.zeros(n * n)
    for k in range(3):
        w = np.where(ms[k].ravel() > 0, 1.0 / ns[k].ravel(), 0.0)
        A += np.diag(w)
        rhs += w * ds[k].ravel()
    s_ref = np.linalg.solve(A, rhs)
    assert np.max(np.abs(res["s"].ravel() - s_ref)) / np.max(np.abs(s_ref)) < 1e-9


def test_healpix_combined_data_fixed_point_is_the_stacked_one(oracle):
    """HEALPix nside 4: the discrete fixed point of the iteration on the
    combined data equals the dense solution of the stacked discrete system
    [S^-1 + sum_k Y^T N_k^-1 Y + (I - Omega Y^T Y)/(tau Omega)] a = sum_k Y^T N_k^-1 d_k."""
    nside, lmax = 4, 8
    P = gen.healpix_problem(nside, lmax, seed=61, fwhm_arcmin=60.0, b_cut_deg=20.0, n_disks=2,
                            disk_radius_deg=15.0, noise_level_ell=lmax)
    basis = oracle.HealpixBasis(nside, lmax)
    sig = basis.synth(P["a_signal"])
    rng = np.random.default_rng(62)
    npix = sig.size
    ds, ns, ms = [], [], []
    for k in range(2):
        nv = P["noise_var"] * (1.0 + 2.0 * k) * rng.uniform(0.5, 1.5, size=npix)
        mk = P["mask"].copy() if k == 0 else (rng.uniform(size=npix) > 0.3).astype(np.uint8)
        ds.append(sig + np.sqrt(nv) * rng.standard_normal(npix))
        ns.append(nv)
        ms.append(mk)
    d, nv, mk = oracle.combine_datasets(ds, ns, ms)
    obs = mk > 0
    nu = np.where(obs, 1.0 / nv, 0.0)
    tau = float(nv[obs].min())
    om = basis.omega
    S = basis.per_mode(P["c_ell"])
    sched = oracle.messenger.HealpixSchedule(P["c_ell"], tau * om, lmax)
    res = oracle.messenger_solve(basis, nu * d, nu, S, tau, schedule=sched, tol=1e-12)
    assert res["converged"]
    th, ph = oracle.pixel_angles(nside)
    l, m = oracle.alm_lm(lmax)
    cols, W, modes = [], [], []
    for k in range(l.size):
        Y = sp.sph_harm_y(int(l[k]), int(m[k]), th, ph)
        if m[k] == 0:
            cols.append(Y.real)
            W.append(1.0)
            modes.append((k, 0))
        else:
            cols += [2 * Y.real, -2 * Y.imag]
            W += [2.0, 2.0]
            modes += [(k, 0), (k, 1)]
    Y = np.array(cols).T
    W = np.array(W)
    Sx = np.array([S[k] for k, _ in modes])
    act = Sx > 0
    Yt = Y.T / W[:, None]
    Mx = np.diag(1.0 / Sx[act]) + (np.eye(act.sum()) - om * (Yt @ Y)[np.ix_(act, act)]) / (tau * om)
    rhs = np.zeros(act.sum())
    for k in range(2):
        w = np.where(ms[k] > 0, 1.0 / ns[k], 0.0)
        Mx += (Yt @ (w[:, None] * Y))[np.ix_(act, act)]
        rhs += (Yt @ (w * ds[k]))[act]
    x_ref = np.linalg.solve(Mx, rhs)
    x = np.array([res["a"][k].real if p == 0 else res["a"][k].imag for k, p in modes])[act]
    assert np.max(np.abs(x - x_ref)) / np.max(np.abs(x_ref)) < 1e-9
