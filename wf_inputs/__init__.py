"""Seeded synthetic inputs for the messenger-field Wiener filter.

Shared by the tests, the oracle-side checks and the benchmark; it holds none
of the method's arithmetic: no transform, no blend, no schedule.  Every
function returns plain numpy arrays drawn from ``numpy.random.Generator``
(PCG64) with an explicit seed.  A signal *map* is never made here: the
generators return the signal's harmonic coefficients, and the caller turns
them into a map with whichever synthesis it is testing or timing.

Workloads (the paper's data, WMAP7 and simulated Planck maps, are not
available; these stand in for them with the same structure):

* ``flat_problem``    periodic n x n grid, P(k) = A / (k + 2)^2.5, noise
                      variance log-uniform over two decades, 8-row band plus
                      20 disks of radius 3 px masked.
* ``healpix_problem`` HEALPix RING map: CMB-like C_l with a Gaussian beam,
                      noise variance sigma0^2 / hits with hits rising towards
                      the ecliptic poles and lognormal jitter, a galactic cut
                      plus point-source disks.
"""
import math

import numpy as np

BASE_SEED = 12104931


def seed_for(config: int, k: int = 0) -> int:
    """Seed of draw ``k`` of workload ``config``."""
    return BASE_SEED + 1000 * config + k


# ---------------------------------------------------------------------------
# unit complex Gaussian draws in the two harmonic layouts
# ---------------------------------------------------------------------------
def flat_unit_gaussian(rng, ny: int, nx: int) -> np.ndarray:
    """Half-plane (ny, nx/2+1) complex coefficients of a real white field with
    unit variance per mode: E|g|^2 = 1 and g(-k) = conj(g(k)) where the half
    plane holds both k and -k (columns kx = 0 and kx = nx/2)."""
    h = nx // 2 + 1
    g = (rng.standard_normal((ny, h)) + 1j * rng.standard_normal((ny, h))) * math.sqrt(0.5)
    cols = [0] + ([nx // 2] if nx % 2 == 0 else [])
    for c in cols:
        col = g[:, c]
        col[0] = rng.standard_normal()
        if ny % 2 == 0:
            col[ny // 2] = rng.standard_normal()
        top = np.arange(1, (ny + 1) // 2)
        col[ny - top] = np.conj(col[top])
    return g


def alm_unit_gaussian(rng, lmax: int) -> np.ndarray:
    """a_lm (m >= 0, m-major) of a real white field: m = 0 real N(0, 1),
    m > 0 real and imaginary parts each N(0, 1/2)."""
    n = (lmax + 1) * (lmax + 2) // 2
    g = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * math.sqrt(0.5)
    g[: lmax + 1] = rng.standard_normal(lmax + 1)
    return g


def alm_ell(lmax: int) -> np.ndarray:
    """l of every stored a_lm (m-major)."""
    return np.concatenate([np.arange(m, lmax + 1) for m in range(lmax + 1)])


# ---------------------------------------------------------------------------
# flat sky
# ---------------------------------------------------------------------------
def flat_kabs(ny: int, nx: int) -> np.ndarray:
    ky = np.concatenate([np.arange(0, (ny + 1) // 2), np.arange(-(ny // 2), 0)]).astype(np.float64)
    kx = np.arange(nx // 2 + 1, dtype=np.float64)
    return np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)


def flat_problem(n: int = 128, seed: int = seed_for(1), k0: float = 2.0, slope: float = 2.5,
                 noise_decades: float = 2.0, band_rows=(60, 68), n_disks: int = 20,
                 disk_radius: float = 3.0, homogeneous: bool = False, masked: bool = True) -> dict:
    """Flat-sky workload on an n x n periodic grid.

    Returns S (per half-plane mode), noise_var, mask (1 = observed),
    a_signal (half-plane coefficients of the signal), noise (pixel noise
    draw), g1 and g2 (fluctuation draws) and the sizes.  ``homogeneous``
    makes the noise variance constant (all pixels equal to the lowest level).
    """
    rng = np.random.default_rng(seed)
    ny = nx = n
    k = flat_kabs(ny, nx)
    P = (k + k0) ** (-slope)
    w = np.full(P.shape, 2.0)
    w[:, 0] = 1.0
    if nx % 2 == 0:
        w[:, nx // 2] = 1.0
    A = ny * nx / float(np.sum(w * P))  # unit pixel variance of the signal
    S = A * P
    if homogeneous:
        noise_var = np.full((ny, nx), 10.0 ** (-noise_decades))
    else:
        noise_var = 10.0 ** rng.uniform(-noise_decades, 0.0, size=(ny, nx))
    mask = np.ones((ny, nx), dtype=np.uint8)
    if masked:
        lo, hi = band_rows
        lo, hi = min(lo, ny), min(hi, ny)
        mask[lo:hi, :] = 0
        yy, xx = np.mgrid[0:ny, 0:nx]
        for _ in range(n_disks):
            cy, cx = rng.uniform(0, ny), rng.uniform(0, nx)
            dy = np.abs(yy - cy)
            dy = np.minimum(dy, ny - dy)
            dx = np.abs(xx - cx)
            dx = np.minimum(dx, nx - dx)
            mask[dy * dy + dx * dx <= disk_radius * disk_radius] = 0
    a_signal = np.sqrt(S) * flat_unit_gaussian(rng, ny, nx)
    noise = np.sqrt(noise_var) * rng.standard_normal((ny, nx))
    g1 = rng.standard_normal((ny, nx))
    g2 = flat_unit_gaussian(rng, ny, nx)
    return {"kind": "flat", "ny": ny, "nx": nx, "S": S, "noise_var": noise_var, "mask": mask,
            "a_signal": a_signal, "noise": noise, "g1": g1, "g2": g2, "kabs": k}


# ---------------------------------------------------------------------------
# HEALPix sphere
# ---------------------------------------------------------------------------
# Rotation from equatorial (J2000) to galactic unit vectors (rows: galactic
# x, y, z).  The maps are in galactic coordinates; the ecliptic pole is the
# equatorial direction (RA 270 deg, Dec 90 deg - obliquity).
_EQ_TO_GAL = np.array([[-0.0548755604, -0.8734370902, -0.4838350155],
                       [0.4941094279, -0.4448296300, 0.7469822445],
                       [-0.8676661490, -0.1980763734, 0.4559837762]])
_OBLIQUITY_DEG = 23.4392911


def _ecliptic_pole_galactic() -> np.ndarray:
    dec = math.radians(90.0 - _OBLIQUITY_DEG)
    ra = math.radians(270.0)
    v = np.array([math.cos(dec) * math.cos(ra), math.cos(dec) * math.sin(ra), math.sin(dec)])
    return _EQ_TO_GAL @ v


def ring_layout(nside: int):
    """z, first-pixel longitude and pixel count of every HEALPix ring (the
    generator's own copy of the RING grid, used only to place masks and
    hit counts)."""
    R = 4 * nside - 1
    i = np.arange(1, R + 1)
    k = np.where(i <= 2 * nside, i, 4 * nside - i)
    cap = k < nside
    z = np.where(cap, 1.0 - k * k / (3.0 * nside * nside), 4.0 / 3.0 - 2.0 * i / (3.0 * nside))
    z = np.where(cap & (i > 2 * nside), -z, z)
    nr = np.where(cap, 4 * k, 4 * nside).astype(np.int64)
    phi0 = np.where(cap, np.pi / (4.0 * np.maximum(k, 1)),
                    np.where((i + nside) % 2 == 1, 0.0, np.pi / (4.0 * nside)))
    return z, phi0, nr


def cmb_like_cl(lmax: int, fwhm_arcmin: float, amp: float = 1.0) -> np.ndarray:
    """C_l = amp 2 pi / (l (l+1)) (1 + 0.3 sin(l / 45)) exp(-l^2 sigma_b^2),
    sigma_b = FWHM / sqrt(8 ln 2); C_0 = C_1 = 0 (monopole and dipole are not
    part of the signal model)."""
    ell = np.arange(lmax + 1, dtype=np.float64)
    sb = math.radians(fwhm_arcmin / 60.0) / math.sqrt(8.0 * math.log(2.0))
    with np.errstate(divide="ignore"):
        c = amp * 2.0 * np.pi / (ell * (ell + 1.0)) * (1.0 + 0.3 * np.sin(ell / 45.0)) * np.exp(-(ell * sb) ** 2)
    c[:2] = 0.0
    return c


def power_law_cl(lmax: int, slope: float, amp: float = 1.0) -> np.ndarray:
    ell = np.arange(lmax + 1, dtype=np.float64)
    with np.errstate(divide="ignore"):
        c = amp * ell ** (-slope)
    c[:2] = 0.0
    return c


def healpix_problem(nside: int, lmax: int, seed: int, *, fwhm_arcmin: float = 13.0,
                    cl=None, b_cut_deg: float = 20.0, n_disks: int = 500,
                    disk_radius_deg: float = 0.6, jitter: float = 0.2,
                    noise_range=None, noise_level_ell=None, homogeneous: bool = False,
                    masked: bool = True, draws: bool = True) -> dict:
    """HEALPix temperature workload.

    noise_var = sigma0^2 / hits, hits = (1 + 4 |sin beta_ecl|^3) * LN(0,
    jitter); if ``noise_range`` is given the hits are raised to the power
    that makes max/min noise variance over observed pixels equal to it.
    sigma0 puts the mean white-noise level sigma0^2 Omega / <hits> at C_l of
    l = ``noise_level_ell`` (default lmax / 2).  Masked: |b| < b_cut plus
    ``n_disks`` disks of radius ``disk_radius_deg`` at uniform random centres.
    """
    rng = np.random.default_rng(seed)
    npix = 12 * nside * nside
    omega = 4.0 * np.pi / npix
    c_ell = cmb_like_cl(lmax, fwhm_arcmin) if cl is None else np.asarray(cl, dtype=np.float64)
    z, phi0, nr = ring_layout(nside)
    off = np.concatenate([[0], np.cumsum(nr)[:-1]])

    zp = np.repeat(z, nr)
    jj = np.arange(npix) - np.repeat(off, nr)
    phi = np.repeat(phi0, nr) + 2.0 * np.pi * jj / np.repeat(nr, nr)
    sth = np.sqrt(np.maximum(0.0, (1.0 - zp) * (1.0 + zp)))
    pole = _ecliptic_pole_galactic()
    sin_beta = sth * np.cos(phi) * pole[0] + sth * np.sin(phi) * pole[1] + zp * pole[2]
    del sth
    hits = (1.0 + 4.0 * np.abs(sin_beta) ** 3) * np.exp(jitter * rng.standard_normal(npix))
    del sin_beta

    mask = np.ones(npix, dtype=np.uint8)
    if masked:
        mask[np.abs(zp) < math.sin(math.radians(b_cut_deg))] = 0
        rad = math.radians(disk_radius_deg)
        theta_r = np.arccos(z)
        for _ in range(n_disks):
            cz = rng.uniform(-1.0, 1.0)
            cphi = rng.uniform(0.0, 2.0 * np.pi)
            cth = math.acos(cz)
            rings = np.nonzero(np.abs(theta_r - cth) <= rad)[0]
            cst = math.sqrt(max(0.0, 1.0 - cz * cz))
            for r in rings:
                n = int(nr[r])
                st = math.sqrt(max(0.0, 1.0 - z[r] * z[r]))
                if st * cst > 0:
                    cosdphi_min = (math.cos(rad) - z[r] * cz) / (st * cst)
                else:
                    cosdphi_min = -1.0 if z[r] * cz >= math.cos(rad) else 2.0
                if cosdphi_min > 1.0:
                    continue
                dphi = math.acos(max(-1.0, cosdphi_min))
                j0 = int(math.floor((cphi - dphi - phi0[r]) * n / (2.0 * np.pi))) - 1
                j1 = int(math.ceil((cphi + dphi - phi0[r]) * n / (2.0 * np.pi))) + 1
                js = np.arange(j0, j1 + 1)
                js = np.unique(np.mod(js, n)) if j1 - j0 + 1 < n else np.arange(n)
                ph = phi0[r] + 2.0 * np.pi * js / n
                cosd = z[r] * cz + st * cst * np.cos(ph - cphi)
                mask[off[r] + js[cosd >= math.cos(rad)]] = 0
    del zp, phi

    obs = mask.astype(bool)
    if noise_range is not None:
        hmax, hmin = hits[obs].max(), hits[obs].min()
        gamma = math.log(noise_range) / math.log(hmax / hmin)
        hits = hits ** gamma
    if homogeneous:
        hits = np.full(npix, float(hits[obs].max()))
    lref = lmax // 2 if noise_level_ell is None else noise_level_ell
    sigma0_sq = c_ell[max(2, lref)] * float(hits.mean()) / omega
    noise_var = sigma0_sq / hits

    out = {"kind": "healpix", "nside": nside, "lmax": lmax, "c_ell": c_ell,
           "noise_var": noise_var, "mask": mask}
    if draws:
        ell = alm_ell(lmax)
        out["a_signal"] = np.sqrt(c_ell[ell]) * alm_unit_gaussian(rng, lmax)
        out["noise"] = np.sqrt(noise_var) * rng.standard_normal(npix)
        out["g1"] = rng.standard_normal(npix)
        out["g2"] = alm_unit_gaussian(rng, lmax)
    return out


def healpix_pol_problem(nside: int, lmax: int, seed: int, *, fwhm_arcmin: float = 13.0, corr: float = 0.1,
                        pol_noise_factor: float = 2.0, bb_ratio: float = 0.0, p_b_cut_deg=None, draws: bool = True,
                        **kw) -> dict:
    """Polarised (I, Q, U) workload.  Spectra: TT CMB-like, EE = 0.05 TT in
    shape, TE = 0.5 sqrt(TT EE), BB = bb_ratio EE; columns (TT, EE, BB, TE).
    Noise per pixel: diag(s_I^2, s_Q^2, s_U^2) with s_I^2 from the temperature
    hit model (healpix_problem, same keywords), s_Q^2 = s_U^2 =
    pol_noise_factor s_I^2, and I-Q, I-U, Q-U correlation coefficients drawn
    in [-corr, corr], redrawn until the block is positive definite.  Draws:
    signal (T, E, B) from the prior blocks, noise from the pixel blocks,
    fluctuation draws g1 (3, npix) and g2 (3, n_alm).  The mask is shared by
    I, Q and U (values 0 / 1), unless ``p_b_cut_deg`` adds a polarisation
    mask |b| < p_b_cut_deg: there observed pixels get the code 2 (I observed,
    Q and U masked)."""
    base = healpix_problem(nside, lmax, seed, fwhm_arcmin=fwhm_arcmin, draws=False, **kw)
    rng = np.random.default_rng(seed + 7919)
    npix = 12 * nside * nside
    tt = base["c_ell"]
    ee = 0.05 * tt
    cl = np.stack([tt, ee, bb_ratio * ee, 0.5 * np.sqrt(tt * ee)], axis=1)
    sI = base["noise_var"]
    var = np.stack([sI, pol_noise_factor * sI, pol_noise_factor * sI], axis=1)
    rho = rng.uniform(-corr, corr, size=(npix, 3))
    N = np.zeros((npix, 3, 3))
    for _ in range(100):
        sd = np.sqrt(var)
        N[:, 0, 0], N[:, 1, 1], N[:, 2, 2] = var[:, 0], var[:, 1], var[:, 2]
        N[:, 0, 1] = N[:, 1, 0] = rho[:, 0] * sd[:, 0] * sd[:, 1]
        N[:, 0, 2] = N[:, 2, 0] = rho[:, 1] * sd[:, 0] * sd[:, 2]
        N[:, 1, 2] = N[:, 2, 1] = rho[:, 2] * sd[:, 1] * sd[:, 2]
        bad = np.linalg.eigvalsh(N).min(axis=1) <= 0
        if not bad.any():
            break
        rho[bad] = rng.uniform(-corr, corr, size=(int(bad.sum()), 3))
    mask = base["mask"].copy()
    if p_b_cut_deg is not None:
        z, _, nr = ring_layout(nside)
        zp = np.repeat(z, nr)
        mask[(mask > 0) & (np.abs(zp) < np.sin(np.radians(p_b_cut_deg)))] = 2
    out = {"kind": "healpix_pol", "nside": nside, "lmax": lmax, "c_ell": cl, "noise_cov": N, "mask": mask}
    if draws:
        out.update(_pol_draws(rng, out))
    return out


def _pol_draws(rng, P: dict) -> dict:
    lmax, npix = P["lmax"], 12 * P["nside"] ** 2
    cl = P["c_ell"]
    tt, ee = cl[:, 0], cl[:, 1]
    ell = alm_ell(lmax)
    g = np.stack([alm_unit_gaussian(rng, lmax) for _ in range(3)])
    a = np.zeros_like(g)
    # T, E correlated through TE (Cholesky of the 2x2 block), B alone
    a[0] = np.sqrt(tt[ell]) * g[0]
    with np.errstate(divide="ignore", invalid="ignore"):
        c = np.where(tt[ell] > 0, cl[ell, 3] / np.sqrt(np.where(tt[ell] > 0, tt[ell], 1.0)), 0.0)
    a[1] = c * g[0] + np.sqrt(np.maximum(ee[ell] - c * c, 0.0)) * g[1]
    a[2] = np.sqrt(cl[ell, 2]) * g[2]
    Lc = np.linalg.cholesky(P["noise_cov"])
    noise = np.einsum("nij,jn->in", Lc, rng.standard_normal((3, npix)))
    g1 = rng.standard_normal((3, npix))
    g2 = np.stack([alm_unit_gaussian(rng, lmax) for _ in range(3)])
    return {"a_signal": a, "noise": noise, "g1": g1, "g2": g2}


def healpix_pol_draws(P: dict, seed: int) -> dict:
    """Another set of draws (signal a_signal, noise, fluctuation g1 and g2)
    for an existing polarised problem P (its spectra and noise blocks), from
    seed: many maps of one geometry without rebuilding its noise model."""
    return _pol_draws(np.random.default_rng(seed), P)


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------
def config_flat_128(k: int = 0) -> dict:
    """128 x 128 flat grid, FP64 (the small case)."""
    return flat_problem(128, seed=seed_for(1, k))


def config_nside512(k: int = 0, **kw) -> dict:
    """nside 512, lmax 1024, 13' beam, |b| < 20 deg plus 500 disks of 0.6 deg."""
    return healpix_problem(512, 1024, seed_for(2, k), fwhm_arcmin=13.0, b_cut_deg=20.0,
                           n_disks=500, disk_radius_deg=0.6, **kw)


def config_nside2048(k: int = 0, **kw) -> dict:
    """nside 2048, lmax 4096, 5' beam, noise dynamic range 1e4, |b| < 15 deg
    plus 3000 disks of 0.3 deg."""
    return healpix_problem(2048, 4096, seed_for(3, k), fwhm_arcmin=5.0, b_cut_deg=15.0,
                           n_disks=3000, disk_radius_deg=0.3, noise_range=1e4, **kw)
