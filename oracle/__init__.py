"""Oracle for the messenger-field Wiener filter (Elsner & Wandelt 2013).

TEST INFRASTRUCTURE.  A plain, slow, FP64 CPU statement of what the GPU path
computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the library never does, and the two share
no code.  The transforms live in ``wf_oracle.c`` (direct Legendre sums and
direct Fourier sums, no FFT); the flat-sky basis uses ``numpy.fft`` as a
library primitive; the messenger iteration itself is in ``messenger.py``.

Functions and the paper passage each follows:

* ``healpix_rings``         -- HEALPix RING grid (Sect. 3, pixelisation cited
                               there; Gorski et al. 2005).
* ``legendre``              -- normalised associated Legendre functions used by
                               the harmonic basis of Sect. 3.
* ``synthesis`` / ``adjoint_synthesis`` -- the basis change between pixel
                               space (where N is diagonal) and harmonic space
                               (where S is diagonal), Sect. 2.1.
* ``spin_legendre``, ``synthesis_pol`` / ``adjoint_pol`` -- the spin-2 basis
                               change of the polarised maps (I, Q, U) that
                               Eqs. (10)-(11) act on, written from the
                               definition (Q + iU) = sum 2a_lm 2Y_lm over all m.
* ``FlatBasis`` / ``HealpixBasis`` -- the two bases; ``messenger.py`` runs
                               Eqs. (3)-(4), the chi^2 of Eq. (6), the cooling
                               schedule of Sect. 3 and the fluctuation source
                               of Eq. (9).
* ``marginalize_templates`` -- monopole/dipole projection of Eq. (12).
* ``combine_datasets``      -- several data sets of one signal with the same
                               beam (the outlook of Sect. 4) reduced exactly
                               to one: N^-1 = sum N_k^-1, N^-1 d = sum N_k^-1 d_k.

Parity status: every function here is pinned by tests in
``tests/test_oracle_*.py`` except the heuristic schedule's plateau constant
and level cap (parity unpinned as to iteration count; they do not change the
converged result beyond the tolerance).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        lib.or_healpix_rings.argtypes = [ctypes.c_int, dp, dp, dp, ip, ip]
        lib.or_healpix_rings.restype = None
        lib.or_legendre.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
        lib.or_legendre.restype = None
        lib.or_synthesis.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int]
        lib.or_synthesis.restype = None
        lib.or_adjoint_synthesis.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int]
        lib.or_adjoint_synthesis.restype = None
        lib.or_spin_legendre.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
        lib.or_spin_legendre.restype = None
        lib.or_synthesis_pol.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ctypes.c_int,
                                         ctypes.c_int]
        lib.or_synthesis_pol.restype = None
        lib.or_adjoint_pol.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        lib.or_adjoint_pol.restype = None
        lib.or_num_threads.argtypes = []
        lib.or_num_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    """OpenMP threads the C core uses (reported with every CPU timing)."""
    return int(_lib().or_num_threads())


# --------------------------------------------------------------------------
# HEALPix geometry and harmonic indexing
# --------------------------------------------------------------------------
def npix(nside: int) -> int:
    return 12 * nside * nside


def nalm(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(lmax: int, l, m):
    """m-major index of a_lm (m >= 0): m (2 lmax + 3 - m) / 2 + (l - m)."""
    return m * (2 * lmax + 3 - m) // 2 + (l - m)


def alm_lm(lmax: int):
    """(l, m) arrays in storage order."""
    ls, ms = [], []
    for m in range(lmax + 1):
        ls.append(np.arange(m, lmax + 1))
        ms.append(np.full(lmax + 1 - m, m))
    return np.concatenate(ls), np.concatenate(ms)


def healpix_rings(nside: int) -> dict:
    """Per-ring z = cos(theta), sin(theta), phi of the first pixel, pixel
    count and offset of the ring's first pixel, rings north to south."""
    R = 4 * nside - 1
    z = np.empty(R)
    st = np.empty(R)
    p0 = np.empty(R)
    nr = np.empty(R, dtype=np.int64)
    off = np.empty(R, dtype=np.int64)
    _lib().or_healpix_rings(nside, _dp(z), _dp(st), _dp(p0),
                            nr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return {"z": z, "sintheta": st, "phi0": p0, "nr": nr, "offset": off}


def pixel_angles(nside: int):
    """(theta, phi) of every pixel centre in RING order."""
    g = healpix_rings(nside)
    th, ph = [], []
    for z, p0, n in zip(g["z"], g["phi0"], g["nr"]):
        th.append(np.full(n, np.arccos(z)))
        ph.append(p0 + 2.0 * np.pi * np.arange(n) / n)
    return np.concatenate(th), np.concatenate(ph)


def legendre(lmax: int, m: int, x: float) -> np.ndarray:
    """lambda_lm(x), l = m..lmax, normalised, Condon-Shortley phase."""
    out = np.zeros(lmax - m + 1)
    st = float(np.sqrt((1.0 - x) * (1.0 + x)))
    _lib().or_legendre(lmax, m, float(x), st, _dp(out))
    return out


def synthesis(nside: int, lmax: int, L: int, alm: np.ndarray, rings=None) -> np.ndarray:
    """Map f = Y a (a restricted to l <= L).  ``rings`` = (lo, hi) computes
    only those rings (other pixels are returned as NaN)."""
    a = np.ascontiguousarray(np.asarray(alm, dtype=np.complex128)).view(np.float64)
    assert a.size == 2 * nalm(lmax)
    out = np.full(npix(nside), np.nan)
    lo, hi = (0, 4 * nside - 1) if rings is None else rings
    _lib().or_synthesis(nside, lmax, L, _dp(a), _dp(out), lo, hi)
    return out


def adjoint_synthesis(nside: int, lmax: int, L: int, f: np.ndarray, ms=None) -> np.ndarray:
    """b = Y^T f (l <= L; zero above L).  ``ms`` = (lo, hi) computes only
    those m (other entries are returned as NaN)."""
    fm = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    assert fm.size == npix(nside)
    out = np.zeros(2 * nalm(lmax))
    lo, hi = (0, L + 1) if ms is None else ms
    if ms is not None:
        out[:] = np.nan
    _lib().or_adjoint_synthesis(nside, lmax, L, _dp(fm), _dp(out), lo, hi)
    res = out.view(np.complex128).copy()
    if ms is not None:
        l, m = alm_lm(lmax)
        sel = (m >= lo) & (m < hi) & (l > L)
        res[sel] = 0.0
    return res


def spin_legendre(lmax: int, m: int, s: int, x: float) -> np.ndarray:
    """slambda_lm(theta) = sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta), l = 0..lmax
    (zero below max(|m|, |s|)); any sign of m and s.  s = 0 is lambda_lm."""
    out = np.zeros(lmax + 1)
    st = float(np.sqrt((1.0 - x) * (1.0 + x)))
    _lib().or_spin_legendre(lmax, m, s, float(x), st, _dp(out))
    return out


def synthesis_pol(nside: int, lmax: int, L: int, E, B, rings=None):
    """(Q, U) maps of (Q + iU) = sum_{l>=2, |m|<=l} 2a_lm 2Y_lm, 2a = -(E + iB),
    l <= L; E, B stored like a_lm (m >= 0).  ``rings`` = (lo, hi) computes
    only those rings (other pixels NaN)."""
    e = np.ascontiguousarray(np.asarray(E, dtype=np.complex128)).view(np.float64)
    b = np.ascontiguousarray(np.asarray(B, dtype=np.complex128)).view(np.float64)
    assert e.size == b.size == 2 * nalm(lmax)
    Q = np.full(npix(nside), np.nan)
    U = np.full(npix(nside), np.nan)
    lo, hi = (0, 4 * nside - 1) if rings is None else rings
    _lib().or_synthesis_pol(nside, lmax, L, _dp(e), _dp(b), _dp(Q), _dp(U), lo, hi)
    return Q, U


def adjoint_pol(nside: int, lmax: int, L: int, Q, U):
    """Adjoint of synthesis_pol: (E, B) with E_lm = -(t_lm + (-1)^m conj t_{l,-m})/2,
    B_lm = (i/2)(t_lm - (-1)^m conj t_{l,-m}), t_lm = sum_p (Q + iU)_p conj 2Y_lm(p)."""
    q = np.ascontiguousarray(np.asarray(Q, dtype=np.float64))
    u = np.ascontiguousarray(np.asarray(U, dtype=np.float64))
    assert q.size == u.size == npix(nside)
    e = np.zeros(2 * nalm(lmax))
    b = np.zeros(2 * nalm(lmax))
    _lib().or_adjoint_pol(nside, lmax, L, _dp(q), _dp(u), _dp(e), _dp(b))
    return e.view(np.complex128).copy(), b.view(np.complex128).copy()


# --------------------------------------------------------------------------
# The two bases of Sect. 2.1: pixel space (N diagonal) and harmonic space
# (S diagonal).  ``synth`` maps harmonic -> pixel; ``adjoint`` is its adjoint
# under the weighted inner product <a, b> = Re sum w conj(a) b, so that
# ``omega * adjoint`` is the analysis (inverse basis change).
# --------------------------------------------------------------------------
class FlatBasis:
    """Periodic ny x nx grid with the unitary 2-D DFT (Omega = 1).  Harmonic
    vectors are the rfft half plane ny x (nx/2 + 1); columns kx = 0 and
    kx = nx/2 count once in norms, the others twice."""

    kind = "flat"

    def __init__(self, ny: int, nx: int):
        self.ny, self.nx = ny, nx
        self.omega = 1.0
        w = np.full((ny, nx // 2 + 1), 2.0)
        w[:, 0] = 1.0
        if nx % 2 == 0:
            w[:, nx // 2] = 1.0
        self.w = w
        self.lmax = None

    def synth(self, a, L=None):
        return np.fft.irfft2(a, s=(self.ny, self.nx), norm="ortho")

    def adjoint(self, t, L=None):
        return np.fft.rfft2(t, norm="ortho")

    def band(self, L):
        return np.ones(self.w.shape, dtype=bool)

    def kabs(self):
        ky = np.fft.fftfreq(self.ny, 1.0 / self.ny)
        kx = np.arange(self.nx // 2 + 1)
        return np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)


class HealpixBasis:
    """HEALPix RING grid with spherical harmonics up to lmax; Omega = 4 pi /
    n_pix.  Harmonic vectors are complex a_lm, m >= 0, m-major; m = 0 counts
    once in norms, m > 0 twice."""

    kind = "healpix"

    def __init__(self, nside: int, lmax: int):
        self.nside, self.lmax = nside, lmax
        self.omega = 4.0 * np.pi / npix(nside)
        self.ell, self.m = alm_lm(lmax)
        self.w = np.where(self.m == 0, 1.0, 2.0)

    def synth(self, a, L=None):
        return synthesis(self.nside, self.lmax, self.lmax if L is None else L, a)

    def adjoint(self, t, L=None):
        return adjoint_synthesis(self.nside, self.lmax, self.lmax if L is None else L, t)

    def band(self, L):
        return self.ell <= L

    def per_mode(self, c_ell):
        """Expand a per-l array to one value per stored a_lm."""
        return np.asarray(c_ell, dtype=np.float64)[self.ell]


from .messenger import (  # noqa: E402
    fluct_source,
    messenger_solve,
    wnorm,
)
from .templates import marginalize_templates, template_matrix  # noqa: E402
from .datasets import combine_datasets  # noqa: E402

__all__ = [
    "FlatBasis",
    "HealpixBasis",
    "adjoint_pol",
    "adjoint_synthesis",
    "alm_index",
    "alm_lm",
    "combine_datasets",
    "fluct_source",
    "healpix_rings",
    "legendre",
    "marginalize_templates",
    "messenger_solve",
    "nalm",
    "npix",
    "num_threads",
    "pixel_angles",
    "spin_legendre",
    "synthesis",
    "synthesis_pol",
    "template_matrix",
    "wnorm",
]
