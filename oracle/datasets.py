"""Several data sets of one signal with the same beam and pixelisation.

TEST INFRASTRUCTURE (part of the oracle; see ``oracle/__init__.py``).

The paper's outlook (Sect. 4) names the generalisation to multiple data sets
measuring the same underlying signal.  When every data set d_k = s + n_k sees
the signal through the same transfer function (the beam enters the prior, as
in Sect. 3) on the same pixels, the stacked Wiener-filter equation (Eq. 2 for
the stacked data vector, with a block-diagonal noise covariance)

    (S^-1 + sum_k N_k^-1) s = sum_k N_k^-1 d_k

is Eq. (2) of a single data set with

    N^-1 = sum_k N_k^-1,      N^-1 d = sum_k N_k^-1 d_k,

summed per pixel over the data sets that observe it (a masked pixel of data
set k has N_k^-1 = 0, Sect. 2.1).  A pixel that no data set observes stays
masked.  This function forms that single data set; the messenger iteration
then runs unchanged.
"""
import numpy as np


def combine_datasets(d_list, noise_list, mask_list=None):
    """Inverse-noise-weighted combination of per-pixel data sets.

    d_list, noise_list: sequences of equal-length pixel maps (noise variance
    per pixel); mask_list: per data set 1 = observed, 0 = masked (None or a
    None entry: all observed).  Returns (d, noise_var, mask) of the single
    equivalent data set; unobserved pixels get d = 0, noise_var = 1, mask 0."""
    k = len(d_list)
    npix = np.asarray(d_list[0]).size
    w = np.zeros(npix)
    wd = np.zeros(npix)
    for j in range(k):
        obs = np.ones(npix, dtype=bool) if mask_list is None or mask_list[j] is None \
            else np.asarray(mask_list[j]) > 0
        nvar = np.asarray(noise_list[j], dtype=np.float64)
        dj = np.asarray(d_list[j], dtype=np.float64)
        inv = np.zeros(npix)
        inv[obs] = 1.0 / nvar[obs]
        w += inv
        wd += np.where(obs, inv * dj, 0.0)
    seen = w > 0
    noise = np.ones(npix)
    noise[seen] = 1.0 / w[seen]
    d = np.zeros(npix)
    d[seen] = wd[seen] / w[seen]
    return d, noise, seen.astype(np.uint8)
