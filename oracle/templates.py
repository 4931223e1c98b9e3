"""Template marginalisation of the input map (paper Sect. 3, Eq. 12).

TEST INFRASTRUCTURE (part of the oracle; see ``oracle/__init__.py``).

The paper removes residual monopole and dipole from the masked data by
d = lim_{sigma -> inf} (1 + sigma V V^T)^-1 d_raw, with the four masked
templates (monopole and the three dipole components) as the columns of V,
evaluated with the Woodbury identity:
    (1 + sigma V V^T)^-1 = 1 - V (sigma^-1 + V^T V)^-1 V^T
      -> 1 - V (V^T V)^-1 V^T            (sigma -> infinity),
the projection of d_raw orthogonal to the templates.
"""
import numpy as np


def template_matrix(nside, mask):
    """n_pix x 4 masked templates: monopole, then the x, y, z components of
    the pixel direction; zero in masked pixels."""
    from . import pixel_angles

    th, ph = pixel_angles(nside)
    st = np.sin(th)
    V = np.stack([np.ones_like(th), st * np.cos(ph), st * np.sin(ph), np.cos(th)], axis=1)
    return V * (np.asarray(mask) > 0)[:, None]


def marginalize_templates(nside, d_raw, mask, sigma=None):
    """sigma None: the sigma -> infinity limit; otherwise the finite-sigma
    Woodbury form.  Returns (d, coefficients of the removed templates)."""
    V = template_matrix(nside, mask)
    G = V.T @ V
    vd = V.T @ np.asarray(d_raw, dtype=np.float64)
    M = G if sigma is None else G + np.eye(4) / sigma
    c = np.linalg.solve(M, vd)
    return d_raw - V @ c, c
