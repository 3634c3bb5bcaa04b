"""Plain FP64 CPU statement of the 3D extension (test infrastructure only).

The paper (arXiv 2510.01190) treats 2D fields and names 3D vector fields as
future work (Sec. 5).  The closed form carries over term by term; what the GPU
library computes for volumes is fixed here (reading R20):

* Eq. 1 gains the z term: D = (u_{i+1} - u_{i-1}) / (2 dx)
  + (v_{j+1} - v_{j-1}) / (2 dy) + (w_{k+1} - w_{k-1}) / (2 dz), with the
  one-sided first-order rule of reading R2 on every face of the box;
* Eqs. 2 and 3 gain the matching mean and variance terms of w;
* a cell (i, j, k) has the 8 vertices (i..i+1, j..j+1, k..k+1) and
  LCP = 1 - prod_8 P(D < c) - prod_8 P(D >= c) (reading R1 with 8 factors);
  the mean-field crossing is "not all 8 on one side" (reading R7).

Arrays are indexed [..., k, j, i] (z, y, x); u is the x component, v the y,
w the z.  Only ``tests/``, ``__graft_entry__.smoke`` and ``bench.py``'s
CPU-baseline leg may import this module.  It imports nothing from the GPU
library.
"""

from __future__ import annotations

import numpy as np

from .lcp_oracle import below_above_probabilities, ensemble_stats, stencil_neighbours

__all__ = [
    "divergence_gaussian_3d",
    "divergence_of_field_3d",
    "level_crossing_probability_3d",
    "mean_field_crossing_3d",
    "lcp_closed_form_3d",
]

_CORNERS = [(dk, dj, di) for dk in (0, 1) for dj in (0, 1) for di in (0, 1)]


def _steps(d, h, w, dx, dy, dz):
    ilo, ihi, isteps = stencil_neighbours(w)
    jlo, jhi, jsteps = stencil_neighbours(h)
    klo, khi, ksteps = stencil_neighbours(d)
    hx = (isteps * float(dx))[None, None, :]
    hy = (jsteps * float(dy))[None, :, None]
    hz = (ksteps * float(dz))[:, None, None]
    return (ilo, ihi, hx), (jlo, jhi, hy), (klo, khi, hz)


def divergence_gaussian_3d(mu_u, var_u, mu_v, var_v, mu_w, var_w, dx: float, dy: float, dz: float):
    """Mean and variance of the 3D divergence Gaussian at every vertex (Eqs. 2
    and 3 with the z terms, reading R20).  Inputs [D, H, W]; returns (mu_d, var_d)."""
    a = [np.asarray(t, np.float64) for t in (mu_u, var_u, mu_v, var_v, mu_w, var_w)]
    mu_u, var_u, mu_v, var_v, mu_w, var_w = a
    d, h, w = mu_u.shape
    (ilo, ihi, hx), (jlo, jhi, hy), (klo, khi, hz) = _steps(d, h, w, dx, dy, dz)
    mu = ((mu_u[:, :, ihi] - mu_u[:, :, ilo]) / hx + (mu_v[:, jhi, :] - mu_v[:, jlo, :]) / hy
          + (mu_w[khi] - mu_w[klo]) / hz)
    var = ((var_u[:, :, ihi] + var_u[:, :, ilo]) / hx ** 2 + (var_v[:, jhi, :] + var_v[:, jlo, :]) / hy ** 2
           + (var_w[khi] + var_w[klo]) / hz ** 2)
    return mu, var


def divergence_of_field_3d(u, v, w, dx: float, dy: float, dz: float):
    """Finite-difference divergence of one (or a stack of) 3D realisations
    (Eq. 1 with the z term).  u, v, w : [..., D, H, W]."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    w = np.asarray(w, np.float64)
    d, h, wd = u.shape[-3:]
    (ilo, ihi, hx), (jlo, jhi, hy), (klo, khi, hz) = _steps(d, h, wd, dx, dy, dz)
    return ((u[..., ihi] - u[..., ilo]) / hx + (v[..., jhi, :] - v[..., jlo, :]) / hy
            + (w[..., khi, :, :] - w[..., klo, :, :]) / hz)


def level_crossing_probability_3d(mu_d, var_d, isovalues):
    """LCP of every hexahedral cell and isovalue (reading R20):
    1 - prod over the 8 vertices of P(D < c) - prod of P(D >= c).
    returns [K, D-1, H-1, W-1]"""
    mu_d = np.asarray(mu_d, np.float64)
    var_d = np.asarray(var_d, np.float64)
    d, h, w = mu_d.shape
    iso = np.atleast_1d(np.asarray(isovalues, np.float64))
    out = np.empty((iso.size, d - 1, h - 1, w - 1))
    for kk, c in enumerate(iso):
        p, q = below_above_probabilities(mu_d, var_d, c)
        pp = np.ones((d - 1, h - 1, w - 1))
        qq = np.ones((d - 1, h - 1, w - 1))
        for dk, dj, di in _CORNERS:
            sl = (slice(dk, d - 1 + dk), slice(dj, h - 1 + dj), slice(di, w - 1 + di))
            pp = pp * p[sl]
            qq = qq * q[sl]
        out[kk] = 1.0 - pp - qq
    return out


def mean_field_crossing_3d(mu_d, isovalues):
    """Mean-field crossing per cell: its 8 vertices are not all below (mu < c)
    and not all not-below.  returns bool [K, D-1, H-1, W-1]"""
    mu_d = np.asarray(mu_d, np.float64)
    d, h, w = mu_d.shape
    iso = np.atleast_1d(np.asarray(isovalues, np.float64))
    out = np.empty((iso.size, d - 1, h - 1, w - 1), dtype=bool)
    for kk, c in enumerate(iso):
        b = (mu_d < c).astype(np.int64)
        n = np.zeros((d - 1, h - 1, w - 1), np.int64)
        for dk, dj, di in _CORNERS:
            n += b[dk:d - 1 + dk, dj:h - 1 + dj, di:w - 1 + di]
        out[kk] = (n > 0) & (n < 8)
    return out


def lcp_closed_form_3d(u, v, w, dx: float, dy: float, dz: float, isovalues, ddof: int = 1):
    """Members [M, D, H, W] of u, v, w -> statistics -> 3D Eqs. 2/3 -> LCP.
    returns dict with mu_d, var_d, lcp, mask"""
    mu_u, var_u = ensemble_stats(u, ddof)
    mu_v, var_v = ensemble_stats(v, ddof)
    mu_w, var_w = ensemble_stats(w, ddof)
    mu_d, var_d = divergence_gaussian_3d(mu_u, var_u, mu_v, var_v, mu_w, var_w, dx, dy, dz)
    return dict(mu_d=mu_d, var_d=var_d, lcp=level_crossing_probability_3d(mu_d, var_d, isovalues),
                mask=mean_field_crossing_3d(mu_d, isovalues))
