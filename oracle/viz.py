"""Plain CPU statement of the visual outputs (test infrastructure only).

The paper (arXiv 2510.01190) shows its results as colour-mapped LCP maps
(Sec. 3.1, last paragraph), the mean-field divergence with its isocontour
(Fig. 1a, Fig. 3c, clamped to a display range in Sec. 4.2), and spaghetti plots
of the isocontours of every ensemble member (Fig. 1b).  This module fixes what
the GPU library computes for those outputs:

* ``colormap_rgba``: the piecewise-linear colour map of reading R17, step by
  step in IEEE fp32 (a quantised code: both sides decide it in the kernel's
  precision);
* ``marching_squares``: the isocontour segments of a scalar field on the grid
  (reading R18), in FP64.

Only ``tests/``, ``__graft_entry__.smoke`` and ``bench.py``'s CPU-baseline leg
may import this module.  It imports nothing from the GPU library.

Readings (listed in the design doc)
------------------------------
R17 Colour map (the paper names none): a table of stops (t, r, g, b, a) with
    t from 0 to 1; t = clamp((x - vmin) R, 0, 1) with R = 1 / (vmax - vmin);
    linear interpolation inside the stop segment s that holds t, as
    f = (t - t_s) r_s and ch = c_s + f d_s with r_s = 1 / (t_{s+1} - t_s) and
    d_s = c_{s+1} - c_s formed once per table; byte = floor(255 ch + 0.5).
    Every step is one fp32 operation rounded to nearest.  NaN values get their
    own colour; an optional crossing mask paints the mean-field contour cells
    in a contour colour (the black / cyan contour of Fig. 1a / Fig. 3c at cell
    resolution).
"""

from __future__ import annotations

import numpy as np

__all__ = ["colormap_rgba", "pack_rgba"]

_F = np.float32


def pack_rgba(r: int, g: int, b: int, a: int) -> int:
    """The packed colour word r | g << 8 | b << 16 | a << 24."""
    return int(r) | (int(g) << 8) | (int(b) << 16) | (int(a) << 24)


def _quantise(ch):
    b = np.floor((ch * _F(255.0)).astype(_F) + _F(0.5)).astype(_F)
    return np.clip(b, 0, 255).astype(np.uint8)


def colormap_rgba(values, vmin: float, vmax: float, stops, nan_rgba: int = 0, mask=None, mask_rgba: int = 0):
    """RGBA8 colour of every value (reading R17), in IEEE fp32 one operation
    at a time (numpy rounds each float32 operation to nearest).

    values : float array [..., rows, cols]
    stops  : [S, 5] (t, r, g, b, a)
    mask   : optional bool array of the shape of ``values`` (True paints
             ``mask_rgba``)
    returns uint8 [..., rows, cols, 4]
    """
    x = np.asarray(values, dtype=_F)
    st = np.asarray(stops, dtype=_F).reshape(-1, 5)
    n_stops = st.shape[0]
    lo, hi = _F(vmin), _F(vmax)
    one = _F(1.0)
    with np.errstate(invalid="ignore", over="ignore"):
        big_r = one / (hi - lo)                               # R (0 when the range overflows)
        r_seg = one / (st[1:, 0] - st[:-1, 0])                # r_s
        d_seg = st[1:, 1:] - st[:-1, 1:]                      # d_s, [n_stops - 1, 4]
        t = ((x - lo).astype(_F) * big_r).astype(_F)
        t = np.fmin(np.fmax(t, _F(0.0)), _F(1.0))  # maxNum / minNum: a NaN operand yields the other
        s = np.zeros(x.shape, dtype=np.int64)
        for q in range(1, n_stops - 1):
            s = np.where(t >= st[q, 0], q, s)
        f = ((t - st[s, 0]).astype(_F) * r_seg[s]).astype(_F)
        out = np.empty(x.shape + (4,), dtype=np.uint8)
        for ch in range(4):
            c = (st[s, 1 + ch] + (f * d_seg[s, ch]).astype(_F)).astype(_F)
            out[..., ch] = _quantise(c)
    nan_bytes = np.array([(nan_rgba >> (8 * k)) & 0xFF for k in range(4)], dtype=np.uint8)
    out[np.isnan(x)] = nan_bytes
    if mask is not None:
        m = np.asarray(mask, dtype=bool) & ~np.isnan(x)
        out[m] = np.array([(mask_rgba >> (8 * k)) & 0xFF for k in range(4)], dtype=np.uint8)
    return out
