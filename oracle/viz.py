"""Plain CPU statement of the visual outputs (test infrastructure only).

The paper (arXiv 2510.01190) shows its results as colour-mapped LCP maps
(Sec. 3.1, last paragraph), the mean-field divergence with its isocontour
(Fig. 1a, Fig. 3c, clamped to a display range in Sec. 4.2), and spaghetti plots
of the isocontours of every ensemble member (Fig. 1b).  This module states
those outputs as mathematics, in FP64 with true divisions:

* ``colormap_levels`` / ``colormap_rgba``: the piecewise-linear colour map of
  reading R17;
* ``marching_squares``: the isocontour segments of a scalar field on the grid
  (reading R18);
* ``spaghetti_contours``: the isocontours of every member's Eq. 1 divergence
  (``lcp_oracle.divergence_of_field``, FP64), the spaghetti plot of Fig. 1b.

A GPU kernel computing these in fp32 can differ from them only where fp32
rounding moves a quantity across a decision threshold (a byte boundary, an
isovalue, the saddle centre); the parity tests state those guard bands.

Only ``tests/``, ``__graft_entry__.smoke`` and ``bench.py``'s CPU-baseline leg
may import this module.  It imports nothing from the GPU library.

Readings
--------
R17 Colour map (the paper names none): a table of stops (t_q, r_q, g_q, b_q,
    a_q), q = 0..S-1, with t_0 = 0 < t_1 < ... < t_{S-1} = 1.  A value x maps to
    t = clamp((x - vmin) / (vmax - vmin), 0, 1) (x = +inf gives 1, -inf 0);
    the segment s is the largest q <= S-2 with t_q <= t; inside it each
    channel is ch = c_s + (t - t_s) / (t_{s+1} - t_s) (c_{s+1} - c_s) and the
    byte is floor(255 ch + 1/2).  NaN values get their own colour; an optional
    crossing mask paints the mean-field contour cells in a contour colour (the
    black / cyan contour of Fig. 1a / Fig. 3c at cell resolution), except NaN.
R18 Isocontour segments (marching squares; the paper shows mean-field
    isocontours in Fig. 1a / Fig. 3c and spaghetti plots of the members'
    isocontours in Fig. 1b without defining the extraction).  Cell (i, j) has
    corners v0 = (i, j), v1 = (i+1, j), v2 = (i+1, j+1), v3 = (i, j+1); a corner
    is below when f < c (reading R7); edges E0 = v0v1, E1 = v1v2, E2 = v3v2,
    E3 = v0v3 cross where their corners differ.  A crossing point is
    interpolated from the edge's lower-coordinate vertex: on a horizontal edge
    x = i + (c - f(i, j)) / (f(i+1, j) - f(i, j)), on a vertical one
    y = j + (c - f(i, j)) / (f(i, j+1) - f(i, j)), so neighbouring cells agree
    on shared points.  Two crossing edges give one segment (lower edge first).
    The saddles (v0, v2 on one side, v1, v3 on the other) give two, decided by
    the cell's centre value (f0 + f1 + f2 + f3) / 4, the bilinear interpolant
    at the cell centre: if it lies on v0's side, (E0, E1) and (E2, E3), else
    (E0, E3) and (E1, E2).  Cells with a NaN corner give none.  Segment
    (x0, y0, x1, y1) carries the key ((j (W-1) + i) K + k) 2 + s (s = 0, 1
    within the cell); for member m of a spaghetti plot the key adds
    m (H-1)(W-1) K 2.  Lists are in key order.  A spaghetti plot contours each
    member's divergence as Eq. 1 defines it (central differences inside,
    first-order one-sided differences on the first and last row and column).
"""

from __future__ import annotations

import numpy as np

from . import lcp_oracle as _core

__all__ = ["colormap_levels", "colormap_rgba", "pack_rgba", "marching_squares", "spaghetti_contours"]


def pack_rgba(r: int, g: int, b: int, a: int) -> int:
    """The packed colour word r | g << 8 | b << 16 | a << 24."""
    return int(r) | (int(g) << 8) | (int(b) << 16) | (int(a) << 24)


def _unpack(word: int):
    return np.array([(int(word) >> (8 * k)) & 0xFF for k in range(4)], dtype=np.uint8)


def colormap_levels(values, vmin: float, vmax: float, stops):
    """Reading R17 before quantisation, in FP64: returns (y, s) where
    y [..., 4] = 255 ch + 1/2 of every channel (its floor is the byte) and
    s [...] is the stop segment of each value (NaN values: y is NaN, s = 0)."""
    x = np.asarray(values, dtype=np.float64)
    st = np.asarray(stops, dtype=np.float64).reshape(-1, 5)
    n_stops = st.shape[0]
    lo, hi = float(vmin), float(vmax)
    with np.errstate(invalid="ignore", over="ignore"):
        t = (x - lo) / (hi - lo)
        t = np.where(np.isnan(t), np.nan, np.clip(t, 0.0, 1.0))
        s = np.zeros(x.shape, dtype=np.int64)
        for q in range(1, n_stops - 1):
            s = np.where(t >= st[q, 0], q, s)
        f = (t - st[s, 0]) / (st[s + 1, 0] - st[s, 0])
        y = np.empty(x.shape + (4,), dtype=np.float64)
        for ch in range(4):
            c = st[s, 1 + ch] + f * (st[s + 1, 1 + ch] - st[s, 1 + ch])
            y[..., ch] = 255.0 * c + 0.5
    return y, s


def colormap_rgba(values, vmin: float, vmax: float, stops, nan_rgba: int = 0, mask=None, mask_rgba: int = 0):
    """RGBA8 colour of every value (reading R17), in FP64.

    values : float array [..., rows, cols]
    stops  : [S, 5] (t, r, g, b, a)
    mask   : optional bool array of the shape of ``values`` (True paints
             ``mask_rgba``)
    returns uint8 [..., rows, cols, 4]
    """
    x = np.asarray(values, dtype=np.float64)
    y, _ = colormap_levels(x, vmin, vmax, stops)
    nan = np.isnan(x)
    with np.errstate(invalid="ignore"):
        out = np.clip(np.floor(np.where(nan[..., None], 0.0, y)), 0, 255).astype(np.uint8)
    out[nan] = _unpack(nan_rgba)
    if mask is not None:
        m = np.asarray(mask, dtype=bool) & ~nan
        out[m] = _unpack(mask_rgba)
    return out


# --------------------------------------------------------------------------
# Isocontour segments (reading R18)
# --------------------------------------------------------------------------
def marching_squares(f, isovalues):
    """Isocontour segments of the scalar field f [H, W] for every isovalue
    (reading R18), in FP64.  returns (keys int64 [n], segs float64 [n, 4]) in
    key order."""
    f = np.asarray(f, np.float64)
    h, w = f.shape
    iso = np.atleast_1d(np.asarray(isovalues, np.float64))
    kk = iso.size
    f0, f1 = f[:-1, :-1], f[:-1, 1:]      # v0 = (i, j), v1 = (i+1, j)
    f3, f2 = f[1:, :-1], f[1:, 1:]        # v3 = (i, j+1), v2 = (i+1, j+1)
    jj, ii = np.meshgrid(np.arange(h - 1, dtype=np.float64), np.arange(w - 1, dtype=np.float64), indexing="ij")
    finite = ~(np.isnan(f0) | np.isnan(f1) | np.isnan(f2) | np.isnan(f3))
    centre = (f0 + f1 + f2 + f3) / 4.0
    cell = (np.arange(h - 1)[:, None] * (w - 1) + np.arange(w - 1)[None, :]).astype(np.int64)
    keys, segs = [], []
    with np.errstate(invalid="ignore", divide="ignore"):
        for k in range(kk):
            c = float(iso[k])
            b0, b1, b2, b3 = f0 < c, f1 < c, f2 < c, f3 < c
            # crossing points of the four edges, interpolated from the lower-coordinate vertex
            p = [np.stack([ii + (c - f0) / (f1 - f0), jj], -1),          # E0: v0 -> v1
                 np.stack([ii + 1.0, jj + (c - f1) / (f2 - f1)], -1),    # E1: v1 -> v2
                 np.stack([ii + (c - f3) / (f2 - f3), jj + 1.0], -1),    # E2: v3 -> v2
                 np.stack([ii, jj + (c - f0) / (f3 - f0)], -1)]          # E3: v0 -> v3
            cross = [b0 != b1, b1 != b2, b3 != b2, b0 != b3]
            n_cross = cross[0].astype(int) + cross[1] + cross[2] + cross[3]
            saddle = finite & (b0 == b2) & (b1 == b3) & (b0 != b1)
            single = finite & (n_cross == 2)
            # one segment: the two crossing edges, lower index first
            for a in range(4):
                for b in range(a + 1, 4):
                    sel = single & cross[a] & cross[b]
                    keys.append(((cell[sel] * kk + k) * 2).ravel())
                    segs.append(np.concatenate([p[a][sel], p[b][sel]], -1))
            # saddles: the centre on v0's side joins v0 and v2
            with_v0 = saddle & ((centre < c) == b0)
            for sel, pairs in ((with_v0, ((0, 1), (2, 3))), (saddle & ~with_v0, ((0, 3), (1, 2)))):
                for s_idx, (a, b) in enumerate(pairs):
                    keys.append(((cell[sel] * kk + k) * 2 + s_idx).ravel())
                    segs.append(np.concatenate([p[a][sel], p[b][sel]], -1))
    keys = np.concatenate(keys) if keys else np.zeros(0, np.int64)
    segs = np.concatenate(segs) if segs else np.zeros((0, 4))
    order = np.argsort(keys, kind="stable")
    return keys[order], segs[order].reshape(-1, 4)


def spaghetti_contours(u, v, dx: float, dy: float, isovalues):
    """Isocontours of every member's Eq. 1 divergence (Fig. 1b), reading R18.
    u, v [M, H, W]; returns (keys int64 [n], segs float64 [n, 4]) in key order."""
    d = _core.divergence_of_field(u, v, dx, dy)
    m, h, w = d.shape
    kk = np.atleast_1d(np.asarray(isovalues)).size
    per = (h - 1) * (w - 1) * kk * 2
    keys, segs = [], []
    for mm in range(m):
        k_m, s_m = marching_squares(d[mm], isovalues)
        keys.append(k_m + mm * per)
        segs.append(s_m)
    if not keys:
        return np.zeros(0, np.int64), np.zeros((0, 4))
    return np.concatenate(keys), np.concatenate(segs)
