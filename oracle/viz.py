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
  (reading R18), in FP64 except for the two decisions R18 fixes in fp32;
* ``member_divergence32`` and ``spaghetti_contours``: every member's Eq. 1
  divergence in fp32 (the operation order of reading R18) and its isocontours,
  the spaghetti plot of Fig. 1b.

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
    The saddles (v0, v2 on one side, v1, v3 on the other) give two: if the
    centre value ((f0 + f1) + (f2 + f3)) / 4, formed in fp32, lies on v0's side,
    (E0, E1) and (E2, E3), else (E0, E3) and (E1, E2).  Cells with a NaN corner
    give none.  Segment (x0, y0, x1, y1) carries the key
    ((j (W-1) + i) K + k) 2 + s (s = 0, 1 within the cell); for member m of a
    spaghetti plot the key adds m (H-1)(W-1) K 2.  Lists are in key order.
    The member divergence of a spaghetti plot is Eq. 1 in fp32 with each
    operation rounded: (u[i+] - u[i-]) * sx + (v[j+] - v[j-]) * sy with
    sx = fp32(1 / ((i+ - i-) dx)) (likewise sy), so that the crossing
    decisions are the kernel's.
"""

from __future__ import annotations

import numpy as np

__all__ = ["colormap_rgba", "pack_rgba", "marching_squares", "member_divergence32", "spaghetti_contours"]

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


# --------------------------------------------------------------------------
# Isocontour segments (reading R18)
# --------------------------------------------------------------------------
def _centre32(f0, f1, f2, f3):
    """The saddle decider's centre value in fp32: ((f0 + f1) + (f2 + f3)) * 0.25."""
    a = (np.float32(f0) + np.float32(f1)).astype(_F)
    b = (np.float32(f2) + np.float32(f3)).astype(_F)
    return ((a + b).astype(_F) * _F(0.25)).astype(_F)


def marching_squares(f, isovalues):
    """Isocontour segments of the scalar field f [H, W] for every isovalue
    (reading R18).  returns (keys int64 [n], segs float64 [n, 4]) in key order."""
    f = np.asarray(f, np.float64)
    h, w = f.shape
    iso = np.atleast_1d(np.asarray(isovalues, np.float32))
    kk = iso.size
    f0, f1 = f[:-1, :-1], f[:-1, 1:]      # v0 = (i, j), v1 = (i+1, j)
    f3, f2 = f[1:, :-1], f[1:, 1:]        # v3 = (i, j+1), v2 = (i+1, j+1)
    jj, ii = np.meshgrid(np.arange(h - 1, dtype=np.float64), np.arange(w - 1, dtype=np.float64), indexing="ij")
    finite = ~(np.isnan(f0) | np.isnan(f1) | np.isnan(f2) | np.isnan(f3))
    cen = _centre32(f0, f1, f2, f3).astype(np.float64)
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
            with_v0 = saddle & ((cen < c) == b0)
            for sel, pairs in ((with_v0, ((0, 1), (2, 3))), (saddle & ~with_v0, ((0, 3), (1, 2)))):
                for s_idx, (a, b) in enumerate(pairs):
                    keys.append(((cell[sel] * kk + k) * 2 + s_idx).ravel())
                    segs.append(np.concatenate([p[a][sel], p[b][sel]], -1))
    keys = np.concatenate(keys) if keys else np.zeros(0, np.int64)
    segs = np.concatenate(segs) if segs else np.zeros((0, 4))
    order = np.argsort(keys, kind="stable")
    return keys[order], segs[order].reshape(-1, 4)


def member_divergence32(u, v, dx: float, dy: float):
    """Eq. 1 divergence of every member in IEEE fp32 with the operation order of
    reading R18.  u, v [M, H, W]; returns float32 [M, H, W]."""
    u = np.asarray(u, _F)
    v = np.asarray(v, _F)
    _, h, w = u.shape
    i = np.arange(w)
    il, ih = np.maximum(i - 1, 0), np.minimum(i + 1, w - 1)
    j = np.arange(h)
    jl, jh = np.maximum(j - 1, 0), np.minimum(j + 1, h - 1)
    sx = np.where(ih - il == 2, _F(0.5 / dx), _F(1.0 / dx)).astype(_F)[None, None, :]
    sy = np.where(jh - jl == 2, _F(0.5 / dy), _F(1.0 / dy)).astype(_F)[None, :, None]
    gx = ((u[:, :, ih] - u[:, :, il]).astype(_F) * sx).astype(_F)
    gy = ((v[:, jh, :] - v[:, jl, :]).astype(_F) * sy).astype(_F)
    return (gx + gy).astype(_F)


def spaghetti_contours(u, v, dx: float, dy: float, isovalues):
    """Isocontours of every member's divergence (Fig. 1b), reading R18.
    returns (keys int64 [n], segs float64 [n, 4]) in key order."""
    d = member_divergence32(u, v, dx, dy)
    m, h, w = d.shape
    kk = np.atleast_1d(np.asarray(isovalues)).size
    per = (h - 1) * (w - 1) * kk * 2
    keys, segs = [], []
    for mm in range(m):
        k_m, s_m = marching_squares(d[mm], isovalues)
        keys.append(k_m + mm * per)
        segs.append(s_m)
    return np.concatenate(keys), np.concatenate(segs)
