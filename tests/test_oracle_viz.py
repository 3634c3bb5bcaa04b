"""Pins of the visual-output oracle (CPU only).

Colour map (reading R17): exact integer byte formulas on dyadic inputs (where
every fp32 step is exact), the stops' own colours, interpolation midpoints
worked by hand, clamping and special values, and monotonicity."""

import math

import numpy as np
import pytest

from oracle import viz as V

GREY = [(0.0, 0.0, 0.0, 0.0, 0.0), (1.0, 1.0, 1.0, 1.0, 1.0)]


def test_grey_ramp_bytes_are_round_half_up_of_255t():
    """Two stops 0 -> 1: ch = t, byte = floor(255 t + 1/2); for t = k/256 every
    fp32 step is exact, so the byte is floor((255 k + 128) / 256) in integers."""
    k = np.arange(257)
    for vmin, vmax in ((0.0, 1.0), (-2.0, 2.0), (8.0, 24.0)):
        x = vmin + (vmax - vmin) * k / 256.0
        got = V.colormap_rgba(x, vmin, vmax, GREY)
        want = (255 * k + 128) // 256
        for ch in range(4):
            assert np.array_equal(got[:, ch], want.astype(np.uint8)), (vmin, vmax, ch)


def test_stops_reproduce_their_own_colours():
    stops = [(0.0, 0.0, 0.25, 0.5, 1.0), (0.25, 0.75, 1.0, 0.0, 0.5), (0.5, 1.0, 0.5, 0.25, 0.0),
             (1.0, 0.125, 0.0, 1.0, 1.0)]
    x = np.array([0.0, 0.25, 0.5, 1.0])
    got = V.colormap_rgba(x, 0.0, 1.0, stops)
    # byte of c: floor(255 c + 1/2); by hand for c in {0, 1/8, 1/4, 1/2, 3/4, 1}
    b = {0.0: 0, 0.125: 32, 0.25: 64, 0.5: 128, 0.75: 191, 1.0: 255}
    for r, s in enumerate(stops):
        assert list(got[r]) == [b[c] for c in s[1:]], r


def test_interpolation_midpoints_by_hand():
    stops = [(0.0, 0.0, 0.0, 0.0, 0.0), (0.5, 1.0, 0.5, 0.25, 0.0), (1.0, 0.0, 1.0, 1.0, 1.0)]
    got = V.colormap_rgba(np.array([0.25, 0.75, 0.5]), 0.0, 1.0, stops)
    # t = 1/4: halfway to stop 1 -> (1/2, 1/4, 1/8, 0) -> (128, 64, 32, 0)
    assert list(got[0]) == [128, 64, 32, 0]
    # t = 3/4: halfway from stop 1 to stop 2 -> (1/2, 3/4, 5/8, 1/2); 255 * 5/8 + 1/2 = 159.875
    # -> (128, 191, 159, 128)
    assert list(got[1]) == [128, 191, 159, 128]
    # t exactly on stop 1 takes stop 1's segment (t_s <= t) with f = 0
    assert list(got[2]) == [255, 128, 64, 0]


def test_clamping_and_special_values():
    stops = [(0.0, 0.0, 0.0, 1.0, 1.0), (1.0, 1.0, 0.0, 0.0, 1.0)]
    nan_c = V.pack_rgba(1, 2, 3, 4)
    x = np.array([-5.0, -math.inf, 7.0, math.inf, math.nan, 0.5])
    got = V.colormap_rgba(x, 0.0, 1.0, stops, nan_rgba=nan_c)
    assert list(got[0]) == [0, 0, 255, 255] and list(got[1]) == [0, 0, 255, 255]
    assert list(got[2]) == [255, 0, 0, 255] and list(got[3]) == [255, 0, 0, 255]
    assert list(got[4]) == [1, 2, 3, 4]
    assert list(got[5]) == [128, 0, 128, 255]


def test_mask_paints_contour_cells_but_not_nan():
    x = np.array([[0.1, 0.2], [math.nan, 0.4]])
    mask = np.array([[True, False], [True, True]])
    got = V.colormap_rgba(x, 0.0, 1.0, GREY, nan_rgba=0, mask=mask, mask_rgba=V.pack_rgba(0, 255, 255, 255))
    assert list(got[0, 0]) == [0, 255, 255, 255] and list(got[1, 1]) == [0, 255, 255, 255]
    assert list(got[1, 0]) == [0, 0, 0, 0]
    assert list(got[0, 1]) == [51, 51, 51, 51]  # floor(255 * 0.2 + 0.5) = 51


def test_monotone_channel_is_non_decreasing():
    g = np.random.Generator(np.random.PCG64(5))
    x = np.sort(g.normal(0.0, 1.0, 5000))
    stops = [(0.0, 0.0, 0.3, 0.0, 1.0), (0.3, 0.2, 0.1, 0.0, 1.0), (0.7, 0.9, 0.8, 0.0, 1.0), (1.0, 1.0, 0.0, 0.0, 1.0)]
    got = V.colormap_rgba(x, -2.0, 2.0, stops)
    assert np.all(np.diff(got[:, 0].astype(int)) >= 0)
    assert x[0] < -2.0 and x[-1] > 2.0  # both clamped ends are reached
    assert got[0, 0] == 0 and got[-1, 0] == 255


def test_overflowing_range_maps_infinities_like_maxnum():
    """vmax - vmin overflows to inf, so R = 0 and x = +inf gives inf * 0 = NaN;
    maxNum turns it into 0, so +inf takes the first stop's colour."""
    got = V.colormap_rgba(np.array([np.inf, 1.0]), -3e38, 3e38, GREY)
    assert list(got[0]) == [0, 0, 0, 0] and list(got[1]) == [0, 0, 0, 0]


# ---------------------------------------------------------------------------
# Marching squares (reading R18)
# ---------------------------------------------------------------------------
import itertools  # noqa: E402

import oracle as O  # noqa: E402

# corner -> (row, col) of the 2 x 2 field: v0 = (i, j), v1 = (i+1, j), v2 = (i+1, j+1), v3 = (i, j+1)
_RC = {0: (0, 0), 1: (0, 1), 2: (1, 1), 3: (1, 0)}
# edge midpoints of the unit cell at t = 1/2: E0 bottom, E1 right, E2 top, E3 left
_MID = {0: (0.5, 0.0), 1: (1.0, 0.5), 2: (0.5, 1.0), 3: (0.0, 0.5)}


@pytest.mark.parametrize("code", range(16))
def test_every_cell_case_by_hand(code):
    """Corners below the isovalue 0 take -1, the others +1, so every crossing
    point is an edge midpoint; the saddles' centre is 0 (not below)."""
    f = np.empty((2, 2))
    for v in range(4):
        f[_RC[v]] = -1.0 if (code >> v) & 1 else 1.0
    keys, segs = V.marching_squares(f, [0.0])
    below = [(code >> v) & 1 for v in range(4)]
    cross = [e for e, (a, b) in enumerate(((0, 1), (1, 2), (3, 2), (0, 3))) if below[a] != below[b]]
    if code in (0, 15):
        want = []
    elif code in (5, 10):
        # centre 0 is not below: it joins the corners that are not below
        want = [(0, 3), (1, 2)] if below[0] else [(0, 1), (2, 3)]
    else:
        want = [tuple(cross)]
    assert list(keys) == list(range(len(want)))
    for s, (a, b) in zip(segs, want):
        assert tuple(s) == _MID[a] + _MID[b]


def test_linear_field_endpoints_lie_on_the_level_line():
    g = np.random.Generator(np.random.PCG64(21))
    a, b, d0 = 0.37, -0.81, 0.2
    y, x = np.mgrid[0:23, 0:31].astype(np.float64)
    f = a * x + b * y + d0
    iso = [-5.0, -1.25, 0.0, 2.25]  # exact in fp32, the isovalues' type
    keys, segs = V.marching_squares(f, iso)
    assert keys.size > 40 and np.all(np.diff(keys) > 0)
    k_of = (keys // 2) % len(iso)
    c = np.asarray(iso)[k_of]
    for p in (segs[:, :2], segs[:, 2:]):
        assert np.max(np.abs(a * p[:, 0] + b * p[:, 1] + d0 - c)) < 1e-12
    assert np.all(keys % 2 == 0)  # a plane has no saddles: one segment per crossing cell
    cells = keys // 2 // len(iso)
    crossing = O.mean_field_crossing(f, iso)
    for k in range(len(iso)):
        got = np.sort(cells[k_of == k])
        want = np.flatnonzero(crossing[k].ravel())
        assert np.array_equal(got, want)
    del g


def test_segments_sit_exactly_on_the_crossing_cells_of_random_fields():
    g = np.random.Generator(np.random.PCG64(22))
    f = g.normal(0, 1, (17, 19))
    iso = [-0.5, 0.0, 0.9]
    keys, _ = V.marching_squares(f, iso)
    crossing = O.mean_field_crossing(f, iso)
    k_of = (keys // 2) % 3
    cells = keys // 2 // 3
    for k in range(3):
        assert set(cells[k_of == k].tolist()) == set(np.flatnonzero(crossing[k].ravel()).tolist())


def test_closed_contour_every_endpoint_shared_by_two_segments():
    y, x = np.mgrid[0:40, 0:40].astype(np.float64)
    f = np.hypot(x - 19.3, y - 20.1)
    keys, segs = V.marching_squares(f, [11.7])
    pts = {}
    for s in segs:
        for p in ((s[0], s[1]), (s[2], s[3])):
            pts[p] = pts.get(p, 0) + 1
    assert len(segs) > 50 and set(pts.values()) == {2}


def test_nan_corner_cells_give_no_segments():
    f = np.array([[0.0, 1.0, 0.0], [1.0, np.nan, 1.0], [0.0, 1.0, 0.0]])
    keys, _ = V.marching_squares(f, [0.5])
    assert keys.size == 0


def test_member_divergence32_fixed_fp32_order():
    g = np.random.Generator(np.random.PCG64(23))
    u = g.normal(0, 1, (3, 6, 7)).astype(np.float32)
    v = g.normal(0, 1, (3, 6, 7)).astype(np.float32)
    d = V.member_divergence32(u, v, 0.5, 2.0)
    assert d.dtype == np.float32
    ref = O.divergence_of_field(u, v, 0.5, 2.0)
    assert np.max(np.abs(d - ref)) <= 4 * 2.0 ** -24 * np.max(np.abs(ref)) * 8
    # dyadic members: every fp32 step is exact
    ud = (g.integers(-64, 64, (2, 5, 6)) / 8.0).astype(np.float32)
    vd = (g.integers(-64, 64, (2, 5, 6)) / 8.0).astype(np.float32)
    assert np.array_equal(V.member_divergence32(ud, vd, 0.5, 0.25), O.divergence_of_field(ud, vd, 0.5, 0.25))


def test_spaghetti_keys_offset_by_member():
    g = np.random.Generator(np.random.PCG64(24))
    u = g.normal(0, 1, (4, 9, 8)).astype(np.float32)
    v = g.normal(0, 1, (4, 9, 8)).astype(np.float32)
    keys, segs = V.spaghetti_contours(u, v, 1.0, 1.0, [0.0, 0.4])
    per = 8 * 7 * 2 * 2
    d = V.member_divergence32(u, v, 1.0, 1.0)
    for m in range(4):
        sel = (keys // per) == m
        k_m, s_m = V.marching_squares(d[m], [0.0, 0.4])
        assert np.array_equal(keys[sel] - m * per, k_m) and np.array_equal(segs[sel], s_m)
    assert np.all(np.diff(keys) > 0)
