"""Pins of the visual-output oracle (CPU only).

Colour map (reading R17): exact integer byte formulas on dyadic inputs, the
stops' own colours, interpolation midpoints worked by hand, rational
arithmetic for the levels, clamping and special values, and monotonicity.
Marching squares (reading R18): all 16 cell cases by hand, the saddle decided
by the exact centre value, linear fields (endpoints on the level line),
agreement with the crossing mask, closed loops, NaN cells, and spaghetti
contours of linear members."""

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


def test_range_beyond_fp32_is_plain_arithmetic_in_fp64():
    """The map is a statement about real numbers: a range wider than fp32 can
    hold still maps its midpoint to the middle of a grey ramp, +inf to the top
    and -inf to the bottom."""
    got = V.colormap_rgba(np.array([np.inf, 0.0, -np.inf]), -3e38, 3e38, GREY)
    assert list(got[0]) == [255] * 4 and list(got[1]) == [128] * 4 and list(got[2]) == [0] * 4


def test_levels_are_the_exact_affine_interpolant():
    """255 ch + 1/2 inside a segment is affine in x with the slope fixed by the
    stop table and the range: check it against rationals."""
    from fractions import Fraction as Fr
    stops = [(0.0, 0.0, 0.25, 0.5, 1.0), (0.3, 0.7, 0.1, 0.9, 0.0), (1.0, 1.0, 1.0, 0.0, 0.5)]
    xs = [-0.7, -0.2, 0.1, 0.35, 0.9]
    y, s = V.colormap_levels(np.array(xs), -0.5, 1.0, stops)
    for n, x in enumerate(xs):
        t = min(max((Fr(x) - Fr(-0.5)) / (Fr(1.0) - Fr(-0.5)), Fr(0)), Fr(1))
        q = 1 if t >= Fr(0.3) else 0
        assert s[n] == q
        a, b = stops[q], stops[q + 1]
        f = (t - Fr(a[0])) / (Fr(b[0]) - Fr(a[0]))
        for ch in range(4):
            want = 255 * (Fr(a[1 + ch]) + f * (Fr(b[1 + ch]) - Fr(a[1 + ch]))) + Fr(1, 2)
            assert abs(y[n, ch] - float(want)) <= 1e-12


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


def test_saddle_pairing_follows_the_exact_centre_value():
    """A saddle whose corners sum to a tiny positive number: the centre
    (f0 + f1 + f2 + f3) / 4 = 2^-42 lies above c = 0 (not below), so the
    below corners v0 and v2 are cut off separately: (E0, E3) and (E1, E2).
    With the sign flipped the centre is below, on v0's side, and the
    segments are (E0, E1) and (E2, E3).  A fp32 centre ((f0 + f1) + (f2 + f3))
    * 0.25 would round both to 0 and take the first pairing twice."""
    tiny = 2.0 ** -40
    f = np.array([[-1.0, 1.0 + tiny], [1.0, -1.0]])  # v0 = -1, v1 = 1 + tiny, v3 = 1, v2 = -1
    keys, segs = V.marching_squares(f, [0.0])
    assert list(keys) == [0, 1]
    # v0 below, centre not below (v0's side is "below"): pairs (E0, E3) and (E1, E2)
    assert segs[0][1] == 0.0 and segs[0][2] == 0.0      # E0 then E3
    assert segs[1][0] == 1.0 and segs[1][3] == 1.0      # E1 then E2
    f2 = np.array([[-1.0 - tiny, 1.0], [1.0, -1.0]])     # centre -2^-42: below, v0's side
    keys, segs = V.marching_squares(f2, [0.0])
    assert segs[0][1] == 0.0 and segs[0][2] == 1.0      # E0 then E1
    assert segs[1][1] == 1.0 and segs[1][2] == 0.0      # E2 then E3


def test_spaghetti_keys_offset_by_member():
    g = np.random.Generator(np.random.PCG64(24))
    u = g.normal(0, 1, (4, 9, 8)).astype(np.float32)
    v = g.normal(0, 1, (4, 9, 8)).astype(np.float32)
    keys, segs = V.spaghetti_contours(u, v, 1.0, 1.0, [0.0, 0.4])
    per = 8 * 7 * 2 * 2
    d = O.divergence_of_field(u, v, 1.0, 1.0)
    for m in range(4):
        sel = (keys // per) == m
        k_m, s_m = V.marching_squares(d[m], [0.0, 0.4])
        assert np.array_equal(keys[sel] - m * per, k_m) and np.array_equal(segs[sel], s_m)
    assert np.all(np.diff(keys) > 0)


def test_spaghetti_of_a_linear_member_lies_on_its_level_line():
    """Eq. 1 is exact on linear members (u = a x, v = b y gives divergence
    a/dx' + b/dy' per unit index), so every endpoint of a member's contour at c
    lies where that member's divergence plane equals c."""
    h, w = 12, 15
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    u = np.stack([0.3 * x * x, -0.2 * x * x])            # divergence 0.6 x / dx (central), -0.4 x / dx
    v = np.stack([0.1 * y * y, 0.5 * y * y])
    dx, dy = 0.5, 2.0
    keys, segs = V.spaghetti_contours(u, v, dx, dy, [1.5])
    d = O.divergence_of_field(u, v, dx, dy)
    per = (h - 1) * (w - 1) * 2
    for k, s in zip(keys, segs):
        m = k // per
        for px, py in ((s[0], s[1]), (s[2], s[3])):
            # bilinear interpolation of the member's divergence at the endpoint equals c on an edge
            i0, j0 = min(int(np.floor(px)), w - 2), min(int(np.floor(py)), h - 2)
            fx, fy = px - i0, py - j0
            val = ((1 - fx) * (1 - fy) * d[m, j0, i0] + fx * (1 - fy) * d[m, j0, i0 + 1]
                   + (1 - fx) * fy * d[m, j0 + 1, i0] + fx * fy * d[m, j0 + 1, i0 + 1])
            assert abs(val - 1.5) < 1e-9
    assert keys.size > 10
