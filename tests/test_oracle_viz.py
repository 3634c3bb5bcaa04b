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
