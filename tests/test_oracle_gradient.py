"""Pins of the speed-gradient preprocessing (Sec. 4.2, reading R19; CPU only).

numpy's own gradient routine (central differences inside, first order at the
ends) is an independent statement of the stencil; Pythagorean members give
exact speeds; a quadratic speed is differentiated exactly by central
differences; identical members reduce the LCP to the mean-field crossing."""

import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("shape,dx,dy", [((4, 7, 9), 1.0, 1.0), ((2, 2, 5), 0.25, 3.0), ((3, 6, 2), 2.0, 0.5)])
def test_gradient_equals_numpy_gradient(shape, dx, dy):
    g = np.random.Generator(np.random.PCG64(sum(shape)))
    u = g.normal(0, 1, shape)
    v = g.normal(0, 1, shape)
    gx, gy = O.speed_gradient(u, v, dx, dy)
    s = np.hypot(u, v)
    assert np.allclose(gx, np.gradient(s, dx, axis=-1, edge_order=1), rtol=0, atol=1e-14)
    assert np.allclose(gy, np.gradient(s, dy, axis=-2, edge_order=1), rtol=0, atol=1e-14)


def test_pythagorean_members_give_exact_speed_and_gradient():
    """u = 3 x, v = 4 x (x = column index >= 0): s = 5 x exactly, so gx = 5 / dx
    at every column (one-sided ends included) and gy = 0."""
    x = np.arange(6, dtype=np.float64)[None, None, :].repeat(4, axis=1)
    u, v = 3.0 * x, 4.0 * x
    gx, gy = O.speed_gradient(u, v, 0.5, 1.0)
    assert np.array_equal(gx, np.full_like(gx, 10.0))
    assert np.array_equal(gy, np.zeros_like(gy))


def test_quadratic_speed_central_difference_is_exact():
    """s = y^2 (u = y^2, v = 0, rows y = 0..H-1): (s[j+1] - s[j-1]) / 2 = 2 y
    inside; the ends take (1 - 0) and (y_n^2 - y_{n-1}^2)."""
    h = 7
    y = np.arange(h, dtype=np.float64)[:, None].repeat(3, axis=1)[None]
    gx, gy = O.speed_gradient(y * y, np.zeros_like(y), 1.0, 1.0)
    want = 2.0 * np.arange(h, dtype=np.float64)
    want[0] = 1.0
    want[-1] = (h - 1) ** 2 - (h - 2) ** 2
    assert np.array_equal(gy[0, :, 0], want)
    assert np.array_equal(gx, np.zeros_like(gx))


def test_identical_members_reduce_to_the_crossing_indicator():
    """Identical members: zero variance, so the LCP is the crossing indicator.
    Members u = 3a, v = 4a with small integers a: speeds 5|a| and their
    gradients are exact, so the ensemble statistics are exact too."""
    g = np.random.Generator(np.random.PCG64(9))
    a = g.integers(-5, 6, size=(1, 9, 11)).astype(np.float64)
    one_u, one_v = 3.0 * a, 4.0 * a
    u, v = one_u.repeat(5, axis=0), one_v.repeat(5, axis=0)
    gx, gy = O.speed_gradient(one_u, one_v, 1.0, 1.0)
    div = O.divergence_of_field(gx[0], gy[0], 1.0, 1.0)
    iso = [float(np.median(div)) + 0.125, float(np.quantile(div, 0.2)) - 0.125]
    r = O.speed_gradient_lcp(u, v, 1.0, 1.0, iso)
    assert np.array_equal(r["var_d"], np.zeros_like(r["var_d"]))
    assert np.array_equal(r["lcp"], O.mean_field_crossing(div, iso).astype(np.float64))


def test_gradient_members_feed_the_closed_form_unchanged():
    g = np.random.Generator(np.random.PCG64(4))
    u = g.normal(1.0, 0.3, (6, 8, 10))
    v = g.normal(-0.5, 0.3, (6, 8, 10))
    gx, gy = O.speed_gradient(u, v, 1.5, 0.75)
    r = O.speed_gradient_lcp(u, v, 1.5, 0.75, [0.0, 0.1])
    want = O.lcp_closed_form(gx, gy, 1.5, 0.75, [0.0, 0.1])
    assert np.array_equal(r["lcp"], want["lcp"])
    assert np.allclose(r["mu_u"], gx.mean(axis=0), rtol=0, atol=1e-14)
