"""Pins of the 3D extension of the oracle (reading R20; CPU only).

Linear fields are differentiated exactly; exact rational arithmetic on integer
statistics; z-invariant fields with w = 0 reduce to the pinned 2D oracle (two
identical layers: LCP = 1 - P4^2 - Q4^2); relabelling the axes transposes every
result; brute-force sampling of the fitted Gaussians with an independent
generator and an explicit triple-loop stencil reproduces the closed form on
interior cells; zero variance gives the crossing indicator."""

import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from oracle import volume as V3


def _stats(g, d, h, w):
    mu = [g.normal(0, 1, (d, h, w)) for _ in range(3)]
    var = [g.uniform(0.05, 0.6, (d, h, w)) for _ in range(3)]
    return mu, var


def test_linear_field_divergence_is_exact():
    d, h, w = 4, 5, 6
    dx, dy, dz = 0.5, 2.0, 0.25
    k, j, i = np.meshgrid(np.arange(d), np.arange(h), np.arange(w), indexing="ij")
    a, b, c = 1.5, -0.75, 0.125
    u, v, ww = a * i * dx, b * j * dy, c * k * dz
    div = V3.divergence_of_field_3d(u, v, ww, dx, dy, dz)
    assert np.array_equal(div, np.full((d, h, w), a + b + c))
    zero = np.zeros((d, h, w))
    mu, var = V3.divergence_gaussian_3d(u, zero, v, zero, ww, zero, dx, dy, dz)
    assert np.array_equal(mu, div) and np.array_equal(var, zero)
    lcp = V3.level_crossing_probability_3d(mu, var, [a + b + c + 0.5, a + b + c - 0.5])
    assert np.array_equal(lcp, np.zeros_like(lcp))  # constant field: never crosses


def test_divergence_gaussian_rational_arithmetic():
    g = np.random.Generator(np.random.PCG64(2))
    d, h, w = 3, 4, 5
    ints = [g.integers(-9, 10, (d, h, w)).astype(np.float64) for _ in range(6)]
    ints[1], ints[3], ints[5] = np.abs(ints[1]), np.abs(ints[3]), np.abs(ints[5])
    dx, dy, dz = 0.5, 1.0, 2.0
    mu, var = V3.divergence_gaussian_3d(*ints, dx, dy, dz)
    for kk, jj, ii in itertools.product(range(d), range(h), range(w)):
        def diff(arr, axis, neg):
            n = arr.shape[axis]
            lo, hi = [kk, jj, ii], [kk, jj, ii]
            c = [kk, jj, ii][axis]
            lo[axis], hi[axis] = max(c - 1, 0), min(c + 1, n - 1)
            step = Fraction(hi[axis] - lo[axis]) * Fraction([dz, dy, dx][axis])
            a_hi, a_lo = Fraction(arr[tuple(hi)]), Fraction(arr[tuple(lo)])
            return (a_hi - a_lo) / step if not neg else (a_hi + a_lo) / step ** 2
        want_mu = diff(ints[0], 2, False) + diff(ints[2], 1, False) + diff(ints[4], 0, False)
        want_var = diff(ints[1], 2, True) + diff(ints[3], 1, True) + diff(ints[5], 0, True)
        assert mu[kk, jj, ii] == float(want_mu)
        assert var[kk, jj, ii] == float(want_var)


def test_z_invariant_fields_reduce_to_the_2d_oracle():
    g = np.random.Generator(np.random.PCG64(3))
    h, w, d = 6, 7, 3
    mu2 = [g.normal(0, 1, (h, w)) for _ in range(2)]
    var2 = [g.uniform(0.1, 0.5, (h, w)) for _ in range(2)]
    mu_d2, var_d2 = O.divergence_gaussian(mu2[0], var2[0], mu2[1], var2[1], 1.0, 0.5)
    rep = lambda a: np.repeat(a[None], d, axis=0)  # noqa: E731
    zero = np.zeros((d, h, w))
    mu_d3, var_d3 = V3.divergence_gaussian_3d(rep(mu2[0]), rep(var2[0]), rep(mu2[1]), rep(var2[1]), zero, zero,
                                              1.0, 0.5, 3.0)
    assert np.allclose(mu_d3, rep(mu_d2), rtol=0, atol=1e-15)
    assert np.allclose(var_d3, rep(var_d2), rtol=0, atol=1e-15)
    iso = [float(np.median(mu_d2)), -0.3]
    lcp3 = V3.level_crossing_probability_3d(mu_d3, var_d3, iso)
    for kk, c in enumerate(iso):
        p, q = O.below_above_probabilities(mu_d2, var_d2, c)
        p4 = p[:-1, :-1] * p[:-1, 1:] * p[1:, :-1] * p[1:, 1:]
        q4 = q[:-1, :-1] * q[:-1, 1:] * q[1:, :-1] * q[1:, 1:]
        for layer in range(d - 1):
            assert np.allclose(lcp3[kk, layer], 1.0 - p4 * p4 - q4 * q4, rtol=0, atol=1e-14)


def test_relabelling_the_axes_transposes_the_results():
    """Swap x and z: u <-> w with their axes transposed and dx <-> dz."""
    g = np.random.Generator(np.random.PCG64(4))
    d, h, w = 4, 5, 6
    (mu_u, mu_v, mu_w), (var_u, var_v, var_w) = _stats(g, d, h, w)
    dx, dy, dz = 0.5, 1.0, 2.0
    mu, var = V3.divergence_gaussian_3d(mu_u, var_u, mu_v, var_v, mu_w, var_w, dx, dy, dz)
    T = lambda a: np.transpose(a, (2, 1, 0))  # noqa: E731
    mu_t, var_t = V3.divergence_gaussian_3d(T(mu_w), T(var_w), T(mu_v), T(var_v), T(mu_u), T(var_u), dz, dy, dx)
    assert np.allclose(mu_t, T(mu), rtol=0, atol=1e-13) and np.allclose(var_t, T(var), rtol=0, atol=1e-13)
    iso = [0.0, 0.7]
    a = V3.level_crossing_probability_3d(mu, var, iso)
    b = V3.level_crossing_probability_3d(mu_t, var_t, iso)
    assert np.allclose(b, np.transpose(a, (0, 3, 2, 1)), rtol=0, atol=1e-13)
    assert np.array_equal(V3.mean_field_crossing_3d(mu_t, iso),
                          np.transpose(V3.mean_field_crossing_3d(mu, iso), (0, 3, 2, 1)))


def test_brute_force_sampling_matches_the_closed_form_on_interior_cells():
    """Sample every vertex component from its fitted Gaussian (independent
    generator), take the stencil with explicit loops, test the 8-vertex
    crossing; interior cells share no stencil input, so the frequency must
    match the closed form within the binomial error."""
    g = np.random.Generator(np.random.PCG64(5))
    d = h = w = 5
    (mu_u, mu_v, mu_w), (var_u, var_v, var_w) = _stats(g, d, h, w)
    mu_d, var_d = V3.divergence_gaussian_3d(mu_u, var_u, mu_v, var_v, mu_w, var_w, 1.0, 1.0, 1.0)
    c = float(np.median(mu_d))
    want = V3.level_crossing_probability_3d(mu_d, var_d, [c])[0]
    rs = np.random.RandomState(12345)  # a different generator from the test data's
    n = 40000
    cnt = np.zeros((d - 1, h - 1, w - 1))
    for _ in range(n // 2000):
        U = mu_u + np.sqrt(var_u) * rs.standard_normal((2000, d, h, w))
        Vv = mu_v + np.sqrt(var_v) * rs.standard_normal((2000, d, h, w))
        Wv = mu_w + np.sqrt(var_w) * rs.standard_normal((2000, d, h, w))
        D = np.zeros((2000, d, h, w))
        for k in range(d):
            for j in range(h):
                for i in range(w):
                    il, ih = max(i - 1, 0), min(i + 1, w - 1)
                    jl, jh = max(j - 1, 0), min(j + 1, h - 1)
                    kl, kh = max(k - 1, 0), min(k + 1, d - 1)
                    D[:, k, j, i] = ((U[:, k, j, ih] - U[:, k, j, il]) / (ih - il)
                                     + (Vv[:, k, jh, i] - Vv[:, k, jl, i]) / (jh - jl)
                                     + (Wv[:, kh, j, i] - Wv[:, kl, j, i]) / (kh - kl))
        below = D < c
        for k in range(d - 1):
            for j in range(h - 1):
                for i in range(w - 1):
                    cube = below[:, k:k + 2, j:j + 2, i:i + 2].reshape(2000, 8)
                    cnt[k, j, i] += np.sum(cube.any(axis=1) & ~cube.all(axis=1))
    freq = cnt / n
    inner = (slice(1, -1),) * 3
    err = np.abs(freq[inner] - want[inner])
    tol = 5.0 * np.sqrt(want[inner] * (1 - want[inner]) / n) + 1e-3
    assert np.all(err <= tol), float(np.max(err - tol))


@pytest.mark.parametrize("seed", [6, 7])
def test_zero_variance_is_the_crossing_indicator(seed):
    g = np.random.Generator(np.random.PCG64(seed))
    mu = g.normal(0, 1, (4, 5, 6))
    iso = [0.0, 0.5, -1.0]
    lcp = V3.level_crossing_probability_3d(mu, np.zeros_like(mu), iso)
    cross = V3.mean_field_crossing_3d(mu, iso)
    assert np.array_equal(lcp, cross.astype(np.float64))
    # the crossing test by brute force: some vertex below and some not below
    for kk, c in enumerate(iso):
        for k, j, i in itertools.product(range(3), range(4), range(5)):
            cube = mu[k:k + 2, j:j + 2, i:i + 2] < c
            assert cross[kk, k, j, i] == (cube.any() and not cube.all())


def test_closed_form_3d_from_members():
    g = np.random.Generator(np.random.PCG64(8))
    u, v, w = (g.normal(0, 1, (6, 3, 4, 5)) for _ in range(3))
    r = V3.lcp_closed_form_3d(u, v, w, 1.0, 1.0, 1.0, [0.1])
    mu_d, var_d = V3.divergence_gaussian_3d(u.mean(0), u.var(0, ddof=1), v.mean(0), v.var(0, ddof=1),
                                            w.mean(0), w.var(0, ddof=1), 1.0, 1.0, 1.0)
    assert np.allclose(r["mu_d"], mu_d, atol=1e-14) and np.allclose(r["var_d"], var_d, atol=1e-14)
    assert np.all((r["lcp"] >= 0) & (r["lcp"] <= 1))
