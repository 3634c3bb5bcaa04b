"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against something the paper or mathematics fixes:
exact rational arithmetic, closed forms, the paper's Fig. 2 worked example,
brute-force sampling with an independent generator (numpy PCG64), an
independent Philox implementation, or brute-force enumeration.  A plausible
slip in the oracle (dropped term, wrong sign, swapped dx/dy, 2dx instead of dx
at the boundary, p/q swapped, wrong crossing rule) fails at least one of them.
"""

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats as sps

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Ensemble statistics
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ddof", [0, 1])
def test_stats_match_exact_rational_arithmetic(ddof):
    g = np.random.default_rng(11)
    x = g.integers(-50, 50, size=(7, 3, 4)).astype(np.float64) / 8.0
    mean, var = O.ensemble_stats(x, ddof)
    for j in range(3):
        for i in range(4):
            vals = [Fraction(float(t)) for t in x[:, j, i]]
            mu = sum(vals) / len(vals)
            s2 = sum((t - mu) ** 2 for t in vals) / (len(vals) - ddof)
            assert mean[j, i] == float(mu)
            assert abs(var[j, i] - float(s2)) <= 1e-15 * max(1.0, float(s2))


@pytest.mark.parametrize("m", [2, 5, 51])
def test_stats_arithmetic_progression_closed_form(m):
    a, h = 3.25, 0.5
    x = (a + h * np.arange(m, dtype=np.float64))[:, None, None] * np.ones((1, 2, 2))
    mean, var1 = O.ensemble_stats(x, 1)
    _, var0 = O.ensemble_stats(x, 0)
    assert np.allclose(mean, a + h * (m - 1) / 2, rtol=0, atol=1e-13)
    assert np.allclose(var1, h * h * m * (m + 1) / 12, rtol=1e-13)
    assert np.allclose(var0, h * h * (m * m - 1) / 12, rtol=1e-13)


def test_stats_large_offset_is_exact_for_two_pass():
    # a two-pass reduction does not cancel catastrophically at |mean|/sigma = 1e8
    x = 1e8 + np.array([-1.0, 0.0, 1.0])[:, None, None] * np.ones((1, 1, 1))
    mean, var = O.ensemble_stats(x, 1)
    assert mean[0, 0] == 1e8 and var[0, 0] == 1.0


# --------------------------------------------------------------------------
# Divergence Gaussian, Eqs. 1-3
# --------------------------------------------------------------------------
def _fig2():
    with open(os.path.join(GOLDEN, "fig2_stencil.json")) as f:
        return json.load(f)


def _fig2_grid():
    g = _fig2()["parameters"]
    mu_u = np.zeros((3, 3)); var_u = np.ones((3, 3))
    mu_v = np.zeros((3, 3)); var_v = np.ones((3, 3))
    # vertex (i, j) = (1, 1); arrays are [j, i]
    mu_u[1, 0], var_u[1, 0] = g["U_i_minus_1"]["mu"], g["U_i_minus_1"]["sigma"] ** 2
    mu_u[1, 2], var_u[1, 2] = g["U_i_plus_1"]["mu"], g["U_i_plus_1"]["sigma"] ** 2
    mu_v[0, 1], var_v[0, 1] = g["V_j_minus_1"]["mu"], g["V_j_minus_1"]["sigma"] ** 2
    mu_v[2, 1], var_v[2, 1] = g["V_j_plus_1"]["mu"], g["V_j_plus_1"]["sigma"] ** 2
    return mu_u, var_u, mu_v, var_v


def test_fig2_worked_example():
    want = _fig2()["hand_derived_from_eqs_2_3"]
    mu_d, var_d = O.divergence_gaussian(*_fig2_grid(), 1.0, 1.0)
    assert abs(mu_d[1, 1] - want["mu"]) < 1e-14
    assert abs(var_d[1, 1] - want["var"]) < 1e-14


def test_fig2_mc_errors_have_the_papers_magnitude():
    """Fig. 2 table: the MC errors of the divergence mean/std at 1e3 and 1e5
    samples.  Seeds are unknown, so the check is statistical: (a) the paper's
    errors are within 3 standard errors of 0 under Eqs. 2/3, and (b) our own
    sampling of the same stencil through Eq. 1 has errors of the same law."""
    f = _fig2()
    want = f["hand_derived_from_eqs_2_3"]
    sd = math.sqrt(want["var"])
    g = f["parameters"]
    rng = np.random.default_rng(5)
    for n, key in ((1000, "samples_1e3"), (100000, "samples_1e5")):
        se_m = sd / math.sqrt(n)
        se_s = sd / math.sqrt(2 * n)
        assert f["paper_mc_errors"][key]["e_m"] < 3 * se_m
        assert f["paper_mc_errors"][key]["e_sigma"] < 3 * se_s
        reps = 200 if n == 1000 else 20
        em, es = [], []
        for _ in range(reps):
            uim = rng.normal(g["U_i_minus_1"]["mu"], g["U_i_minus_1"]["sigma"], n)
            uip = rng.normal(g["U_i_plus_1"]["mu"], g["U_i_plus_1"]["sigma"], n)
            vjm = rng.normal(g["V_j_minus_1"]["mu"], g["V_j_minus_1"]["sigma"], n)
            vjp = rng.normal(g["V_j_plus_1"]["mu"], g["V_j_plus_1"]["sigma"], n)
            u = np.zeros((n, 3, 3)); v = np.zeros((n, 3, 3))
            u[:, 1, 0], u[:, 1, 2], v[:, 0, 1], v[:, 2, 1] = uim, uip, vjm, vjp
            d = O.divergence_of_field(u, v, 1.0, 1.0)[:, 1, 1]
            em.append(d.mean() - want["mu"])
            es.append(d.std(ddof=1) - sd)
        rms_m = math.sqrt(np.mean(np.square(em)))
        assert 0.7 * se_m < rms_m < 1.4 * se_m
        assert abs(np.mean(em)) < 4 * se_m / math.sqrt(reps)
        assert math.sqrt(np.mean(np.square(es))) < 2.0 * se_s


@pytest.mark.parametrize("h,w,dx,dy", [(5, 7, 1.0, 1.0), (4, 3, 0.5, 2.0), (2, 2, 3.0, 0.25)])
def test_divergence_of_linear_field_is_exact_everywhere(h, w, dx, dy):
    # u = a x + b y, v = c x + e y with x = i dx, y = j dy: divergence a + e,
    # at the one-sided boundary vertices too; swapping dx and dy breaks it.
    a, b, c, e = 1.5, -0.75, 2.0, -0.25
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    x *= dx; y *= dy
    u, v = a * x + b * y, c * x + e * y
    d = O.divergence_of_field(u, v, dx, dy)
    assert np.allclose(d, a + e, rtol=0, atol=1e-12)
    mu_d, var_d = O.divergence_gaussian(u, np.zeros_like(u), v, np.zeros_like(v), dx, dy)
    assert np.allclose(mu_d, a + e, rtol=0, atol=1e-12)
    assert np.all(var_d == 0)


def test_boundary_rule_is_first_order_one_sided():
    # u = x^2: central difference exact (2x) inside; forward difference at i=0
    # gives dx; backward difference at i=W-1 gives (2W-3) dx.
    w, dx = 6, 0.5
    x = np.arange(w) * dx
    u = np.tile(x * x, (3, 1))
    d = O.divergence_of_field(u, np.zeros_like(u), dx, 1.0)[1]
    assert np.allclose(d[1:-1], 2 * x[1:-1], atol=1e-12)
    assert abs(d[0] - dx) < 1e-12
    assert abs(d[-1] - (2 * w - 3) * dx) < 1e-12
    # the same along y for v
    v = np.tile((x * x)[:, None], (1, 3))
    d = O.divergence_of_field(np.zeros_like(v), v, 1.0, dx)[:, 1]
    assert abs(d[0] - dx) < 1e-12 and abs(d[-1] - (2 * w - 3) * dx) < 1e-12


def test_gaussian_propagation_matches_brute_force_sampling():
    """Eqs. 2/3 (with the boundary weights) against the sample mean / variance
    of Eq. 1 on 200k independent field realisations (numpy PCG64)."""
    rng = np.random.default_rng(7)
    h, w, dx, dy = 4, 5, 0.7, 1.3
    mu_u, mu_v = rng.normal(size=(h, w)), rng.normal(size=(h, w))
    sd_u, sd_v = rng.uniform(0.2, 1.5, (h, w)), rng.uniform(0.2, 1.5, (h, w))
    mu_d, var_d = O.divergence_gaussian(mu_u, sd_u**2, mu_v, sd_v**2, dx, dy)
    n = 200_000
    acc1 = np.zeros((h, w)); acc2 = np.zeros((h, w))
    for _ in range(4):
        uu = mu_u + sd_u * rng.standard_normal((n // 4, h, w))
        vv = mu_v + sd_v * rng.standard_normal((n // 4, h, w))
        d = O.divergence_of_field(uu, vv, dx, dy)
        acc1 += d.sum(0); acc2 += (d * d).sum(0)
    m_hat = acc1 / n
    v_hat = acc2 / n - m_hat**2
    assert np.all(np.abs(m_hat - mu_d) < 5 * np.sqrt(var_d / n))
    assert np.all(np.abs(v_hat - var_d) < 5 * var_d * math.sqrt(2.0 / n))


def test_interior_vertex_divergences_are_uncorrelated_and_ring_ones_are_not():
    rng = np.random.default_rng(3)
    h, w, n = 5, 6, 100_000
    sd = rng.uniform(0.5, 1.5, (h, w))
    uu = sd * rng.standard_normal((n, h, w))
    vv = sd * rng.standard_normal((n, h, w))
    d = O.divergence_of_field(uu, vv, 1.0, 1.0)
    # interior cell (i, j) = (1, 1): vertices (1,1), (2,1), (1,2), (2,2) are all interior
    quad = np.stack([d[:, 1, 1], d[:, 1, 2], d[:, 2, 1], d[:, 2, 2]])
    rho = np.corrcoef(quad)
    assert np.all(np.abs(rho[np.triu_indices(4, 1)]) < 5 / math.sqrt(n))
    # ring: vertex i=0 (forward, uses U_0, U_1) and i=1 (central, uses U_0, U_2)
    # share U_0: Cov = sigma_0^2 / (1 * 2) for dx = 1
    cov = np.cov(d[:, 2, 0], d[:, 2, 1])[0, 1]
    assert abs(cov - sd[2, 0] ** 2 / 2) < 5 * 0.02


# --------------------------------------------------------------------------
# LCP, Sec. 3.1 (reading R1)
# --------------------------------------------------------------------------
def test_lcp_iid_vertices_closed_form():
    mu, sd, c = 0.3, 0.8, 0.1
    p = sps.norm.cdf(c, loc=mu, scale=sd)
    lcp = O.level_crossing_probability(np.full((2, 2), mu), np.full((2, 2), sd * sd), [c])
    assert abs(lcp[0, 0, 0] - (1 - p**4 - (1 - p) ** 4)) < 1e-15


def test_lcp_three_deterministic_vertices_reduce_to_a_normal_tail():
    mu_d = np.array([[-2.0, -1.0], [-3.0, 0.4]])
    var_d = np.array([[0.0, 0.0], [0.0, 0.36]])
    for c in (-0.5, 0.0, 0.4, 1.5):
        lcp = O.level_crossing_probability(mu_d, var_d, [c])[0, 0, 0]
        assert abs(lcp - sps.norm.sf(c, loc=0.4, scale=0.6)) < 1e-15


def test_lcp_zero_variance_equals_mean_field_crossing():
    rng = np.random.default_rng(1)
    mu_d = np.round(rng.normal(size=(9, 11)) * 8) / 8
    iso = [-0.25, 0.0, 0.125]
    lcp = O.level_crossing_probability(mu_d, np.zeros_like(mu_d), iso)
    mask = O.mean_field_crossing(mu_d, iso)
    assert np.array_equal(lcp, mask.astype(np.float64))


def test_mean_field_crossing_brute_force_loop():
    rng = np.random.default_rng(2)
    mu_d = np.round(rng.normal(size=(6, 7)) * 4) / 4
    iso = [0.0, 0.25]
    mask = O.mean_field_crossing(mu_d, iso)
    for k, c in enumerate(iso):
        for j in range(5):
            for i in range(6):
                vals = [mu_d[j, i], mu_d[j, i + 1], mu_d[j + 1, i], mu_d[j + 1, i + 1]]
                below = [t < c for t in vals]
                assert mask[k, j, i] == (any(below) and not all(below))


def test_lcp_matches_brute_force_sampling_of_independent_vertices():
    rng = np.random.default_rng(9)
    mu_d = rng.normal(size=(3, 4)) * 0.5
    var_d = rng.uniform(0.05, 1.0, (3, 4))
    iso = [-0.2, 0.0, 0.3]
    lcp = O.level_crossing_probability(mu_d, var_d, iso)
    n = 400_000
    d = mu_d + np.sqrt(var_d) * rng.standard_normal((n, 3, 4))
    quad = np.stack([d[:, :-1, :-1], d[:, :-1, 1:], d[:, 1:, :-1], d[:, 1:, 1:]])
    lo, hi = quad.min(0), quad.max(0)
    for k, c in enumerate(iso):
        emp = ((lo < c) & (hi >= c)).mean(0)
        se = np.sqrt(lcp[k] * (1 - lcp[k]) / n)
        assert np.all(np.abs(emp - lcp[k]) < 5 * se + 1e-9)


def test_lcp_range_symmetry_and_limits():
    rng = np.random.default_rng(4)
    mu_d = rng.normal(size=(8, 9)) * 2
    var_d = rng.uniform(0, 2, (8, 9))
    var_d[rng.random((8, 9)) < 0.1] = 0
    iso = np.array([-1.0, 0.0, 0.5])
    a = O.level_crossing_probability(mu_d, var_d, iso)
    assert np.all(a >= -1e-15) and np.all(a <= 1 + 1e-15)
    # reflection (mu - c) -> -(mu - c) swaps p and q; LCP unchanged (up to ties at var 0)
    b = O.level_crossing_probability(-mu_d, var_d, -iso)
    nz = var_d > 0
    nzc = nz[:-1, :-1] & nz[:-1, 1:] & nz[1:, :-1] & nz[1:, 1:]
    assert np.allclose(a[:, nzc], b[:, nzc], atol=1e-14)
    # transposing the grid permutes the vertices of each cell
    t = O.level_crossing_probability(mu_d.T, var_d.T, iso)
    assert np.allclose(a, np.transpose(t, (0, 2, 1)), atol=1e-15)
    far = O.level_crossing_probability(mu_d, var_d, [1e6, -1e6])
    assert np.all(far == 0)


def test_below_above_use_the_right_tail():
    p, q = O.below_above_probabilities(np.array([1.0]), np.array([4.0]), 0.0)
    assert abs(p[0] - sps.norm.cdf(0.0, 1.0, 2.0)) < 4e-16
    assert abs(q[0] - sps.norm.sf(0.0, 1.0, 2.0)) < 4e-16
    # deep tail keeps relative accuracy (no 1 - Phi cancellation)
    p, q = O.below_above_probabilities(np.array([0.0]), np.array([1.0]), 12.0)
    assert abs(q[0] / sps.norm.sf(12.0) - 1) < 1e-12


# --------------------------------------------------------------------------
# Philox-4x32-10 and Box-Muller
# --------------------------------------------------------------------------
def test_philox_published_known_answer_vectors():
    """The generator's published known-answer vectors (Random123, SC'11):
    counter and key in, four output words, bit for bit."""
    kat = json.load(open(os.path.join(GOLDEN, "philox4x32_10_kat.json")))
    for vec in kat["vectors"]:
        ctr = np.array([[int(x, 16) for x in vec["counter"]]], dtype=np.uint32)
        key = tuple(int(x, 16) for x in vec["key"])
        got = O.philox4x32_10(ctr, key)[0]
        assert [int(x) for x in got] == [int(x, 16) for x in vec["output"]]


def test_philox_matches_independent_implementation():
    """Pin against Triton's open-source Philox-4x32-10 run in its CPU interpreter."""
    os.environ.setdefault("TRITON_INTERPRET", "1")
    if os.environ.get("TRITON_INTERPRET") != "1":
        pytest.skip("Triton interpreter not enabled")
    triton = pytest.importorskip("triton")
    import torch
    import triton.language as tl

    @triton.jit
    def _k(c0p, c1p, c2p, c3p, o0, o1, o2, o3, seed, N: tl.constexpr):
        off = tl.arange(0, N)
        a, b, c, d = tl.philox(seed, tl.load(c0p + off), tl.load(c1p + off), tl.load(c2p + off),
                               tl.load(c3p + off), 10)
        tl.store(o0 + off, a); tl.store(o1 + off, b); tl.store(o2 + off, c); tl.store(o3 + off, d)

    n = 64
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    seed = int(rng.integers(0, 2**63))
    cs = [torch.from_numpy(ctr[:, i].view(np.int32).copy()) for i in range(4)]
    outs = [torch.empty(n, dtype=torch.int32) for _ in range(4)]
    _k[(1,)](*cs, *outs, seed, N=n)
    theirs = np.stack([o.numpy().view(np.uint32) for o in outs], axis=-1)
    ours = O.philox4x32_10(ctr, (seed & 0xFFFFFFFF, seed >> 32))
    assert np.array_equal(ours, theirs)


def test_philox_uniformity_and_avalanche():
    n = 1 << 16
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n)
    out = O.philox4x32_10(ctr, (123, 456))
    bins = np.bincount((out.ravel() >> np.uint32(24)).astype(np.int64), minlength=256)
    chi2 = ((bins - bins.mean()) ** 2 / bins.mean()).sum()
    assert sps.chi2.sf(chi2, 255) > 1e-4
    flipped = ctr.copy(); flipped[:, 1] ^= 1
    diff = O.philox4x32_10(flipped, (123, 456)) ^ out
    bits = np.unpackbits(diff.view(np.uint8)).mean()
    assert abs(bits - 0.5) < 0.01


def test_box_muller_identities_and_normality():
    rng = np.random.default_rng(8)
    xa = rng.integers(0, 2**32, 200_000, dtype=np.uint64).astype(np.uint32)
    xb = rng.integers(0, 2**32, 200_000, dtype=np.uint64).astype(np.uint32)
    z0, z1 = O.box_muller(xa, xb)
    u1, u2 = O.uniform01(xa), O.uniform01(xb)
    assert np.allclose(z0 * z0 + z1 * z1, -2 * np.log(u1), rtol=1e-12)
    assert np.allclose(np.mod(np.arctan2(z1, z0), 2 * np.pi), 2 * np.pi * u2, atol=1e-9)
    assert sps.kstest(z0, "norm").pvalue > 1e-3 and sps.kstest(z1, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(z0, z1)[0, 1]) < 0.01
    u = O.uniform01(np.array([0, 0xFFFFFFFF], np.uint32))
    assert u[0] == 2.0**-25 and u[1] == 1 - 2.0**-25


# --------------------------------------------------------------------------
# Monte Carlo estimator (Sec. 3.2, Sec. 4)
# --------------------------------------------------------------------------
def _small_stats(h=12, w=14, seed=0):
    rng = np.random.default_rng(seed)
    mu_u = np.cumsum(rng.normal(size=(h, w)) * 0.3, axis=1)
    mu_v = np.cumsum(rng.normal(size=(h, w)) * 0.3, axis=0)
    var_u = rng.uniform(0.05, 0.4, (h, w))
    var_v = rng.uniform(0.05, 0.4, (h, w))
    return mu_u, var_u, mu_v, var_v


def test_mc_converges_to_closed_form_on_interior_cells():
    st = _small_stats()
    mu_d, var_d = O.divergence_gaussian(*st, 1.0, 1.0)
    iso = [float(np.median(mu_d)), float(np.percentile(mu_d, 20))]
    exact = O.level_crossing_probability(mu_d, var_d, iso)
    s = 4000
    est, counts = O.mc_lcp(iso, s, seed=99, dx=1.0, dy=1.0, mode="gauss", stats=st)
    assert counts.dtype == np.int64 and counts.max() <= s
    inner = (slice(None), slice(1, -1), slice(1, -1))
    se = np.sqrt(exact[inner] * (1 - exact[inner]) / s) + 1e-12
    z = (est[inner] - exact[inner]) / se
    assert np.mean(np.abs(z) < 3) > 0.98 and np.abs(z).max() < 5.5


def test_mc_error_falls_as_inverse_sqrt_samples():
    st = _small_stats(10, 10, seed=1)
    mu_d, var_d = O.divergence_gaussian(*st, 1.0, 1.0)
    iso = [float(np.median(mu_d))]
    exact = O.level_crossing_probability(mu_d, var_d, iso)[:, 1:-1, 1:-1]
    ss = [200, 800, 3200]
    rms = []
    for s in ss:
        errs = []
        for rep in range(4):
            est, _ = O.mc_lcp(iso, s, seed=1000 + rep, dx=1.0, dy=1.0, stats=st)
            errs.append(np.sqrt(np.mean((est[:, 1:-1, 1:-1] - exact) ** 2)))
        rms.append(np.mean(errs))
    slope = np.polyfit(np.log(ss), np.log(rms), 1)[0]
    assert -0.62 < slope < -0.38


def test_mc_streams_are_seeded_and_offset_disjoint():
    st = _small_stats(6, 7)
    a, _ = O.mc_lcp([0.0], 64, seed=5, dx=1.0, dy=1.0, stats=st)
    b, _ = O.mc_lcp([0.0], 64, seed=5, dx=1.0, dy=1.0, stats=st)
    c, _ = O.mc_lcp([0.0], 64, seed=5, dx=1.0, dy=1.0, stats=st, offset=1)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_mc_odd_sample_count_uses_first_half_of_last_pair():
    st = _small_stats(5, 6)
    _, c5 = O.mc_lcp([0.1], 5, seed=2, dx=1.0, dy=1.0, stats=st)
    _, c4 = O.mc_lcp([0.1], 4, seed=2, dx=1.0, dy=1.0, stats=st)
    _, c6 = O.mc_lcp([0.1], 6, seed=2, dx=1.0, dy=1.0, stats=st)
    assert np.all(c4 <= c5) and np.all(c5 <= c6)


# --------------------------------------------------------------------------
# Exact empirical judge (reading R12)
# --------------------------------------------------------------------------
def test_exact_empirical_below_equals_enumeration():
    rng = np.random.default_rng(12)
    m, h, w = 4, 4, 5
    u = rng.normal(size=(m, h, w)); v = rng.normal(size=(m, h, w))
    dx, dy, c = 0.8, 1.2, 0.05
    p = O.exact_empirical_below(u, v, dx, dy, c)
    for j in range(1, h - 1):
        for i in range(1, w - 1):
            n = 0
            for a in range(m):
                for b in range(m):
                    for e in range(m):
                        for f in range(m):
                            d = (u[a, j, i + 1] - u[b, j, i - 1]) / (2 * dx) + (v[e, j + 1, i] - v[f, j - 1, i]) / (2 * dy)
                            n += d < c
            assert p[j - 1, i - 1] == n / m**4


def test_empirical_mc_converges_to_exact_empirical_lcp():
    rng = np.random.default_rng(13)
    m, h, w = 6, 7, 8
    u = rng.gamma(2.0, 1.0, size=(m, h, w)) + np.linspace(0, 2, w)
    v = rng.gamma(2.0, 1.0, size=(m, h, w)) - np.linspace(0, 2, h)[:, None]
    iso = [0.0, 0.5]
    exact = O.exact_empirical_lcp(u, v, 1.0, 1.0, iso)
    s = 6000
    est, _ = O.mc_lcp(iso, s, seed=4, dx=1.0, dy=1.0, mode="empirical", members=(u, v))
    inner = est[:, 1:-1, 1:-1]  # cells whose 4 vertices are interior
    se = np.sqrt(exact * (1 - exact) / s) + 1e-12
    assert np.abs((inner - exact) / se).max() < 5.0


def test_sse_definition():
    assert O.sum_squared_error([[0.5, 0.25]], [[0.25, 0.25]]) == 0.0625


def test_stencil_neighbours_boundary_rule_by_hand():
    """Sec. 3.1 boundary rule (reading R2), written out for small axes: central
    neighbours (i-1, i+1) inside, first-order one-sided (0, 1) and (n-2, n-1) at
    the two ends, so the index distance is 2 inside and 1 at the ends."""
    lo, hi, steps = O.stencil_neighbours(2)
    assert lo.tolist() == [0, 0] and hi.tolist() == [1, 1] and steps.tolist() == [1, 1]
    lo, hi, steps = O.stencil_neighbours(5)
    assert lo.tolist() == [0, 0, 1, 2, 3]
    assert hi.tolist() == [1, 2, 3, 4, 4]
    assert steps.tolist() == [1, 2, 2, 2, 1]
    with pytest.raises(ValueError):
        O.stencil_neighbours(1)
