"""Plain FP64 CPU statement of the LCP-of-divergence method (test infrastructure only).

Source: Ouermi, Li, Moreland, Pugmire, Johnson, Athawale, "Efficient
Probabilistic Visualization of Local Divergence of 2D Vector Fields with
Independent Gaussian Uncertainty", arXiv 2510.01190.  Section numbers below
are the paper's: Sec. 3 (Methods), Sec. 3.1 (Analytical Probabilistic
Divergence, Eqs. 1-3), Sec. 3.2 (Divergence Uncertainty Validation, Fig. 2),
Sec. 4 (Results: the Monte Carlo baseline, sample counts, SSE).

Only ``tests/``, ``__graft_entry__.smoke`` and ``bench.py``'s CPU-baseline leg
may import this module.  It imports nothing from the GPU library.

Conventions (shared with the GPU library by documentation, not by code)
-------------------------------------------------------------------------
* A field is sampled on an ``H x W`` uniform grid.  Vertex ``(i, j)`` has
  ``i`` = x = column and ``j`` = y = row (Sec. 3.1); arrays are indexed
  ``[..., j, i]``.  ``u`` is the x component, ``v`` the y component.
* An ensemble is an array ``[M, H, W]`` per component.
* Cell ``(i, j)`` has the vertices ``(i, j), (i+1, j), (i, j+1), (i+1, j+1)``;
  LCP maps are ``[K, H-1, W-1]`` for ``K`` isovalues.

Readings taken where the paper is silent
----------------------------------------------------------------------
R1  LCP (Sec. 3.1 cites Poethkow et al. without printing the formula): with
    independent vertex values, P(crossing) = 1 - prod_k P(D_k < c)
    - prod_k P(D_k >= c) over the 4 cell vertices.
R2  Boundary rule (Sec. 3.1, "forward and backward differences"): first-order
    one-sided differences with step dx (dy), not 2 dx.
R3  Variance estimator (Sec. 3.1 only says "estimate"): divisor M - ddof,
    ddof = 1 by default.
R7  "Below" means d < c; a cell crosses iff it has a vertex below and a vertex
    not below.  With zero variance P(D < c) is the indicator [mu < c].
R9  The Monte Carlo baseline (Sec. 3.2, Sec. 4) samples the fitted per-vertex
    Gaussians; each sample is one realisation of the whole field.
R12 Empirical (non-Gaussian) model: every vertex component is an independent
    draw from its own ensemble members, uniformly.
R19 Speed-gradient preprocessing (Sec. 4.2, Red Sea): per member the velocity
    magnitude s = sqrt(u^2 + v^2) and its "pixelwise gradient" with the stencil
    of Eq. 1 (central differences inside, first-order one-sided at the ends,
    spacing dx, dy); the gradient vectors are then the ensemble whose
    divergence LCP is mapped, every step of the closed form unchanged.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

__all__ = [
    "ensemble_stats",
    "stencil_neighbours",
    "divergence_gaussian",
    "divergence_of_field",
    "below_above_probabilities",
    "level_crossing_probability",
    "mean_field_crossing",
    "lcp_closed_form",
    "philox4x32_10",
    "uniform01",
    "box_muller",
    "mc_lcp",
    "exact_empirical_below",
    "exact_empirical_lcp",
    "sum_squared_error",
    "speed_gradient",
    "speed_gradient_lcp",
]


# --------------------------------------------------------------------------
# Sec. 3 / Sec. 3.1: per-vertex Gaussian model estimated from the ensemble
# --------------------------------------------------------------------------
def ensemble_stats(x, ddof: int = 1):
    """Per-vertex mean and variance of one vector component over the members.

    Sec. 3.1 (closing paragraph): mu-hat and sigma-hat^2 are estimated from the
    ensemble.  Reading R3: the divisor is ``M - ddof``.  Two passes in FP64.

    x : array [M, H, W] (any float dtype; upcast to float64)
    returns (mean [H, W], var [H, W]) as float64
    """
    x = np.asarray(x, dtype=np.float64)
    m = x.shape[0]
    if m - ddof < 1:
        raise ValueError("need M - ddof >= 1")
    mean = x.sum(axis=0) / m
    dev = x - mean
    var = (dev * dev).sum(axis=0) / (m - ddof)
    return mean, var


def stencil_neighbours(n: int):
    """Neighbour indices and index distance for the divergence stencil along one axis.

    Eq. 1 uses the central difference (index-1, index+1); at the two ends the
    paper replaces it by forward / backward differences (Sec. 3.1; reading R2:
    first order, so the neighbours are (0, 1) and (n-2, n-1)).

    returns (lo [n], hi [n], steps [n]) with steps = hi - lo (2 inside, 1 at the ends)
    """
    if n < 2:
        raise ValueError("an axis needs at least 2 vertices")
    idx = np.arange(n)
    lo = np.maximum(idx - 1, 0)
    hi = np.minimum(idx + 1, n - 1)
    return lo, hi, (hi - lo)


def divergence_gaussian(mu_u, var_u, mu_v, var_v, dx: float, dy: float):
    """Mean and variance of the divergence Gaussian at every vertex (Eqs. 2 and 3).

    Eq. 2: mu_ij = (mu_{i+1} - mu_{i-1}) / (2 dx) + (mu_{j+1} - mu_{j-1}) / (2 dy)
    Eq. 3: sigma^2_ij = (sigma_{i+1}/(2dx))^2 + (sigma_{i-1}/(2dx))^2
                        + (sigma_{j+1}/(2dy))^2 + (sigma_{j-1}/(2dy))^2
    with u statistics used along x and v statistics along y (Eq. 1), and the
    one-sided boundary rule of ``stencil_neighbours`` (step dx instead of 2 dx).

    All inputs [H, W]; returns (mu_d, var_d) [H, W] float64.
    """
    mu_u = np.asarray(mu_u, np.float64)
    var_u = np.asarray(var_u, np.float64)
    mu_v = np.asarray(mu_v, np.float64)
    var_v = np.asarray(var_v, np.float64)
    h, w = mu_u.shape
    ilo, ihi, isteps = stencil_neighbours(w)
    jlo, jhi, jsteps = stencil_neighbours(h)
    hx = (isteps * float(dx))[None, :]  # 2 dx inside, dx on the first/last column
    hy = (jsteps * float(dy))[:, None]
    mu_d = (mu_u[:, ihi] - mu_u[:, ilo]) / hx + (mu_v[jhi, :] - mu_v[jlo, :]) / hy
    var_d = (var_u[:, ihi] + var_u[:, ilo]) / hx**2 + (var_v[jhi, :] + var_v[jlo, :]) / hy**2
    return mu_d, var_d


def divergence_of_field(u, v, dx: float, dy: float):
    """Finite-difference divergence of one (or a stack of) realisations (Eq. 1).

    u, v : [..., H, W].  Same stencil and boundary rule as ``divergence_gaussian``.
    """
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    h, w = u.shape[-2:]
    ilo, ihi, isteps = stencil_neighbours(w)
    jlo, jhi, jsteps = stencil_neighbours(h)
    hx = isteps * float(dx)
    hy = (jsteps * float(dy))[:, None]
    return (u[..., :, ihi] - u[..., :, ilo]) / hx + (v[..., jhi, :] - v[..., jlo, :]) / hy


# --------------------------------------------------------------------------
# Sec. 3.1 (last paragraph): level-crossing probability per cell
# --------------------------------------------------------------------------
def below_above_probabilities(mu, var, c: float):
    """p = P(D < c) and q = P(D >= c) for D ~ N(mu, var), elementwise.

    Written with the complementary error function so that neither tail is
    formed as 1 - (something close to 1):
        P(D < c)  = 1/2 erfc((mu - c) / (sigma sqrt 2))
        P(D >= c) = 1/2 erfc((c - mu) / (sigma sqrt 2))
    Reading R7: with var == 0, p = [mu < c] and q = 1 - p.
    """
    mu = np.asarray(mu, np.float64)
    var = np.asarray(var, np.float64)
    c = float(c)
    sd = np.sqrt(var)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (mu - c) / (sd * math.sqrt(2.0))
        p = 0.5 * erfc(t)
        q = 0.5 * erfc(-t)
    zero = var == 0
    if np.any(zero):
        ind = (mu[zero] < c).astype(np.float64)
        p = np.where(zero, 0.0, p)
        q = np.where(zero, 0.0, q)
        p[zero] = ind
        q[zero] = 1.0 - ind
    return p, q


def level_crossing_probability(mu_d, var_d, isovalues):
    """LCP of every cell for every isovalue (Sec. 3.1, reading R1).

    LCP(cell, c) = 1 - prod_{4 vertices} P(D_k < c) - prod_{4 vertices} P(D_k >= c)

    mu_d, var_d : [H, W];  isovalues : sequence of K floats
    returns [K, H-1, W-1] float64
    """
    mu_d = np.asarray(mu_d, np.float64)
    var_d = np.asarray(var_d, np.float64)
    h, w = mu_d.shape
    iso = np.atleast_1d(np.asarray(isovalues, np.float64))
    out = np.empty((iso.size, h - 1, w - 1))
    for k, c in enumerate(iso):
        p, q = below_above_probabilities(mu_d, var_d, c)
        all_below = p[:-1, :-1] * p[:-1, 1:] * p[1:, :-1] * p[1:, 1:]
        all_above = q[:-1, :-1] * q[:-1, 1:] * q[1:, :-1] * q[1:, 1:]
        out[k] = 1.0 - all_below - all_above
    return out


def mean_field_crossing(mu_d, isovalues):
    """Mean-field isocontour crossing per cell (Fig. 1a, Fig. 3c; reading R7).

    A cell of the mean-field divergence crosses isovalue c iff its 4 vertices
    are not all on the same side, with "below" meaning mu_d < c.
    returns bool [K, H-1, W-1]
    """
    mu_d = np.asarray(mu_d, np.float64)
    iso = np.atleast_1d(np.asarray(isovalues, np.float64))
    h, w = mu_d.shape
    out = np.empty((iso.size, h - 1, w - 1), dtype=bool)
    for k, c in enumerate(iso):
        b = mu_d < c
        n_below = (b[:-1, :-1].astype(int) + b[:-1, 1:] + b[1:, :-1] + b[1:, 1:])
        out[k] = (n_below > 0) & (n_below < 4)
    return out


def lcp_closed_form(u, v, dx: float, dy: float, isovalues, ddof: int = 1):
    """The whole analytical path: ensemble -> Gaussians -> Eqs. 2/3 -> LCP.

    returns dict with mu_u, var_u, mu_v, var_v, mu_d, var_d, lcp, mask
    """
    mu_u, var_u = ensemble_stats(u, ddof)
    mu_v, var_v = ensemble_stats(v, ddof)
    mu_d, var_d = divergence_gaussian(mu_u, var_u, mu_v, var_v, dx, dy)
    return dict(
        mu_u=mu_u, var_u=var_u, mu_v=mu_v, var_v=var_v, mu_d=mu_d, var_d=var_d,
        lcp=level_crossing_probability(mu_d, var_d, isovalues),
        mask=mean_field_crossing(mu_d, isovalues),
    )


# --------------------------------------------------------------------------
# Random numbers for the Monte Carlo baseline
# --------------------------------------------------------------------------
_MASK32 = np.uint64(0xFFFFFFFF)
_PHILOX_M0 = np.uint64(0xD2511F53)  # multipliers of Philox-4x32 (Salmon et al., SC'11)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = 0x9E3779B9  # Weyl key increments (golden ratio, sqrt(3) - 1)
_PHILOX_W1 = 0xBB67AE85


def philox4x32_10(ctr, key):
    """Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11).

    One round maps counter words (x0, x1, x2, x3) and key (k0, k1) to
        (hi(M1*x2) ^ x1 ^ k0,  lo(M1*x2),  hi(M0*x0) ^ x3 ^ k1,  lo(M0*x0)),
    where hi/lo are the upper/lower 32 bits of the 64-bit product; the key is
    bumped by the Weyl constants after every round.

    ctr : uint32 array [..., 4];  key : two uint32 values
    returns uint32 array [..., 4]
    """
    c = np.asarray(ctr, dtype=np.uint64)
    x0, x1, x2, x3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = int(key[0]) & 0xFFFFFFFF
    k1 = int(key[1]) & 0xFFFFFFFF
    for _ in range(10):
        p0 = _PHILOX_M0 * x0
        p1 = _PHILOX_M1 * x2
        x0, x1, x2, x3 = (
            (p1 >> np.uint64(32)) ^ x1 ^ np.uint64(k0),
            p1 & _MASK32,
            (p0 >> np.uint64(32)) ^ x3 ^ np.uint64(k1),
            p0 & _MASK32,
        )
        k0 = (k0 + _PHILOX_W0) & 0xFFFFFFFF
        k1 = (k1 + _PHILOX_W1) & 0xFFFFFFFF
    return np.stack([x0, x1, x2, x3], axis=-1).astype(np.uint32)


def uniform01(x):
    """Map a uint32 word to a uniform value in the open interval (0, 1).

    The top 24 bits index one of 2^24 equal sub-intervals; the value is its
    midpoint, (floor(x / 2^8) + 1/2) / 2^24, exactly representable in FP32.
    """
    x = np.asarray(x, dtype=np.uint64)
    return ((x >> np.uint64(8)).astype(np.float64) + 0.5) * 2.0**-24


def box_muller(xa, xb):
    """Two independent standard normals from two uint32 words (Box & Muller, 1958).

    r = sqrt(-2 ln U1), theta = 2 pi U2;  returns (r cos theta, r sin theta).
    """
    u1 = uniform01(xa)
    u2 = uniform01(xb)
    r = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * np.pi * u2
    return r * np.cos(th), r * np.sin(th)


def _draw_words(n_vertices: int, pairs, seed: int, offset: int):
    """Philox output for every (sample pair, vertex): counter = (vertex, pair, offset lo, offset hi),
    key = (seed lo, seed hi).  returns uint32 [len(pairs), n_vertices, 4]."""
    pairs = np.asarray(pairs, dtype=np.uint64)
    n = np.arange(n_vertices, dtype=np.uint64)
    ctr = np.empty((pairs.size, n_vertices, 4), dtype=np.uint64)
    ctr[..., 0] = n[None, :]
    ctr[..., 1] = pairs[:, None]
    ctr[..., 2] = offset & 0xFFFFFFFF
    ctr[..., 3] = (offset >> 32) & 0xFFFFFFFF
    return philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))


def mc_lcp(isovalues, n_samples: int, seed: int, dx: float, dy: float, *, mode: str = "gauss",
           stats=None, members=None, offset: int = 0, pair_chunk: int = 32):
    """Classical Monte Carlo LCP estimator (Sec. 3.2 and Sec. 4; reading R9).

    For every sample s: draw one realisation (U, V) of the whole field, take its
    finite-difference divergence (Eq. 1, same boundary rule), and count the
    cells whose four divergence values straddle c (min < c <= max, reading R7).
    The estimate is count / n_samples.

    mode "gauss": U ~ N(mu_u, var_u), V ~ N(mu_v, var_v) independently per vertex;
        stats = (mu_u, var_u, mu_v, var_v), each [H, W].
    mode "empirical": U, V are members drawn uniformly and independently per
        vertex and component (reading R12); members = (u, v), each [M, H, W].

    Random numbers: Philox-4x32-10 with counter (vertex index j*W + i, sample
    pair t, offset lo, offset hi) and key (seed lo, seed hi) gives 4 words per
    vertex and pair; sample 2t uses words (0, 1), sample 2t+1 words (2, 3).
    gauss: (z_u, z_v) = Box-Muller(words); U = mu_u + sqrt(var_u) z_u (V alike).
    empirical: member index = floor(word * M / 2^32) for u and v respectively.

    returns (estimate [K, H-1, W-1] float64, counts [K, H-1, W-1] int64)
    """
    iso = np.atleast_1d(np.asarray(isovalues, np.float64))
    if mode == "gauss":
        mu_u, var_u, mu_v, var_v = (np.asarray(a, np.float64) for a in stats)
        h, w = mu_u.shape
        sd_u = np.sqrt(var_u).ravel()
        sd_v = np.sqrt(var_v).ravel()
        mu_u_f, mu_v_f = mu_u.ravel(), mu_v.ravel()
    elif mode == "empirical":
        mu_u = np.asarray(members[0], np.float64)
        mv = np.asarray(members[1], np.float64)
        m, h, w = mu_u.shape
        u_flat = mu_u.reshape(m, h * w)
        v_flat = mv.reshape(m, h * w)
        cols = np.arange(h * w)
    else:
        raise ValueError(mode)
    nv = h * w
    counts = np.zeros((iso.size, h - 1, w - 1), dtype=np.int64)
    n_pairs = (n_samples + 1) // 2
    for t0 in range(0, n_pairs, pair_chunk):
        pairs = np.arange(t0, min(n_pairs, t0 + pair_chunk))
        words = _draw_words(nv, pairs, seed, offset)  # [T, N, 4]
        for half in (0, 1):
            wa = words[..., 2 * half]
            wb = words[..., 2 * half + 1]
            if mode == "gauss":
                z_u, z_v = box_muller(wa, wb)
                uu = mu_u_f[None, :] + sd_u[None, :] * z_u
                vv = mu_v_f[None, :] + sd_v[None, :] * z_v
            else:
                iu = ((wa.astype(np.uint64) * np.uint64(m)) >> np.uint64(32)).astype(np.int64)
                iv = ((wb.astype(np.uint64) * np.uint64(m)) >> np.uint64(32)).astype(np.int64)
                uu = u_flat[iu, cols[None, :]]
                vv = v_flat[iv, cols[None, :]]
            sample_ids = 2 * pairs + half
            keep = sample_ids < n_samples
            if not np.any(keep):
                continue
            d = divergence_of_field(uu[keep].reshape(-1, h, w), vv[keep].reshape(-1, h, w), dx, dy)
            quad = np.stack([d[:, :-1, :-1], d[:, :-1, 1:], d[:, 1:, :-1], d[:, 1:, 1:]], axis=0)
            lo = quad.min(axis=0)
            hi = quad.max(axis=0)
            for k, c in enumerate(iso):
                counts[k] += ((lo < c) & (hi >= c)).sum(axis=0)
    return counts / float(n_samples), counts


# --------------------------------------------------------------------------
# Exact LCP under the independent empirical model (reading R12), interior cells
# --------------------------------------------------------------------------
def exact_empirical_below(u, v, dx: float, dy: float, c: float):
    """P(D < c) at every interior vertex when each of the four stencil values of
    Eq. 1 is an independent uniform draw from its own ensemble members.

    D = X + Y with X = (U_{i+1} - U_{i-1}) / (2 dx) taking M^2 equally likely
    values and Y = (V_{j+1} - V_{j-1}) / (2 dy) likewise.  P(X + Y < c) is the
    number of (x, y) pairs with y < c - x divided by M^4, counted by sorting the
    Y values and binary search (meet in the middle), O(M^2 log M) per vertex.

    u, v : [M, H, W];  returns [H-2, W-2] float64 for vertices 1..H-2 x 1..W-2
    """
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    m, h, w = u.shape
    out = np.empty((h - 2, w - 2))
    for j in range(1, h - 1):
        for i in range(1, w - 1):
            xs = (u[:, j, i + 1][:, None] - u[:, j, i - 1][None, :]).ravel() / (2.0 * dx)
            ys = np.sort((v[:, j + 1, i][:, None] - v[:, j - 1, i][None, :]).ravel() / (2.0 * dy))
            n_less = np.searchsorted(ys, c - xs, side="left").sum()
            out[j - 1, i - 1] = n_less / float(m) ** 4
    return out


def exact_empirical_lcp(u, v, dx: float, dy: float, isovalues):
    """Exact LCP of the cells whose four vertices are all interior, under the
    independent empirical model (reading R12).  Interior vertex stencils share
    no input value, so the four vertex divergences are independent and
    LCP = 1 - prod P(D_k < c) - prod P(D_k >= c) holds exactly.

    returns [K, H-3, W-3]: cells (i, j) with 1 <= i <= W-3, 1 <= j <= H-3
    """
    iso = np.atleast_1d(np.asarray(isovalues, np.float64))
    u = np.asarray(u, np.float64)
    _, h, w = u.shape
    out = np.empty((iso.size, h - 3, w - 3))
    for k, c in enumerate(iso):
        p = exact_empirical_below(u, v, dx, dy, c)
        q = 1.0 - p
        out[k] = (1.0 - p[:-1, :-1] * p[:-1, 1:] * p[1:, :-1] * p[1:, 1:]
                  - q[:-1, :-1] * q[:-1, 1:] * q[1:, :-1] * q[1:, 1:])
    return out


def sum_squared_error(a, b):
    """SSE between two LCP maps (Sec. 4, accuracy of MC against the analytical LCP)."""
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return float((d * d).sum())


# --------------------------------------------------------------------------
# Sec. 4.2 (Red Sea): divergence of the gradient of the velocity magnitude
# --------------------------------------------------------------------------
def speed_gradient(u, v, dx: float, dy: float):
    """Per member, the gradient of the velocity magnitude (reading R19).

    s = sqrt(u^2 + v^2);  gx = (s[i+] - s[i-]) / ((i+ - i-) dx),
    gy = (s[j+] - s[j-]) / ((j+ - j-) dy), with the neighbours of
    ``stencil_neighbours`` (central inside, one-sided at the ends).

    u, v : [..., H, W];  returns (gx, gy) float64 of the same shape
    """
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    s = np.sqrt(u * u + v * v)
    h, w = s.shape[-2:]
    ilo, ihi, isteps = stencil_neighbours(w)
    jlo, jhi, jsteps = stencil_neighbours(h)
    gx = (s[..., :, ihi] - s[..., :, ilo]) / (isteps * float(dx))
    gy = (s[..., jhi, :] - s[..., jlo, :]) / (jsteps * float(dy))[:, None]
    return gx, gy


def speed_gradient_lcp(u, v, dx: float, dy: float, isovalues, ddof: int = 1):
    """The closed-form path on the speed-gradient ensemble (Sec. 4.2, Fig. 3d):
    ``lcp_closed_form`` of the members' (gx, gy).  returns its dict."""
    gx, gy = speed_gradient(u, v, dx, dy)
    return lcp_closed_form(gx, gy, dx, dy, isovalues, ddof)
