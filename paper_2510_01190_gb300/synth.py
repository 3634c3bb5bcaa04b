"""Seeded synthetic ensembles shaped like the paper's workloads.

This module only makes inputs: base velocity fields, per-member noise and
isovalue lists.  It contains none of the method's arithmetic (no ensemble
statistics, no finite-difference divergence, no crossing probabilities); the
isovalue lists come from the *analytic* derivative of each generator's own
closed-form base field.  Both the GPU tests and the CPU oracle consume the
arrays it returns, so every generator is deterministic in its seed.

The wind (IRI/LDEO S2S, 68x68x15) and Red Sea (SciVis 2020, 500x500x20)
ensembles of the paper's Sec. 4 are not available; these generators stand in
for their shapes:

* ``point_sources_ensemble``  64x64, 20 members: Gaussian sources/sinks plus
  Rankine vortices, heteroscedastic noise sigma = 0.1 |v| + 0.01 (wind-sized).
* ``fourier_ensemble``  721x1440 (lat-lon 0.25 deg), 51 members: random
  Fourier modes with a k^-3 energy spectrum plus log-normal noise levels.
* ``eddy_ensemble_torch``  8192^2, 20 members, BF16 storage: Gaussian
  mesoscale eddies plus white noise (Red-Sea-like, larger), made on a device.
* ``non_gaussian_ensemble``  1024^2, 50 members: Fourier mean field with
  skew-normal or two-component Gaussian-mixture noise per vertex.
* ``batch_descriptors``  256 fields of uneven size for the batched launch.
* ``fourier_volume_torch``  3D volumes (256^3, 20 members by default) of random
  3D Fourier modes plus log-normal noise levels, made on a torch device.
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "point_sources_ensemble",
    "fourier_ensemble",
    "fourier_base_field",
    "eddy_ensemble_torch",
    "non_gaussian_ensemble",
    "dyadic_ensemble",
    "random_stats",
    "batch_descriptors",
    "fourier_batch_torch",
    "mlp_init_params",
    "fourier_volume_torch",
]


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


# ---------------------------------------------------------------------------
# 64 x 64: Gaussian point sources / sinks + Rankine vortices
# ---------------------------------------------------------------------------
def point_sources_ensemble(seed: int = 0, h: int = 64, w: int = 64, m: int = 20, n_sources: int = 4,
                           n_vortices: int = 2, width: float = 6.0):
    """Base field: ``n_sources`` Gaussian sources/sinks (random sign, width 6
    cells: velocity = s (r - r_c) / width * exp(-|r - r_c|^2 / (2 width^2)))
    plus ``n_vortices`` Rankine vortices (core radius U[4, 10], random turning
    sense), scaled so that the peak base speed is 1.  Every member adds i.i.d.
    Gaussian noise per vertex and component with sigma = 0.1 |v| + 0.01.

    returns dict(u, v: float32 [m, h, w]; dx, dy; isovalues: float32 [1] = 0)
    """
    g = _rng(seed, 1)
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    bu = np.zeros((h, w))
    bv = np.zeros((h, w))
    for _ in range(n_sources):
        xc, yc = g.uniform(0.15 * w, 0.85 * w), g.uniform(0.15 * h, 0.85 * h)
        s = g.choice([-1.0, 1.0])
        rx, ry = x - xc, y - yc
        e = np.exp(-(rx * rx + ry * ry) / (2 * width * width))
        bu += s * rx / width * e
        bv += s * ry / width * e
    for _ in range(n_vortices):
        xc, yc = g.uniform(0.15 * w, 0.85 * w), g.uniform(0.15 * h, 0.85 * h)
        core = g.uniform(4.0, 10.0)
        s = g.choice([-1.0, 1.0])
        rx, ry = x - xc, y - yc
        r = np.sqrt(rx * rx + ry * ry)
        vt = np.where(r < core, r / core, core / np.maximum(r, 1e-12))
        inv_r = np.where(r > 0, 1.0 / np.maximum(r, 1e-12), 0.0)
        bu += s * vt * (-ry) * inv_r
        bv += s * vt * rx * inv_r
    speed = np.sqrt(bu * bu + bv * bv)
    scale = 1.0 / speed.max()
    bu *= scale
    bv *= scale
    sigma = 0.1 * speed * scale + 0.01
    u = bu[None] + sigma[None] * g.standard_normal((m, h, w))
    v = bv[None] + sigma[None] * g.standard_normal((m, h, w))
    return dict(u=u.astype(np.float32), v=v.astype(np.float32), dx=1.0, dy=1.0,
                isovalues=np.array([0.0], np.float32))


# ---------------------------------------------------------------------------
# 721 x 1440: random Fourier modes with a k^-3 energy spectrum
# ---------------------------------------------------------------------------
def _fourier_component(g, h, w, n_modes, kmax):
    """Coefficients of ``n_modes`` random integer wavevectors with |k| <= kmax,
    amplitude |k|^-3/2 and random phase, on the periodic h x w domain."""
    kk = [(kx, ky) for kx in range(-kmax, kmax + 1) for ky in range(-kmax, kmax + 1)
          if 0 < kx * kx + ky * ky <= kmax * kmax]
    pick = g.choice(len(kk), size=n_modes, replace=False)
    coef = np.zeros((h, w), np.complex128)
    dcoef_dx = np.zeros((h, w), np.complex128)
    dcoef_dy = np.zeros((h, w), np.complex128)
    for p in pick:
        kx, ky = kk[p]
        a = (kx * kx + ky * ky) ** -0.75 * np.exp(1j * g.uniform(0, 2 * np.pi))
        coef[ky % h, kx % w] += a
        dcoef_dx[ky % h, kx % w] += a * 1j * 2 * np.pi * kx / w
        dcoef_dy[ky % h, kx % w] += a * 1j * 2 * np.pi * ky / h
    field = np.real(np.fft.ifft2(coef)) * h * w
    ddx = np.real(np.fft.ifft2(dcoef_dx)) * h * w
    ddy = np.real(np.fft.ifft2(dcoef_dy)) * h * w
    return field, ddx, ddy


def fourier_base_field(seed: int, h: int, w: int, n_modes: int = 200, kmax: int = 30, rms: float = 10.0):
    """Mean field of the lat-lon-shaped generator and its analytic divergence
    (derivative of the Fourier series itself, with unit grid spacing).

    returns (u [h,w], v [h,w], analytic_divergence [h,w]) float64
    """
    g = _rng(seed, 2)
    u, dudx, _ = _fourier_component(g, h, w, n_modes, kmax)
    v, _, dvdy = _fourier_component(g, h, w, n_modes, kmax)
    su = rms / np.sqrt(np.mean(u * u))
    sv = rms / np.sqrt(np.mean(v * v))
    return u * su, v * sv, dudx * su + dvdy * sv


def fourier_ensemble(seed: int = 0, h: int = 721, w: int = 1440, m: int = 51, k: int = 8,
                     n_modes: int = 200, kmax: int = 30, noise_median: float = 0.5,
                     noise_shape: float = 0.5, dtype=np.float32):
    """Lat-lon-shaped ensemble: u, v each from 200 random Fourier modes
    (integer wavenumber <= 30, energy ~ k^-3, RMS 10 m/s) plus heteroscedastic
    Gaussian noise whose per-vertex, per-component sigma is log-normal with
    median 0.5 m/s and shape 0.5.  ``k`` isovalues sit at evenly spaced
    percentiles from the 5th to the 95th of the analytic mean divergence.

    returns dict(u, v [m, h, w] of ``dtype``; dx = dy = 1; isovalues float32 [k])
    """
    bu, bv, div = fourier_base_field(seed, h, w, n_modes, kmax)
    g = _rng(seed, 3)
    su = noise_median * np.exp(noise_shape * g.standard_normal((h, w)))
    sv = noise_median * np.exp(noise_shape * g.standard_normal((h, w)))
    u = np.empty((m, h, w), dtype)
    v = np.empty((m, h, w), dtype)
    for i in range(m):  # member by member keeps the float64 temporaries small
        u[i] = bu + su * g.standard_normal((h, w))
        v[i] = bv + sv * g.standard_normal((h, w))
    iso = np.percentile(div, np.linspace(5, 95, k)).astype(np.float32) if k > 1 else \
        np.array([np.median(div)], np.float32)
    return dict(u=u, v=v, dx=1.0, dy=1.0, isovalues=iso)


# ---------------------------------------------------------------------------
# 8192^2 BF16: Gaussian mesoscale eddies (made on a torch device)
# ---------------------------------------------------------------------------
def eddy_ensemble_torch(seed: int = 0, h: int = 8192, w: int = 8192, m: int = 20, n_eddies: int = 5000,
                        rmin: float = 10.0, rmax: float = 60.0, noise: float = 0.05, offset: float = 0.0,
                        device="cuda", dtype=None, k: int = 4):
    """Red-Sea-like eddy field: ``n_eddies`` Gaussian vortices (stream function
    A exp(-r^2 / (2 R^2)), radius R in U[10, 60] cells, peak speed U[0.1, 1]
    with random sense) plus white Gaussian noise of sigma ``noise`` per member,
    vertex and component; ``offset`` is added to both components (it exercises
    the large |mean| / sigma regime).  Made on ``device`` with a seeded torch
    generator; stored in ``dtype`` (default bfloat16).

    Eddies are divergence-free, so the mean divergence is the ensemble-mean
    noise; the ``k`` isovalues sit at the 5/35/65/95th percentiles of that
    noise's law, N(0, noise^2 / m).
    returns dict(u, v [m, h, w] torch tensors on ``device``; dx, dy; isovalues np.float32 [k])
    """
    import torch

    if dtype is None:
        dtype = torch.bfloat16
    g = _rng(seed, 4)
    bu = torch.zeros((h, w), dtype=torch.float32, device=device)
    bv = torch.zeros((h, w), dtype=torch.float32, device=device)
    xs = g.uniform(0, w, n_eddies)
    ys = g.uniform(0, h, n_eddies)
    rs = g.uniform(rmin, rmax, n_eddies)
    amp = g.uniform(0.1, 1.0, n_eddies) * g.choice([-1.0, 1.0], n_eddies)
    for xc, yc, r, a in zip(xs, ys, rs, amp):
        half = int(math.ceil(4 * r))
        i0, i1 = max(0, int(xc) - half), min(w, int(xc) + half + 1)
        j0, j1 = max(0, int(yc) - half), min(h, int(yc) + half + 1)
        if i0 >= i1 or j0 >= j1:
            continue
        yy = torch.arange(j0, j1, device=device, dtype=torch.float32)[:, None] - yc
        xx = torch.arange(i0, i1, device=device, dtype=torch.float32)[None, :] - xc
        e = torch.exp(-(xx * xx + yy * yy) / (2 * r * r))
        # peak speed of a Gaussian vortex is |A| / (R sqrt(e)) at r = R
        s = a * math.sqrt(math.e) / r
        bu[j0:j1, i0:i1] += -s * yy * e
        bv[j0:j1, i0:i1] += s * xx * e
    tg = torch.Generator(device=device)
    tg.manual_seed(int(seed) * 1000003 + 17)
    u = torch.empty((m, h, w), dtype=dtype, device=device)
    v = torch.empty((m, h, w), dtype=dtype, device=device)
    for i in range(m):
        u[i] = (bu + offset + noise * torch.randn((h, w), generator=tg, device=device)).to(dtype)
        v[i] = (bv + offset + noise * torch.randn((h, w), generator=tg, device=device)).to(dtype)
    from statistics import NormalDist

    sd = noise / math.sqrt(m)
    iso = np.array([NormalDist(0.0, sd).inv_cdf(p) for p in (0.05, 0.35, 0.65, 0.95)][:k], np.float32)
    return dict(u=u, v=v, dx=1.0, dy=1.0, isovalues=iso)


# Isovalues for the divergence of the speed gradient of an eddy ensemble
# (Sec. 4.2 maps sources at 0.003 on the Red Sea).  With noise 0.05 per member
# the mean-field value is noise-dominated at about 0.01, so the table brackets
# it: a sink level, zero, the paper's source level, a source level.
EDDY_GRADIENT_ISOVALUES = np.array([-0.01, 0.0, 0.003, 0.01], np.float32)


# ---------------------------------------------------------------------------
# 1024^2 non-Gaussian: skew-normal or 2-component Gaussian-mixture noise
# ---------------------------------------------------------------------------
def non_gaussian_ensemble(seed: int = 0, h: int = 1024, w: int = 1024, m: int = 50, k: int = 8,
                          noise_median: float = 0.5, noise_shape: float = 0.5):
    """Fourier mean field (as ``fourier_ensemble``) with per-vertex noise that is
    skew-normal (shape alpha ~ U[-5, 5]) at half of the vertex-components and a
    two-component Gaussian mixture (weight U[0.2, 0.8], means +-1.5 sigma) at the
    others; noise is standardised to the vertex's log-normal sigma.

    returns dict(u, v float32 [m, h, w]; dx = dy = 1; isovalues float32 [k])
    """
    bu, bv, div = fourier_base_field(seed, h, w)
    g = _rng(seed, 5)

    def noise(shape_hw):
        sig = noise_median * np.exp(noise_shape * g.standard_normal(shape_hw))
        kind = g.random(shape_hw) < 0.5
        alpha = g.uniform(-5, 5, shape_hw)
        delta = alpha / np.sqrt(1 + alpha * alpha)
        sn_mean = delta * np.sqrt(2 / np.pi)
        sn_sd = np.sqrt(1 - 2 * delta * delta / np.pi)
        wgt = g.uniform(0.2, 0.8, shape_hw)
        out = np.empty((m,) + shape_hw, np.float32)
        for i in range(m):
            z0 = g.standard_normal(shape_hw)
            z1 = g.standard_normal(shape_hw)
            sn = delta * np.abs(z0) + np.sqrt(1 - delta * delta) * z1  # skew-normal(alpha)
            sn = (sn - sn_mean) / sn_sd
            comp = g.random(shape_hw) < wgt
            gm_mu = np.where(comp, -1.5, 1.5)
            gm = (z1 * 0.5 + gm_mu)
            gm_mean = wgt * -1.5 + (1 - wgt) * 1.5
            gm_sd = np.sqrt(0.25 + wgt * (1 - wgt) * 9.0)
            gm = (gm - gm_mean) / gm_sd
            out[i] = (sig * np.where(kind, sn, gm)).astype(np.float32)
        return out

    u = (bu[None] + noise((h, w))).astype(np.float32)
    v = (bv[None] + noise((h, w))).astype(np.float32)
    iso = np.percentile(div, np.linspace(5, 95, k)).astype(np.float32)
    return dict(u=u, v=v, dx=1.0, dy=1.0, isovalues=iso)


# ---------------------------------------------------------------------------
# Small structured inputs for exactness tests
# ---------------------------------------------------------------------------
def dyadic_ensemble(seed: int, h: int, w: int, m: int, k: int = 3, identical_members: bool = True):
    """Values on the dyadic grid 2^-10 * integer with |x| < 2^10, so that sums,
    differences and halvings are exact in FP32.  With identical members every
    variance is exactly zero; isovalues are dyadic too.
    returns dict(u, v float32 [m, h, w]; isovalues float32 [k])
    """
    g = _rng(seed, 6)
    base_u = g.integers(-4096, 4096, size=(h, w)) / 1024.0
    base_v = g.integers(-4096, 4096, size=(h, w)) / 1024.0
    if identical_members:
        u = np.broadcast_to(base_u, (m, h, w)).copy()
        v = np.broadcast_to(base_v, (m, h, w)).copy()
    else:
        u = base_u[None] + g.integers(-64, 64, size=(m, h, w)) / 1024.0
        v = base_v[None] + g.integers(-64, 64, size=(m, h, w)) / 1024.0
    iso = (g.integers(-512, 512, size=k) / 1024.0).astype(np.float32)
    return dict(u=u.astype(np.float32), v=v.astype(np.float32), isovalues=iso)


def random_stats(seed: int, h: int, w: int, mean_scale: float = 1.0, sd_scale: float = 0.5,
                 zero_fraction: float = 0.0):
    """Per-vertex Gaussian parameters (mu_u, var_u, mu_v, var_v) as float32
    [h, w] arrays; a ``zero_fraction`` of the variances is exactly 0."""
    g = _rng(seed, 7)
    mu_u = (mean_scale * g.standard_normal((h, w))).astype(np.float32)
    mu_v = (mean_scale * g.standard_normal((h, w))).astype(np.float32)
    var_u = ((sd_scale * np.exp(0.5 * g.standard_normal((h, w)))) ** 2).astype(np.float32)
    var_v = ((sd_scale * np.exp(0.5 * g.standard_normal((h, w)))) ** 2).astype(np.float32)
    if zero_fraction > 0:
        var_u[g.random((h, w)) < zero_fraction] = 0
        var_v[g.random((h, w)) < zero_fraction] = 0
    return mu_u, var_u, mu_v, var_v


# ---------------------------------------------------------------------------
# 256 fields of uneven size for the batched launch
# ---------------------------------------------------------------------------
def batch_descriptors(seed: int = 0, n_fields: int = 256, hw_min: int = 128, hw_max: int = 2048,
                      m_min: int = 10, m_max: int = 100):
    """Sizes of the batched workload: H and W log-uniform in [128, 2048],
    M uniform in {10..100}.  returns list of dict(h, w, m, seed)."""
    g = _rng(seed, 8)
    lo, hi = math.log(hw_min), math.log(hw_max)
    out = []
    for f in range(n_fields):
        h = int(round(math.exp(g.uniform(lo, hi))))
        w = int(round(math.exp(g.uniform(lo, hi))))
        m = int(g.integers(m_min, m_max + 1))
        out.append(dict(h=h, w=w, m=m, seed=int(seed) * 100003 + f))
    return out


def _fourier_component_torch(g, h, w, n_modes, kmax, device):
    """``_fourier_component`` with the inverse FFTs on a torch device: the same
    random wavevectors, amplitudes and phases drawn from ``g``."""
    import torch

    kk = [(kx, ky) for kx in range(-kmax, kmax + 1) for ky in range(-kmax, kmax + 1)
          if 0 < kx * kx + ky * ky <= kmax * kmax]
    pick = g.choice(len(kk), size=n_modes, replace=False)
    coef = np.zeros((3, h, w), np.complex128)  # field, d/dx, d/dy (only n_modes nonzero entries)
    for p in pick:
        kx, ky = kk[p]
        a = (kx * kx + ky * ky) ** -0.75 * np.exp(1j * g.uniform(0, 2 * np.pi))
        coef[0, ky % h, kx % w] += a
        coef[1, ky % h, kx % w] += a * 1j * 2 * np.pi * kx / w
        coef[2, ky % h, kx % w] += a * 1j * 2 * np.pi * ky / h
    out = torch.fft.ifft2(torch.from_numpy(coef).to(device)).real * (h * w)
    return out[0], out[1], out[2]


def fourier_batch_torch(descs, k: int = 16, device="cuda", dtype=None, n_modes: int = 200, kmax: int = 30,
                        rms: float = 10.0, noise_median: float = 0.5, noise_shape: float = 0.5):
    """Fields of the batched workload, made on ``device``: for every descriptor
    of ``batch_descriptors`` (h, w, m, seed) the lat-lon generator's recipe --
    200 random Fourier modes per component (|k| <= 30, energy ~ k^-3, RMS 10),
    log-normal per-vertex noise levels (median 0.5, shape 0.5), Gaussian member
    noise -- and ``k`` isovalues at the 5th..95th percentiles of the field's
    analytic mean divergence.

    returns list of dict(u, v [m, h, w] torch tensors of ``dtype`` (default
    float32); dx = dy = 1; isovalues float32 [k])
    """
    import torch

    if dtype is None:
        dtype = torch.float32
    fields = []
    for d in descs:
        h, w, m, seed = d["h"], d["w"], d["m"], d["seed"]
        g = _rng(seed, 2)
        u0, dudx, _ = _fourier_component_torch(g, h, w, n_modes, kmax, device)
        v0, _, dvdy = _fourier_component_torch(g, h, w, n_modes, kmax, device)
        su = rms / torch.sqrt(torch.mean(u0 * u0))
        sv = rms / torch.sqrt(torch.mean(v0 * v0))
        bu, bv = (u0 * su).float(), (v0 * sv).float()
        div = (dudx * su + dvdy * sv).cpu().numpy()
        tg = torch.Generator(device=device)
        tg.manual_seed(int(seed) * 1000003 + 3)
        nu = noise_median * torch.exp(noise_shape * torch.randn((h, w), generator=tg, device=device))
        nv = noise_median * torch.exp(noise_shape * torch.randn((h, w), generator=tg, device=device))
        u = (bu + nu * torch.randn((m, h, w), generator=tg, device=device)).to(dtype)
        v = (bv + nv * torch.randn((m, h, w), generator=tg, device=device)).to(dtype)
        iso = np.percentile(div, np.linspace(5, 95, k)).astype(np.float32) if k > 1 else \
            np.array([np.median(div)], np.float32)
        fields.append(dict(u=u, v=v, dx=1.0, dy=1.0, isovalues=iso))
    return fields


def mlp_init_params(seed: int = 0, n_in: int = 17, hidden: int = 64, zero_output: bool = False):
    """Initial weights of the 17 -> 64 -> 64 -> 1 surrogate network: Glorot-
    uniform matrices (bound sqrt(6 / (fan_in + fan_out))), zero biases;
    ``zero_output`` sets the output weights to 0 as well (a network that starts
    as its prior).  Layout as the network is written, x @ W: W1 [17, 64],
    W2 [64, 64], w3 [64].

    returns dict of float32 arrays (b3 a 0-d array)
    """
    g = _rng(seed, 9)

    def glorot(a, b, shape):
        lim = math.sqrt(6.0 / (a + b))
        return g.uniform(-lim, lim, shape).astype(np.float32)

    p = dict(W1=glorot(n_in, hidden, (n_in, hidden)), b1=np.zeros(hidden, np.float32),
             W2=glorot(hidden, hidden, (hidden, hidden)), b2=np.zeros(hidden, np.float32),
             w3=glorot(hidden, 1, (hidden,)), b3=np.zeros((), np.float32))
    if zero_output:
        p["w3"][:] = 0.0
    return p


# ---------------------------------------------------------------------------
# 3D volumes: random Fourier modes (made on a torch device)
# ---------------------------------------------------------------------------
def fourier_volume_torch(seed: int = 0, d: int = 256, h: int = 256, w: int = 256, m: int = 20, k: int = 4,
                         n_modes: int = 64, kmax: int = 12, rms: float = 1.0, noise_median: float = 0.1,
                         noise_shape: float = 0.5, device="cuda", dtype=None):
    """3D ensemble: each of u, v, w a sum of ``n_modes`` modes
    a cos(2 pi (kx x / W + ky y / H + kz z / D) + phi) with random integer
    wavevectors 0 < |k| <= kmax and amplitude |k|^(-11/6) (energy ~ k^(-5/3)
    in 3D), scaled to RMS ``rms``; every member adds Gaussian noise whose
    per-vertex, per-component sigma is log-normal (median ``noise_median``).
    ``k`` isovalues sit at evenly spaced percentiles from the 5th to the 95th of
    the analytic divergence of the base field (the derivative of the series
    itself, unit spacing), taken on a strided subsample.

    returns dict(u, v, w [m, d, h, w] torch tensors; dx = dy = dz = 1; isovalues np.float32 [k])
    """
    import torch

    if dtype is None:
        dtype = torch.float32
    g = _rng(seed, 7)
    z = torch.arange(d, device=device, dtype=torch.float32)[:, None, None] / d
    y = torch.arange(h, device=device, dtype=torch.float32)[None, :, None] / h
    x = torch.arange(w, device=device, dtype=torch.float32)[None, None, :] / w
    vecs = [(a, b, c) for a in range(-kmax, kmax + 1) for b in range(-kmax, kmax + 1) for c in range(-kmax, kmax + 1)
            if 0 < a * a + b * b + c * c <= kmax * kmax]
    base, div = [], torch.zeros((d, h, w), device=device, dtype=torch.float32)
    for comp in range(3):
        f = torch.zeros((d, h, w), device=device, dtype=torch.float32)
        df = torch.zeros((d, h, w), device=device, dtype=torch.float32)
        for q in g.choice(len(vecs), size=n_modes, replace=False):
            kx, ky, kz = vecs[q]
            amp = (kx * kx + ky * ky + kz * kz) ** (-11.0 / 12.0)
            phase = g.uniform(0.0, 2.0 * math.pi)
            theta = 2.0 * math.pi * (kx * x + ky * y + kz * z) + phase
            f += amp * torch.cos(theta)
            # derivative along this component's own axis (x for u, y for v, z for w), per grid step
            kk, n = ((kx, w), (ky, h), (kz, d))[comp]
            df += -amp * (2.0 * math.pi * kk / n) * torch.sin(theta)
        scale = rms / float(torch.sqrt(torch.mean(f * f)))
        base.append(f * scale)
        div += df * scale
    tg = torch.Generator(device=device)
    tg.manual_seed(int(seed) * 7919 + 3)
    comps = []
    for comp in range(3):
        sig = noise_median * torch.exp(noise_shape * torch.randn((d, h, w), generator=tg, device=device))
        out = torch.empty((m, d, h, w), dtype=dtype, device=device)
        for i in range(m):
            out[i] = (base[comp] + sig * torch.randn((d, h, w), generator=tg, device=device)).to(dtype)
        comps.append(out)
    sample = div.reshape(-1)[:: max(1, div.numel() // 1000003)].double().cpu().numpy()
    iso = np.percentile(sample, np.linspace(5, 95, k)).astype(np.float32) if k > 1 else \
        np.array([np.median(sample)], np.float32)
    return dict(u=comps[0], v=comps[1], w=comps[2], dx=1.0, dy=1.0, dz=1.0, isovalues=iso)
