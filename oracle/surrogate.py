"""Plain FP64 CPU statement of the learned surrogate (test infrastructure only).

The paper (arXiv 2510.01190) treats the independent-Gaussian closed form and
Monte Carlo; it mentions neural-network surrogates only among related work
(Sec. 2).  The learned surrogate below is this library's addition for
ensembles that are not Gaussian.  What it computes is fixed here, in plain
numpy, so that the GPU kernels can be checked against it:

* the plug-in (divisor M) central moments of every vertex component;
* the cumulants of each vertex divergence D under the independent empirical
  model (reading R12): D is the Eq. 1 stencil sum of independent vertex values,
  so its n-th cumulant is the sum of the n-th cumulants of the terms, each
  scaled by the stencil weight to the n-th power (one-sided weights at the
  grid's edges, reading R2);
* 17 features per cell and isovalue (reading R14);
* a 17 -> 64 -> 64 -> 1 network (tanh hidden units, sigmoid output, reading
  R15), its mean-squared-error gradient by the chain rule, and the Adam update
  (Kingma and Ba, ICLR 2015, Algorithm 1).

Only ``tests/``, ``__graft_entry__.smoke`` and ``bench.py``'s CPU-baseline leg
may import this module.  It imports nothing from the GPU library.

Readings
------------------------------
R14 Features of cell (i, j), isovalue c, vertices in the order (i, j),
    (i+1, j), (i, j+1), (i+1, j+1), each with divergence cumulants k1..k4,
    sigma = sqrt(k2):
      4v+0  z     = (c - k1) / sigma, clipped to [-8, 8] (sigma = 0: -8, 0, 8
                    by the sign of c - k1)
      4v+1  s     = sigma / mean of the cell's four sigmas (1 when all are 0)
      4v+2  skew  = k3 / sigma^3, clipped to [-5, 5] (0 when sigma = 0)
      4v+3  exkurt= k4 / sigma^4, clipped to [-2, 10] (0 when sigma = 0)
      16    the independent-Gaussian closed-form LCP of the cell at c with
            means k1 and variances k2 (the fallback's own value)
    The isovalue enters through z (mean measured from c in units of sigma) and
    through feature 16; the raw c is not an input, because shifting the field
    and c together leaves the crossing probability unchanged.
R15 Network: h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2),
    y = sigmoid(h2 . w3 + b3 + prior), with prior = logit of feature 16 (the
    Gaussian closed form) clamped to [1e-6, 1 - 1e-6]: the network learns the
    non-Gaussian correction in logit space, and an untrained output layer
    (w3 = 0, b3 = 0) reproduces the closed form.  loss = mean over rows of
    (y - t)^2.
"""

from __future__ import annotations

import numpy as np
from scipy.special import erfc

__all__ = [
    "N_FEATURES",
    "HIDDEN",
    "ensemble_moments",
    "divergence_cumulants",
    "surrogate_features",
    "surrogate_prior",
    "mlp_forward",
    "mlp_backward",
    "mse_loss",
    "adam_step",
]

N_FEATURES = 17
HIDDEN = 64


# --------------------------------------------------------------------------
# Moments and divergence cumulants (empirical model, reading R12)
# --------------------------------------------------------------------------
def ensemble_moments(x):
    """Plug-in central moments of one component over the members, two passes.

    x : [M, H, W];  returns [4, H, W] float64: mean, m2, m3, m4 (divisor M)
    """
    x = np.asarray(x, np.float64)
    mean = x.mean(axis=0)
    d = x - mean
    return np.stack([mean, (d ** 2).mean(axis=0), (d ** 3).mean(axis=0), (d ** 4).mean(axis=0)])


def _cumulants(mom):
    """Cumulants k1..k4 of a variable from its mean and central moments."""
    mean, m2, m3, m4 = mom
    return np.stack([mean, m2, m3, m4 - 3.0 * m2 * m2])


def divergence_cumulants(mom_u, mom_v, dx: float, dy: float):
    """Cumulants of the vertex divergence D (Eq. 1, boundary rule R2) when the
    stencil's vertex values are independent with the given moments.

    D = (U_hi - U_lo) / hx + (V_hi - V_lo) / hy, with (lo, hi) = (i-1, i+1) and
    hx = 2 dx inside, (0, 1) or (W-2, W-1) and hx = dx at the ends (likewise
    along y).  Cumulants of independent terms add; a term a X has cumulants
    a^n k_n(X).

    mom_u, mom_v : [4, H, W] from ensemble_moments;  returns [4, H, W]
    """
    ku, kv = _cumulants(np.asarray(mom_u, np.float64)), _cumulants(np.asarray(mom_v, np.float64))
    _, h, w = ku.shape
    idx = np.arange(w)
    ilo, ihi = np.maximum(idx - 1, 0), np.minimum(idx + 1, w - 1)
    jdx = np.arange(h)
    jlo, jhi = np.maximum(jdx - 1, 0), np.minimum(jdx + 1, h - 1)
    ax = 1.0 / ((ihi - ilo) * float(dx))[None, :]
    ay = 1.0 / ((jhi - jlo) * float(dy))[:, None]
    out = np.empty_like(ku)
    for n in range(4):
        p = n + 1
        out[n] = (ax ** p) * ku[n][:, ihi] + ((-ax) ** p) * ku[n][:, ilo] \
            + (ay ** p) * kv[n][jhi, :] + ((-ay) ** p) * kv[n][jlo, :]
    return out


def _gauss_lcp(mu4, var4, c):
    """Independent-Gaussian LCP of cells from their four vertex means/variances."""
    p = np.empty_like(mu4)
    sd = np.sqrt(var4)
    pos = sd > 0
    p[pos] = 0.5 * erfc((mu4[pos] - c) / (sd[pos] * np.sqrt(2.0)))
    p[~pos] = (mu4[~pos] < c).astype(np.float64)
    q = 1.0 - p
    return 1.0 - p.prod(axis=0) - q.prod(axis=0)


def surrogate_features(kappa, isovalues):
    """Features of every cell and isovalue (reading R14).

    kappa : [4, H, W] from divergence_cumulants
    returns [K, H-1, W-1, 17] float64
    """
    kappa = np.asarray(kappa, np.float64)
    iso = np.atleast_1d(np.asarray(isovalues, np.float64))
    k1, k2, k3, k4 = kappa
    sig = np.sqrt(np.maximum(k2, 0.0))
    corners = [(slice(None, -1), slice(None, -1)), (slice(None, -1), slice(1, None)),
               (slice(1, None), slice(None, -1)), (slice(1, None), slice(1, None))]
    mu4 = np.stack([k1[c] for c in corners])
    sd4 = np.stack([sig[c] for c in corners])
    k3_4 = np.stack([k3[c] for c in corners])
    k4_4 = np.stack([k4[c] for c in corners])
    mean_sd = sd4.mean(axis=0)
    ratio = np.where(mean_sd > 0, sd4 / np.where(mean_sd > 0, mean_sd, 1.0), 1.0)
    pos = sd4 > 0
    safe = np.where(pos, sd4, 1.0)
    skew = np.where(pos, np.clip(k3_4 / safe ** 3, -5.0, 5.0), 0.0)
    kurt = np.where(pos, np.clip(k4_4 / safe ** 4, -2.0, 10.0), 0.0)
    hc, wc = k1.shape[0] - 1, k1.shape[1] - 1
    out = np.empty((iso.size, hc, wc, N_FEATURES))
    for kk, c in enumerate(iso):
        diff = c - mu4
        z = np.where(pos, np.clip(diff / safe, -8.0, 8.0), 8.0 * np.sign(diff))
        for v in range(4):
            out[kk, :, :, 4 * v + 0] = z[v]
            out[kk, :, :, 4 * v + 1] = ratio[v]
            out[kk, :, :, 4 * v + 2] = skew[v]
            out[kk, :, :, 4 * v + 3] = kurt[v]
        out[kk, :, :, 16] = _gauss_lcp(mu4, sd4 ** 2, c)
    return out


def surrogate_prior(features):
    """The network's prior of every row (reading R15): logit of feature 16,
    clamped to [1e-6, 1 - 1e-6].  features [..., 17];  returns [...]"""
    g = np.clip(np.asarray(features, np.float64)[..., 16], 1e-6, 1.0 - 1e-6)
    return np.log(g) - np.log1p(-g)


# --------------------------------------------------------------------------
# The network (reading R15) and its training arithmetic
# --------------------------------------------------------------------------
def _sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def mlp_forward(params, x, prior=None):
    """y = sigmoid(tanh(tanh(x W1 + b1) W2 + b2) . w3 + b3 + prior).

    params : dict W1 [17, 64], b1 [64], W2 [64, 64], b2 [64], w3 [64], b3 scalar
    x      : [N, 17];  prior : [N] or None (zero)
    returns (y [N], cache)
    """
    x = np.asarray(x, np.float64)
    h1 = np.tanh(x @ params["W1"] + params["b1"])
    h2 = np.tanh(h1 @ params["W2"] + params["b2"])
    z3 = h2 @ params["w3"] + params["b3"]
    if prior is not None:
        z3 = z3 + np.asarray(prior, np.float64)
    y = _sigmoid(z3)
    return y, dict(x=x, h1=h1, h2=h2, y=y)


def mse_loss(y, t):
    d = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    return float((d * d).mean())


def mlp_backward(params, cache, t):
    """Gradient of mse_loss(mlp_forward(params, x), t) by the chain rule.

    returns dict with the shapes of ``params``
    """
    x, h1, h2, y = cache["x"], cache["h1"], cache["h2"], cache["y"]
    n = x.shape[0]
    dz3 = 2.0 * (y - np.asarray(t, np.float64)) / n * y * (1.0 - y)  # dL/dz3, sigmoid' = y (1 - y)
    dh2 = dz3[:, None] * params["w3"][None, :]
    dz2 = dh2 * (1.0 - h2 * h2)  # tanh' = 1 - tanh^2
    dh1 = dz2 @ params["W2"].T
    dz1 = dh1 * (1.0 - h1 * h1)
    return dict(W1=x.T @ dz1, b1=dz1.sum(axis=0), W2=h1.T @ dz2, b2=dz2.sum(axis=0), w3=h2.T @ dz3,
                b3=np.asarray(dz3.sum()))


def adam_step(params, grads, state, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1): m, v moving averages of the
    gradient and its square, bias-corrected by 1 - beta^t.  ``state`` holds
    m, v (dicts like params) and the step count t; params and state change in
    place."""
    state["t"] += 1
    t = state["t"]
    for k in params:
        g = np.asarray(grads[k], np.float64)
        state["m"][k] = beta1 * state["m"][k] + (1.0 - beta1) * g
        state["v"][k] = beta2 * state["v"][k] + (1.0 - beta2) * g * g
        mhat = state["m"][k] / (1.0 - beta1 ** t)
        vhat = state["v"][k] / (1.0 - beta2 ** t)
        params[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return params
