"""Pins of the learned surrogate's oracle (CPU only): exact rational moments,
the divergence cumulants against the exact distribution of D enumerated over
every combination of stencil members, hand-evaluated features and networks, a
finite-difference gradient check and Adam's first-step property."""

import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from oracle import surrogate as S
from paper_2510_01190_gb300 import synth


def _int_ensemble(m, h, w, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    return g.integers(-7, 8, size=(m, h, w)).astype(np.float64)


def test_moments_equal_exact_rational_arithmetic():
    x = _int_ensemble(5, 3, 4, 1)
    got = S.ensemble_moments(x)
    for j in range(3):
        for i in range(4):
            vals = [Fraction(int(a)) for a in x[:, j, i]]
            mean = sum(vals) / len(vals)
            for n, want in enumerate([mean] + [sum((a - mean) ** p for a in vals) / len(vals) for p in (2, 3, 4)]):
                assert got[n, j, i] == pytest.approx(float(want), rel=1e-13, abs=1e-13)


@pytest.mark.parametrize("h,w,dx,dy", [(4, 5, 1.0, 2.0), (2, 3, 0.5, 1.0), (3, 2, 1.0, 1.0)])
def test_divergence_cumulants_equal_enumerated_distribution(h, w, dx, dy):
    """D at a vertex takes M^4 equally likely values (one member per stencil
    vertex); its exact cumulants must equal the additive formula."""
    m = 3
    u = _int_ensemble(m, h, w, 2)
    v = _int_ensemble(m, h, w, 3)
    kap = S.divergence_cumulants(S.ensemble_moments(u), S.ensemble_moments(v), dx, dy)
    fdx, fdy = Fraction(dx), Fraction(dy)
    for j in range(h):
        for i in range(w):
            ilo, ihi = max(i - 1, 0), min(i + 1, w - 1)
            jlo, jhi = max(j - 1, 0), min(j + 1, h - 1)
            hx, hy = (ihi - ilo) * fdx, (jhi - jlo) * fdy
            ds = []
            for a, b, c, d in itertools.product(range(m), repeat=4):
                ds.append((Fraction(int(u[a, j, ihi])) - Fraction(int(u[b, j, ilo]))) / hx
                          + (Fraction(int(v[c, jhi, i])) - Fraction(int(v[d, jlo, i]))) / hy)
            n = len(ds)
            mean = sum(ds) / n
            m2, m3, m4 = (sum((x - mean) ** p for x in ds) / n for p in (2, 3, 4))
            want = [mean, m2, m3, m4 - 3 * m2 * m2]
            for q in range(4):
                assert kap[q, j, i] == pytest.approx(float(want[q]), rel=1e-12, abs=1e-12), (q, j, i)


def test_features_hand_evaluated():
    k1 = np.array([[0.1, 0.2], [0.3, 0.4]])
    k2 = np.array([[1.0, 4.0], [0.25, 0.0]])
    k3 = np.array([[0.5, -80.0], [0.0, 3.0]])
    k4 = np.array([[0.3, 16.0], [-1.0, 2.0]])
    c = 0.35
    f = S.surrogate_features(np.stack([k1, k2, k3, k4]), [c])
    assert f.shape == (1, 1, 1, 17)
    f = f[0, 0, 0]
    sig = [1.0, 2.0, 0.5, 0.0]
    mus = [0.1, 0.2, 0.3, 0.4]
    mean_sig = sum(sig) / 4
    want_z = [(c - 0.1) / 1.0, (c - 0.2) / 2.0, (c - 0.3) / 0.5, -8.0]  # sigma 0, c < mu: -8
    want_skew = [0.5, max(-5.0, -80.0 / 8.0), 0.0, 0.0]
    want_kurt = [0.3, 16.0 / 16.0, max(-2.0, -1.0 / 0.0625), 0.0]
    for vtx in range(4):
        assert f[4 * vtx + 0] == pytest.approx(want_z[vtx], abs=1e-15)
        assert f[4 * vtx + 1] == pytest.approx(sig[vtx] / mean_sig, abs=1e-15)
        assert f[4 * vtx + 2] == pytest.approx(want_skew[vtx], abs=1e-15)
        assert f[4 * vtx + 3] == pytest.approx(want_kurt[vtx], abs=1e-15)
    # feature 16: the independent-Gaussian LCP, cross-checked with the pinned closed form
    p = [0.5 * math.erfc((mu - c) / (s * math.sqrt(2.0))) if s > 0 else float(mu < c) for mu, s in zip(mus, sig)]
    want16 = 1.0 - np.prod(p) - np.prod([1 - x for x in p])
    assert f[16] == pytest.approx(want16, abs=1e-14)
    lcp = O.level_crossing_probability(np.array([[0.1, 0.2], [0.3, 0.4]]), k2, [c])
    assert f[16] == pytest.approx(lcp[0, 0, 0], abs=1e-14)


def test_features_clip_and_equal_sigma():
    kap = np.zeros((4, 2, 2))
    kap[1] = 1e-4  # all sigmas 0.01
    f = S.surrogate_features(kap, [1.0, 0.0])
    assert np.all(f[0, ..., [0, 4, 8, 12]] == 8.0)   # z = 100 clipped
    assert np.all(f[1, ..., [0, 4, 8, 12]] == 0.0)   # c at the mean
    assert np.all(f[..., [1, 5, 9, 13]] == 1.0)
    assert f[1, 0, 0, 16] == pytest.approx(1.0 - 2 * 0.5 ** 4)  # four fair coins


def _params64(seed):
    p = {k: np.asarray(v, np.float64) for k, v in synth.mlp_init_params(seed).items()}
    g = np.random.Generator(np.random.PCG64(seed + 100))
    p["b1"] = g.normal(0, 0.3, 64)
    p["b2"] = g.normal(0, 0.3, 64)
    p["b3"] = np.asarray(g.normal(0, 0.3))
    return p


def test_mlp_forward_hand_evaluated():
    zero = {k: np.zeros_like(np.asarray(v, np.float64)) for k, v in synth.mlp_init_params(0).items()}
    zero["b3"] = np.asarray(0.7)
    y, _ = S.mlp_forward(zero, np.ones((3, 17)))
    assert np.allclose(y, 1.0 / (1.0 + math.exp(-0.7)), atol=1e-15, rtol=0)
    one = {k: v.copy() for k, v in zero.items()}
    one["W1"][5, 2] = 0.8
    one["b1"][2] = -0.1
    one["W2"][2, 7] = -1.3
    one["b2"][7] = 0.2
    one["w3"][7] = 2.5
    x = np.zeros((1, 17))
    x[0, 5] = 0.6
    h1 = math.tanh(0.8 * 0.6 - 0.1)
    # units other than 2 / 7 are tanh(0) = 0 and carry no weight forward
    h2 = math.tanh(-1.3 * h1 + 0.2)
    want = 1.0 / (1.0 + math.exp(-(2.5 * h2 + 0.7)))
    y, _ = S.mlp_forward(one, x)
    assert y[0] == pytest.approx(want, abs=1e-15)
    # the prior adds to the output's pre-activation; a zero output layer returns sigmoid(prior)
    y, _ = S.mlp_forward(one, x, prior=np.array([-1.25]))
    assert y[0] == pytest.approx(1.0 / (1.0 + math.exp(-(2.5 * h2 + 0.7 - 1.25))), abs=1e-15)
    y, _ = S.mlp_forward(zero | {"b3": np.asarray(0.0)}, np.ones((1, 17)), prior=np.array([2.0]))
    assert y[0] == pytest.approx(1.0 / (1.0 + math.exp(-2.0)), abs=1e-15)


def test_prior_is_the_closed_form_logit():
    kap = np.zeros((4, 3, 3))
    kap[0] = np.arange(9).reshape(3, 3) * 0.1
    kap[1] = 0.04
    f = S.surrogate_features(kap, [0.25, 5.0])
    pr = S.surrogate_prior(f)
    g = np.clip(f[..., 16], 1e-6, 1 - 1e-6)
    assert np.allclose(1.0 / (1.0 + np.exp(-pr)), g, rtol=1e-12, atol=1e-15)
    assert np.all(pr[1] == pytest.approx(math.log(1e-6 / (1 - 1e-6))))  # c far above: LCP 0, clamped


def test_mlp_backward_matches_finite_differences():
    p = _params64(3)
    g = np.random.Generator(np.random.PCG64(7))
    x = g.normal(0, 1, (20, 17))
    t = g.uniform(0, 1, 20)
    prior = g.normal(0, 2, 20)
    y, cache = S.mlp_forward(p, x, prior)
    grads = S.mlp_backward(p, cache, t)
    eps = 1e-6
    for k in p:
        flat = np.asarray(p[k]).reshape(-1)
        gk = np.asarray(grads[k]).reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 40)):
            q = {kk: np.array(vv, copy=True) for kk, vv in p.items()}
            fq = q[k].reshape(-1)
            fq[idx] += eps
            lp = S.mse_loss(S.mlp_forward(q, x, prior)[0], t)
            fq[idx] -= 2 * eps
            lm = S.mse_loss(S.mlp_forward(q, x, prior)[0], t)
            fd = (lp - lm) / (2 * eps)
            assert gk[idx] == pytest.approx(fd, rel=1e-5, abs=1e-10), (k, idx)


def test_adam_first_steps_move_by_lr():
    """With a constant gradient the bias-corrected moments are g and g^2, so
    every step moves each weight by lr * g / (|g| + eps)."""
    p = {"a": np.array([1.0, -2.0, 3.0]), "b": np.asarray(0.5)}
    g = {"a": np.array([0.3, -4.0, 0.0]), "b": np.asarray(-1e-3)}
    st = {"t": 0, "m": {k: np.zeros_like(v) for k, v in p.items()}, "v": {k: np.zeros_like(v) for k, v in p.items()}}
    lr, eps = 0.01, 1e-8
    start = {k: np.array(v, copy=True) for k, v in p.items()}
    for step in (1, 2, 3):
        S.adam_step(p, g, st, lr, eps=eps)
        for k in p:
            want = start[k] - step * lr * g[k] / (np.abs(g[k]) + eps)
            assert np.allclose(p[k], want, rtol=0, atol=1e-13)
    assert p["a"][2] == 3.0  # zero gradient: no move
