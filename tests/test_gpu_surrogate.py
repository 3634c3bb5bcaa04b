"""Learned surrogate on the GPU against its FP64 oracle: moments, features, the
network's forward pass, its gradient, Adam, and the fused inference kernel.

Tolerances (BF16 operands, FP32 accumulation): the oracle evaluates the
network with the same bf16-rounded weights and feature rows, so the remaining
differences are the GPU's bf16 rounding of the hidden activations (relative
2^-9) and the hardware tanh (relative ~2^-11); propagated through the 64-wide
layers they stay below 1e-2 on the output; each gradient entry is compared
with its own bound (test_backward_parity)."""

import numpy as np
import pytest
import torch

import oracle as O
from oracle import surrogate as S
from paper_2510_01190_gb300 import surrogate as G
from paper_2510_01190_gb300 import synth

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def _bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _ng(h, w, m, seed, k=4):
    return synth.non_gaussian_ensemble(seed, h=h, w=w, m=m, k=k)


def _params(seed):
    p = synth.mlp_init_params(seed)
    g = np.random.Generator(np.random.PCG64(seed + 50))
    p["b1"] = g.normal(0, 0.2, 64).astype(np.float32)
    p["b2"] = g.normal(0, 0.2, 64).astype(np.float32)
    p["b3"] = np.asarray(g.normal(0, 0.2), np.float32)
    return p


def _oracle_params_bf16(p):
    """The oracle's copy of the weights the GPU uses: matrices rounded to bf16."""
    q = {k: np.asarray(v, np.float64) for k, v in p.items()}
    q["W1"] = _bf16(q["W1"])
    q["W2"] = _bf16(q["W2"])
    return q


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("h,w,m", [(37, 53, 12), (16, 64, 50), (2, 3, 1)])
def test_moments_parity(lib, h, w, m, dtype):
    d = _ng(h, w, m, seed=h + w)
    u = torch.from_numpy(d["u"]).cuda().to(dtype)
    v = torch.from_numpy(d["v"]).cuda().to(dtype)
    mom = _np(G.lcp_moments(u, v))
    for comp, x in enumerate((u, v)):
        ref = S.ensemble_moments(_np(x))
        sd = np.sqrt(ref[1]) + 1e-30
        assert np.max(np.abs(mom[comp, ..., 0] - ref[0]) / (np.abs(ref[0]) + sd)) <= 1e-5
        for q, p in ((1, 2), (2, 3), (3, 4)):
            assert np.max(np.abs(mom[comp, ..., q] - ref[q]) / (sd ** p + 1e-30)) <= 2e-4, (comp, q)


def _features_ref(u, v, iso, dx=1.0, dy=1.0):
    kap = S.divergence_cumulants(S.ensemble_moments(u), S.ensemble_moments(v), dx, dy)
    return S.surrogate_features(kap, iso)


def test_features_parity(lib):
    d = _ng(41, 67, 20, seed=3)
    u, v = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()
    iso = d["isovalues"]
    feat, prior = G.lcp_surrogate_features(G.lcp_moments(u, v), iso, 1.0, 0.5)
    ref = _features_ref(d["u"], d["v"], iso, 1.0, 0.5).reshape(-1, 17)
    got = _np(feat)
    assert np.all(got[:, 17:] == 0.0)
    err = np.abs(got[:, :17] - ref)
    assert np.all(err <= 2e-2 + 1e-2 * np.abs(ref)), float(err.max())
    # the prior from the fp32 closed form: logit error ~ (closed-form error) / (g (1 - g)), clamped at 1e-6
    pr_ref = S.surrogate_prior(ref)
    g = 1.0 / (1.0 + np.exp(-pr_ref))
    assert np.all(np.abs(_np(prior) - pr_ref) <= 1e-3 + 1e-5 / (g * (1 - g)))


def test_forward_parity(lib):
    d = _ng(30, 40, 20, seed=5)
    feat, prior = G.lcp_surrogate_features(
        G.lcp_moments(torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()), d["isovalues"])
    p = _params(1)
    y = _np(G.lcp_mlp_forward(torch.from_numpy(G.mlp_pack(p)).cuda(), feat, prior))
    ref, _ = S.mlp_forward(_oracle_params_bf16(p), _np(feat)[:, :17], _np(prior))
    assert np.max(np.abs(y - ref)) <= 1e-2


def test_backward_parity(lib):
    d = _ng(30, 40, 20, seed=6)
    feat, prior = G.lcp_surrogate_features(
        G.lcp_moments(torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()), d["isovalues"])
    n = feat.shape[0]
    g = np.random.Generator(np.random.PCG64(9))
    t = g.uniform(0, 1, n).astype(np.float32)
    p = _params(2)
    grad, loss = G.lcp_mlp_backward(torch.from_numpy(G.mlp_pack(p)).cuda(), feat, prior, torch.from_numpy(t).cuda())
    po = _oracle_params_bf16(p)
    y, cache = S.mlp_forward(po, _np(feat)[:, :17], _np(prior))
    ref = S.mlp_backward(po, cache, t)
    got = G.mlp_unpack(_np(grad))
    # element by element: every gradient entry is a sum over rows of a product
    # of two per-row factors; the GPU rounds h1, dZ2 and dZ1 to bf16 (2^-9
    # relative), evaluates tanh in hardware (~2^-11) and carries those errors
    # through one more layer, so each product is within 2^-6 of the magnitude
    # of its terms and a sum within 2^-6 of the sum of magnitudes
    # (Sigma_r |a_r b_r| / n, the oracle's gradient of the same network with
    # absolute values), plus 2^-9 of the tensor's largest magnitude for the
    # saturated units whose tanh' = 1 - h^2 the rounding of h moves.
    mag = _abs_gradient(po, cache, t)
    for k in ref:
        a, b, m = (np.asarray(z, np.float64).ravel() for z in (got[k], ref[k], mag[k]))
        tol = 2.0 ** -6 * m + 2.0 ** -9 * m.max() + 1e-12
        assert np.all(np.abs(a - b) <= tol), (k, float(np.max(np.abs(a - b) / tol)))
    assert float(loss.item()) == pytest.approx(S.mse_loss(y, t), rel=1e-2)
    raw = _np(grad)
    assert np.all(raw[0:2048].reshape(64, 32)[:, 17:] == 0.0) and np.all(raw[6337:] == 0.0)


def _abs_gradient(params, cache, t):
    """Sigma over rows of |a_r b_r| / n for every gradient entry a^T b: the
    chain rule of the oracle with every factor replaced by its magnitude."""
    x, h1, h2, y = cache["x"], cache["h1"], cache["h2"], cache["y"]
    n = x.shape[0]
    dz3 = np.abs(2.0 * (y - np.asarray(t, np.float64)) / n * y * (1.0 - y))
    dz2 = dz3[:, None] * np.abs(params["w3"])[None, :] * (1.0 - h2 * h2)
    dz1 = (dz2 @ np.abs(params["W2"]).T) * (1.0 - h1 * h1)
    return dict(W1=np.abs(x).T @ dz1, b1=dz1.sum(axis=0), W2=np.abs(h1).T @ dz2, b2=dz2.sum(axis=0),
                w3=np.abs(h2).T @ dz3, b3=np.asarray(dz3.sum()))


def test_deterministic_backward_repeats_bit_for_bit_and_matches(lib):
    """lcp_mlp_backward_ws: the same bits on every call; the same gradient as
    the atomic variant up to fp32 summation order; the oracle bound of
    test_backward_parity holds for it too."""
    d = _ng(30, 40, 20, seed=6)
    feat, prior = G.lcp_surrogate_features(
        G.lcp_moments(torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()), d["isovalues"])
    n = feat.shape[0]
    t = torch.from_numpy(np.random.Generator(np.random.PCG64(9)).uniform(0, 1, n).astype(np.float32)).cuda()
    prm = torch.from_numpy(G.mlp_pack(_params(2))).cuda()
    g1, l1 = G.lcp_mlp_backward_ws(prm, feat, prior, t)
    g1, l1 = g1.clone(), l1.clone()
    for _ in range(3):
        g2, l2 = G.lcp_mlp_backward_ws(prm, feat, prior, t)
        assert torch.equal(g1, g2) and torch.equal(l1, l2)
    ga, la = G.lcp_mlp_backward(prm, feat, prior, t)
    assert torch.allclose(g1, ga, rtol=1e-4, atol=1e-9) and torch.allclose(l1, la, rtol=1e-5)
    po = _oracle_params_bf16(_params(2))
    _, cache = S.mlp_forward(po, _np(feat)[:, :17], _np(prior))
    ref, mag = S.mlp_backward(po, cache, _np(t)), _abs_gradient(po, cache, _np(t))
    got = G.mlp_unpack(_np(g1))
    for k in ref:
        a, b, m = (np.asarray(z, np.float64).ravel() for z in (got[k], ref[k], mag[k]))
        assert np.all(np.abs(a - b) <= 2.0 ** -6 * m + 2.0 ** -9 * m.max() + 1e-12), k


def test_training_resumes_from_a_checkpoint_bit_for_bit(lib, tmp_path):
    """Stop a run mid-epoch, save and restore it, and finish: parameters, Adam
    moments and step count equal the uninterrupted run's exactly."""
    d = _ng(48, 64, 20, seed=11)
    u, v = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()
    feat, prior = G.lcp_surrogate_features(G.lcp_moments(u, v), d["isovalues"])
    est, _ = lib.lcp_mc(d["isovalues"], 1000, 5, mode="empirical", members=(u, v))
    target = est.reshape(-1).contiguous()
    kw = dict(epochs=3, batch=1024, lr=3e-3, lr_final=1e-4, seed=4)
    a = G.Surrogate(synth.mlp_init_params(0, zero_output=True))
    a.fit(feat, prior, target, **kw)
    b = G.Surrogate(synth.mlp_init_params(0, zero_output=True))
    b.fit(feat, prior, target, stop_after=7, **kw)  # 7 batches: inside the first epoch of 16
    assert b.step == 7 and b.t == 7
    b.save(str(tmp_path / "ck.npz"))
    c = G.Surrogate.from_checkpoint(str(tmp_path / "ck.npz"))
    c.fit(feat, prior, target, **kw)
    assert c.step == a.step and c.t == a.t
    assert torch.equal(c.params, a.params) and torch.equal(c.m, a.m) and torch.equal(c.v, a.v)
    assert not torch.equal(b.params, a.params)  # the stopped run really was behind


def test_backward_ragged_batch_equals_sum_of_parts(lib):
    """Rows beyond n contribute nothing; the gradient of the mean is the
    row-weighted mean of the parts' gradients."""
    d = _ng(20, 25, 10, seed=7)
    feat, prior = G.lcp_surrogate_features(
        G.lcp_moments(torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()), d["isovalues"])
    n = feat.shape[0]
    t = torch.rand(n, generator=torch.Generator().manual_seed(3)).cuda()
    prm = torch.from_numpy(G.mlp_pack(_params(3))).cuda()
    full, _ = G.lcp_mlp_backward(prm, feat, prior, t)
    full = full.clone()
    cut = 777
    a, _ = G.lcp_mlp_backward(prm, feat[:cut], prior[:cut], t[:cut])
    a = a.clone()
    b, _ = G.lcp_mlp_backward(prm, feat[cut:], prior[cut:], t[cut:])
    comb = (a * cut + b * (n - cut)) / n
    # per-row bf16 values do not depend on n (the mean's 1/n is applied to the sums): only fp32 summation order differs
    assert torch.allclose(full, comb, rtol=1e-4, atol=1e-9)


def test_adam_parity(lib):
    p = _params(4)
    g = np.random.Generator(np.random.PCG64(11))
    grads = [G.mlp_pack({k: g.normal(0, 1, np.shape(v)) for k, v in p.items()}) for _ in range(3)]
    flat = torch.from_numpy(G.mlp_pack(p)).cuda()
    m, v = torch.zeros_like(flat), torch.zeros_like(flat)
    po = G.mlp_unpack(G.mlp_pack(p))
    st = {"t": 0, "m": {k: np.zeros_like(x) for k, x in po.items()}, "v": {k: np.zeros_like(x) for k, x in po.items()}}
    for step, gr in enumerate(grads, start=1):
        G.lcp_adam_step(flat, torch.from_numpy(gr).cuda(), m, v, step, 1e-2)
        S.adam_step(po, G.mlp_unpack(gr), st, 1e-2)
    got = G.mlp_unpack(_np(flat))
    for k in po:
        assert np.allclose(got[k], po[k], rtol=1e-5, atol=1e-6), k


@pytest.mark.parametrize("h,w", [(37, 53), (9, 100)])
def test_infer_equals_forward_over_features_and_oracle(lib, h, w):
    d = _ng(h, w, 20, seed=h)
    u, v = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()
    iso = d["isovalues"]
    p = _params(5)
    prm = torch.from_numpy(G.mlp_pack(p)).cuda()
    mom = G.lcp_moments(u, v)
    out = G.lcp_mlp_infer(mom, iso, prm)
    feat, prior = G.lcp_surrogate_features(mom, iso)
    via = G.lcp_mlp_forward(prm, feat, prior).reshape(len(iso), h - 1, w - 1)
    # the fused kernel (layer-1 tanh in bf16) and the row kernel (layer-1 tanh in fp32), both tcgen05, on the same feature
    # rows: both round h1 to bf16; they differ by an ulp of h1 here and there and the summation order
    assert torch.allclose(out, via, atol=5e-3, rtol=0), float((out - via).abs().max())
    fref = _features_ref(d["u"], d["v"], iso).reshape(-1, 17)
    ref, _ = S.mlp_forward(_oracle_params_bf16(p), fref, S.surrogate_prior(fref))
    assert np.max(np.abs(_np(out).ravel() - ref)) <= 2e-2
    # an untrained output layer reproduces the Gaussian closed form (feature 16) through the prior
    p0 = dict(p, w3=np.zeros(64, np.float32), b3=np.zeros((), np.float32))
    y0 = _np(G.lcp_mlp_infer(mom, iso, torch.from_numpy(G.mlp_pack(p0)).cuda())).ravel()
    g = np.clip(fref[:, 16], 1e-6, 1 - 1e-6)
    assert np.max(np.abs(y0 - g)) <= 1e-5
    o16 = G.lcp_mlp_infer(mom, iso, prm, out_dtype=torch.float16)
    assert torch.allclose(o16.float(), out, atol=1e-3, rtol=0)


def _training_rows(lib, seed, h, w, label_seed):
    """Feature rows, priors and empirical-mode Monte Carlo labels (S = 1e4) of
    the interior cells of one non-Gaussian field."""
    d = synth.non_gaussian_ensemble(seed, h=h, w=w, m=50, k=8)
    u, v = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()
    feat, prior = G.lcp_surrogate_features(G.lcp_moments(u, v), d["isovalues"])
    est, _ = lib.lcp_mc(d["isovalues"], 10000, label_seed, mode="empirical", members=(u, v))
    inner = torch.zeros(est.shape, dtype=torch.bool, device="cuda")
    inner[:, 1:-1, 1:-1] = True
    sel = inner.reshape(-1)
    return feat[sel], prior[sel], est.reshape(-1)[sel]


@pytest.mark.slow
def test_trained_network_beats_the_closed_form_on_held_out_data(lib):
    """Trained on five non-Gaussian fields (skew-normal / Gaussian-mixture
    noise), judged on two others against the exact LCP of the empirical model:
    the network's RMS and its largest error are both below the Gaussian closed
    form's (the method without it, which it starts from)."""
    parts = [_training_rows(lib, s, h, w, ls) for s, h, w, ls in
             ((1, 384, 384, 123), (3, 192, 256, 321), (4, 384, 384, 444), (5, 384, 384, 555), (7, 384, 384, 777))]
    X, P, T = (torch.cat([p[q] for p in parts]).contiguous() for q in range(3))
    net = G.Surrogate(synth.mlp_init_params(0, zero_output=True))
    losses = net.fit(X, P, T, epochs=40, batch=8192, lr=3e-3, lr_final=1e-4)
    assert losses[-1] < losses[0]
    for seed, (y0, x0, n) in ((2, (40, 50, 36)), (6, (100, 100, 40))):
        d = synth.non_gaussian_ensemble(seed, h=160, w=160, m=50, k=8)
        u, v = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()
        iso = d["isovalues"]
        exact = O.exact_empirical_lcp(d["u"][:, y0:y0 + n, x0:x0 + n], d["v"][:, y0:y0 + n, x0:x0 + n], 1.0, 1.0, iso)

        def err(m):
            e = _np(m)[:, y0 + 1:y0 + n - 2, x0 + 1:x0 + n - 2] - exact
            return float(np.sqrt((e * e).mean())), float(np.abs(e).max())

        closed, _ = lib.lcp_fused(u, v, iso, 1.0, 1.0, 0)  # plug-in variances: the empirical model's
        learned = net.infer(G.lcp_moments(u, v), iso)
        rms_c, max_c = err(closed)
        rms_l, max_l = err(learned)
        assert rms_l < 0.9 * rms_c, (seed, rms_l, rms_c)
        assert max_l <= max_c, (seed, max_l, max_c)
