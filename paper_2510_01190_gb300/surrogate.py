"""Learned surrogate of the LCP for ensembles that are not Gaussian.

Thin marshalling over the C ABI (``lcp_moments``, ``lcp_surrogate_features``,
``lcp_mlp_forward``, ``lcp_mlp_backward``, ``lcp_adam_step``,
``lcp_mlp_infer``): every arithmetic step runs in the library's kernels; this
module allocates tensors, packs parameters and sequences the training steps.

The network (17 -> 64 -> 64 -> 1, tanh, tanh, sigmoid) maps per-cell features
of the divergence cumulants (see ``include/lcp.h``) to the crossing
probability; it is trained on Monte Carlo labels of the empirical model
(``lcp_mc`` in empirical mode) and evaluated in one fused kernel from the
members' moments.
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._binding import _check, _dtype_code, _iso, _members, _ptr, _stream, load

__all__ = [
    "MLP_NPARAMS",
    "FEAT_STRIDE",
    "mlp_pack",
    "mlp_unpack",
    "lcp_moments",
    "lcp_surrogate_features",
    "lcp_mlp_forward",
    "lcp_mlp_backward",
    "lcp_mlp_backward_ws",
    "lcp_adam_step",
    "lcp_mlp_infer",
    "Surrogate",
]

MLP_NPARAMS = 6340
FEAT_STRIDE = 32
_OFF = dict(W1=0, b1=2048, W2=2112, b2=6208, w3=6272, b3=6336)

c_vp, c_int, c_i64, c_double, c_float = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_float
c_fp = ctypes.POINTER(ctypes.c_float)
_SIGS = {
    "lcp_moments": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int, c_i64, c_vp, c_vp]),
    "lcp_surrogate_features": (c_int, [c_vp, c_int, c_int, c_double, c_double, c_fp, c_int, c_vp, c_vp, c_vp]),
    "lcp_mlp_forward": (c_int, [c_vp, c_vp, c_vp, c_i64, c_vp, c_vp]),
    "lcp_mlp_backward": (c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp]),
    "lcp_mlp_backward_workspace_bytes": (ctypes.c_size_t, [c_i64]),
    "lcp_mlp_backward_ws": (c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "lcp_adam_step": (c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_int, c_float, c_float, c_float, c_float, c_vp]),
    "lcp_mlp_infer": (c_int, [c_vp, c_int, c_int, c_double, c_double, c_fp, c_int, c_vp, c_vp, c_int, c_vp]),
}


def _lib():
    lib = load()
    if not getattr(lib, "_surrogate_sigs", False):
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        lib._surrogate_sigs = True
    return lib


def mlp_pack(params) -> np.ndarray:
    """Network parameters (dict: W1 [17, 64], b1, W2 [64, 64], b2, w3 [64], b3,
    written as x @ W) into the library's flat fp32 layout (W1 and W2 stored
    [output unit][input]; W1 padded to 32 inputs)."""
    flat = np.zeros(MLP_NPARAMS, np.float32)
    w1 = np.zeros((64, FEAT_STRIDE), np.float32)
    w1[:, :17] = np.asarray(params["W1"], np.float32).T
    flat[_OFF["W1"]:_OFF["W1"] + 2048] = w1.ravel()
    flat[_OFF["b1"]:_OFF["b1"] + 64] = params["b1"]
    flat[_OFF["W2"]:_OFF["W2"] + 4096] = np.asarray(params["W2"], np.float32).T.ravel()
    flat[_OFF["b2"]:_OFF["b2"] + 64] = params["b2"]
    flat[_OFF["w3"]:_OFF["w3"] + 64] = params["w3"]
    flat[_OFF["b3"]] = float(np.asarray(params["b3"]))
    return flat


def mlp_unpack(flat) -> dict:
    """Inverse of ``mlp_pack`` (float64 arrays)."""
    f = np.asarray(flat, np.float64)
    return dict(W1=f[0:2048].reshape(64, FEAT_STRIDE)[:, :17].T.copy(), b1=f[2048:2112].copy(),
                W2=f[2112:6208].reshape(64, 64).T.copy(), b2=f[6208:6272].copy(), w3=f[6272:6336].copy(),
                b3=np.asarray(f[6336]))


def lcp_moments(u, v, out=None):
    """Plug-in moments (mean, m2, m3, m4) of every vertex component: [2, H, W, 4] fp32."""
    m, h, w, stride = _members(u, v)
    if out is None:
        out = torch.empty((2, h, w, 4), dtype=torch.float32, device=u.device)
    _check(_lib().lcp_moments(_ptr(u), _ptr(v), _dtype_code(u.dtype), m, h, w, stride, _ptr(out), _stream()))
    return out


def lcp_surrogate_features(mom, isovalues, dx: float = 1.0, dy: float = 1.0, out=None, prior=None):
    """Feature rows of every cell and isovalue, bf16 [K (H-1)(W-1), 32], and
    their priors (logit of the Gaussian closed form), fp32 [K (H-1)(W-1)]."""
    _, h, w, _ = mom.shape
    iso, k, iso_p = _iso(isovalues)
    n = k * (h - 1) * (w - 1)
    if out is None:
        out = torch.empty((n, FEAT_STRIDE), dtype=torch.bfloat16, device=mom.device)
    if prior is None:
        prior = torch.empty(n, dtype=torch.float32, device=mom.device)
    _check(_lib().lcp_surrogate_features(_ptr(mom), h, w, float(dx), float(dy), iso_p, k, _ptr(out), _ptr(prior),
                                         _stream()))
    return out, prior


def lcp_mlp_forward(params, feat, prior=None, out=None):
    n = feat.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=feat.device)
    _check(_lib().lcp_mlp_forward(_ptr(params), _ptr(feat), _ptr(prior), n, _ptr(out), _stream()))
    return out


def lcp_mlp_backward(params, feat, prior, target, grad=None, loss=None):
    """Gradient of the mean squared error and the loss (device tensors)."""
    n = feat.shape[0]
    if grad is None:
        grad = torch.empty(MLP_NPARAMS, dtype=torch.float32, device=feat.device)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
    _check(_lib().lcp_mlp_backward(_ptr(params), _ptr(feat), _ptr(prior), _ptr(target), n, _ptr(grad), _ptr(loss),
                                   _stream()))
    return grad, loss


def lcp_mlp_backward_ws(params, feat, prior, target, grad=None, loss=None, workspace=None):
    """lcp_mlp_backward with a result that is bitwise the same on every run
    (per-CTA partial sums reduced in CTA order through ``workspace``, a uint8
    device tensor of lcp_mlp_backward_workspace_bytes(n); one is allocated if
    none is given)."""
    n = feat.shape[0]
    lib = _lib()
    if grad is None:
        grad = torch.empty(MLP_NPARAMS, dtype=torch.float32, device=feat.device)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
    need = int(lib.lcp_mlp_backward_workspace_bytes(n))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=feat.device)
    _check(lib.lcp_mlp_backward_ws(_ptr(params), _ptr(feat), _ptr(prior), _ptr(target), n, _ptr(grad), _ptr(loss),
                                   _ptr(workspace), workspace.numel(), _stream()))
    return grad, loss


def lcp_adam_step(params, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                  eps: float = 1e-8):
    _check(_lib().lcp_adam_step(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(), int(t), float(lr),
                                float(beta1), float(beta2), float(eps), _stream()))


def lcp_mlp_infer(mom, isovalues, params, dx: float = 1.0, dy: float = 1.0, out_dtype=torch.float32, out=None):
    """The learned LCP map [K, H-1, W-1] from moments, one fused kernel."""
    _, h, w, _ = mom.shape
    iso, k, iso_p = _iso(isovalues)
    if out is None:
        out = torch.empty((k, h - 1, w - 1), dtype=out_dtype, device=mom.device)
    _check(_lib().lcp_mlp_infer(_ptr(mom), h, w, float(dx), float(dy), iso_p, k, _ptr(params), _ptr(out),
                                _dtype_code(out.dtype), _stream()))
    return out


class Surrogate:
    """The network's parameters and Adam state on a device, trained and used
    through the library's kernels.  Training is reproducible bit for bit (the
    deterministic backward, element-wise Adam, a seeded shuffle), so a run
    stopped at any step and resumed from ``checkpoint()`` ends with the same
    parameters and Adam moments as the run that never stopped."""

    def __init__(self, init_params: dict, device="cuda"):
        self.params = torch.from_numpy(mlp_pack(init_params)).to(device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.empty_like(self.params)
        self.loss = torch.empty(1, dtype=torch.float32, device=device)
        self.t = 0          # Adam steps taken
        self.step = 0       # position in the current fit's schedule (batches done)
        self.ws = None

    def fit(self, feat, prior, target, epochs: int = 4, batch: int = 8192, lr: float = 3e-3,
            lr_final: float = 3e-4, seed: int = 0, stop_after: int | None = None):
        """Minibatch Adam on (feat [n, 32] bf16, prior [n] fp32, target [n] fp32).  The rows are
        shuffled once (seeded); each epoch walks them in batches, the learning
        rate decaying geometrically from lr to lr_final.  The schedule starts at
        batch ``self.step`` (0 for a fresh network, the checkpoint's step for a
        resumed one) and stops after ``stop_after`` batches of this call, or at
        its end.  Returns the loss of every epoch's last batch done here."""
        n = feat.shape[0]
        g = torch.Generator(device=feat.device)
        g.manual_seed(int(seed))
        perm = torch.randperm(n, generator=g, device=feat.device)
        feat, prior, target = feat[perm].contiguous(), prior[perm].contiguous(), target[perm].contiguous()
        per_epoch = (n + batch - 1) // batch
        steps = epochs * per_epoch
        decay = (lr_final / lr) ** (1.0 / max(1, steps - 1))
        rate = lr
        for _ in range(self.step):  # the rate at the resumed step, by the same products as an unbroken run
            rate *= decay
        need = int(_lib().lcp_mlp_backward_workspace_bytes(min(n, batch)))
        if self.ws is None or self.ws.numel() < need:
            self.ws = torch.empty(need, dtype=torch.uint8, device=feat.device)
        losses, done = [], 0
        while self.step < steps and (stop_after is None or done < stop_after):
            s = (self.step % per_epoch) * batch
            e = min(n, s + batch)
            lcp_mlp_backward_ws(self.params, feat[s:e], prior[s:e], target[s:e], self.grad, self.loss, self.ws)
            self.t += 1
            lcp_adam_step(self.params, self.grad, self.m, self.v, self.t, rate)
            rate *= decay
            self.step += 1
            done += 1
            if self.step % per_epoch == 0:
                losses.append(float(self.loss.item()))  # loss of the epoch's last batch
        return losses

    def predict(self, feat, prior):
        return lcp_mlp_forward(self.params, feat, prior)

    def infer(self, mom, isovalues, dx: float = 1.0, dy: float = 1.0, out_dtype=torch.float32, out=None):
        return lcp_mlp_infer(mom, isovalues, self.params, dx, dy, out_dtype, out)

    def state(self) -> dict:
        return mlp_unpack(self.params.detach().cpu().numpy())

    def checkpoint(self) -> dict:
        """Everything training needs to continue: parameters, Adam moments and
        step count, and the position in the schedule (host numpy arrays)."""
        return {"params": self.params.detach().cpu().numpy().copy(), "m": self.m.detach().cpu().numpy().copy(),
                "v": self.v.detach().cpu().numpy().copy(), "t": np.int64(self.t), "step": np.int64(self.step)}

    def save(self, path: str):
        np.savez(path, **self.checkpoint())

    @classmethod
    def from_checkpoint(cls, ck, device="cuda"):
        """A network restored from ``checkpoint()`` (a dict, or the path of a ``save()`` file)."""
        if isinstance(ck, str):
            with np.load(ck) as z:
                ck = {k: z[k] for k in z.files}
        net = cls.__new__(cls)
        net.params = torch.from_numpy(np.asarray(ck["params"], np.float32).copy()).to(device)
        net.m = torch.from_numpy(np.asarray(ck["m"], np.float32).copy()).to(device)
        net.v = torch.from_numpy(np.asarray(ck["v"], np.float32).copy()).to(device)
        net.grad = torch.empty_like(net.params)
        net.loss = torch.empty(1, dtype=torch.float32, device=device)
        net.t = int(ck["t"])
        net.step = int(ck["step"])
        net.ws = None
        return net
