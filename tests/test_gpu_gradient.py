"""Speed-gradient preprocessing (Sec. 4.2, reading R19) on the GPU against the
FP64 oracle: the gradient members, and the LCP map with the preprocessing fused
into the statistics pass (single and multi-band, K up to 40, fp16 maps, bf16
members, the full 8192 x 8192 eddy workload on sampled crops)."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2510_01190_gb300 import synth

pytestmark = pytest.mark.gpu

LCP_TOL = 1e-5
EPS32 = 2.0 ** -23


def _np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def _members(seed, m, h, w, dtype, scale=1.0):
    g = np.random.Generator(np.random.PCG64(seed))
    u = torch.from_numpy(g.normal(0.3, scale, (m, h, w)).astype(np.float32)).cuda().to(dtype)
    v = torch.from_numpy(g.normal(-0.2, scale, (m, h, w)).astype(np.float32)).cuda().to(dtype)
    return u, v


def _mask_guard(mu_d, iso, band=1e-5):
    """Cells none of whose vertices lies within ``band`` of the isovalue."""
    out = []
    for c in iso:
        far = np.abs(mu_d - float(c)) > band
        out.append(far[:-1, :-1] & far[:-1, 1:] & far[1:, :-1] & far[1:, 1:])
    return np.stack(out)


@pytest.mark.parametrize("m,h,w,dx,dy,dtype", [(5, 7, 9, 1.0, 1.0, torch.float32), (3, 2, 2, 0.5, 2.0, torch.float32),
                                               (20, 37, 65, 1.0, 1.0, torch.bfloat16), (1, 5, 33, 0.25, 1.0, torch.float32)])
def test_speed_gradient_members(lib, m, h, w, dx, dy, dtype):
    u, v = _members(m * h + w, m, h, w, dtype)
    gx, gy = lib.lcp_speed_gradient(u, v, dx, dy)
    rx, ry = O.speed_gradient(_np(u), _np(v), dx, dy)
    s_max = float(np.max(np.hypot(_np(u), _np(v))))
    tol = 8 * EPS32 * s_max / min(dx, dy)
    assert np.max(np.abs(_np(gx) - rx)) <= tol
    assert np.max(np.abs(_np(gy) - ry)) <= tol


def _check_lcp(lib, u, v, iso, dx, dy, ddof=1, out_dtype=torch.float32, tol=LCP_TOL):
    lcp, mask = lib.lcp_speed_gradient_ws(u, v, iso, dx, dy, ddof, out_dtype=out_dtype, mask=True)
    ref = O.speed_gradient_lcp(_np(u), _np(v), dx, dy, iso, ddof)
    got = _np(lcp)
    assert got.shape == ref["lcp"].shape
    err = np.max(np.abs(got - ref["lcp"]))
    assert err <= tol, err
    h, w = u.shape[1:]
    guard = _mask_guard(ref["mu_d"], iso)
    gm = lib.unpack_mask(mask, w).cpu().numpy()
    assert np.array_equal(gm[guard], ref["mask"][guard])
    return lcp, ref


@pytest.mark.parametrize("m,h,w,dtype", [(20, 96, 130, torch.bfloat16), (12, 19, 241, torch.float32),
                                         (4, 2, 2, torch.float32), (7, 3, 31, torch.float32)])
def test_speed_gradient_ws_eddies(lib, m, h, w, dtype):
    d = synth.eddy_ensemble_torch(3, h=h, w=w, m=m, n_eddies=max(2, h * w // 2000), dtype=dtype)
    _check_lcp(lib, d["u"], d["v"], synth.EDDY_GRADIENT_ISOVALUES, 1.0, 1.0)


def test_speed_gradient_ws_spacing_ddof0_single_member(lib):
    u, v = _members(5, 1, 23, 40, torch.float32)
    _check_lcp(lib, u, v, [-0.5, 0.0, 0.7], 0.5, 1.5, ddof=0)
    u, v = _members(6, 9, 23, 40, torch.float32)
    _check_lcp(lib, u, v, [-0.5, 0.0, 0.7], 2.0, 0.75, ddof=0)


@pytest.mark.parametrize("k,out_dtype", [(11, torch.float32), (40, torch.float16)])
def test_speed_gradient_ws_many_isovalues(lib, k, out_dtype):
    d = synth.fourier_ensemble(8, h=45, w=70, m=10, k=4)
    u, v = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()
    gx, gy = O.speed_gradient(d["u"], d["v"], 1.0, 1.0)
    mu = O.divergence_of_field(gx.mean(axis=0), gy.mean(axis=0), 1.0, 1.0)
    iso = np.quantile(mu, np.linspace(0.03, 0.97, k)).astype(np.float32)
    tol = LCP_TOL if out_dtype == torch.float32 else 2.0 ** -11  # fp16 maps: half an ulp of 1 plus the fp32 error
    _check_lcp(lib, u, v, iso, 1.0, 1.0, out_dtype=out_dtype, tol=tol)


def test_speed_gradient_ws_several_bands(lib):
    """8192 columns: the 96 MB record budget holds 376 cell rows, so 400 rows
    run as two bands whose halo rows must join seamlessly."""
    u, v = _members(12, 3, 400, 8192, torch.float32, scale=0.5)
    _check_lcp(lib, u, v, [-0.2, 0.1], 1.0, 1.0)


def test_fused_equals_preprocess_then_lcp_fused_ws(lib):
    d = synth.eddy_ensemble_torch(4, h=150, w=211, m=16, n_eddies=20, dtype=torch.float32)
    iso = synth.EDDY_GRADIENT_ISOVALUES
    fused, _ = lib.lcp_speed_gradient_ws(d["u"], d["v"], iso)
    gx, gy = lib.lcp_speed_gradient(d["u"], d["v"])
    two_step, _ = lib.lcp_fused_ws(gx, gy, iso)
    assert torch.max(torch.abs(fused - two_step)).item() <= 1e-6


def test_speed_gradient_ws_8192_bf16_sampled(lib):
    """The full eddy workload (8192^2, 20 bf16 members, the bench's launch
    configuration); the oracle evaluates crops and the cells whose stencils
    (speeds within 3 vertices) lie inside a crop are compared."""
    if torch.cuda.get_device_properties(0).total_memory < 60e9:
        pytest.skip("needs the full-size device memory")
    d = synth.eddy_ensemble_torch(0)
    u, v = d["u"], d["v"]
    iso = synth.EDDY_GRADIENT_ISOVALUES
    H, W = u.shape[1:]
    lcp, mask = lib.lcp_speed_gradient_ws(u, v, iso, mask=True)
    torch.cuda.synchronize()
    for (y0, x0) in ((0, 0), (5003, 2999), (H - 60, W - 90)):
        y1, x1 = min(y0 + 60, H), min(x0 + 90, W)
        ref = O.speed_gradient_lcp(_np(u[:, y0:y1, x0:x1]), _np(v[:, y0:y1, x0:x1]), 1.0, 1.0, iso)
        vy = np.ones(y1 - y0, bool)
        vx = np.ones(x1 - x0, bool)
        if y0 > 0:
            vy[:3] = False
        if y1 < H:
            vy[-3:] = False
        if x0 > 0:
            vx[:3] = False
        if x1 < W:
            vx[-3:] = False
        sel = (vy[:-1] & vy[1:])[:, None] & (vx[:-1] & vx[1:])[None, :]
        got = _np(lcp[:, y0:y1 - 1, x0:x1 - 1])
        assert np.max(np.abs(got - ref["lcp"])[:, sel]) <= LCP_TOL
        guard = _mask_guard(ref["mu_d"], iso) & sel[None]
        gm = lib.unpack_mask(mask[:, y0:y1 - 1], W).cpu().numpy()[:, :, x0:x1 - 1]
        assert np.array_equal(gm[guard], ref["mask"][guard])
    del u, v, lcp, mask, d
    torch.cuda.empty_cache()
