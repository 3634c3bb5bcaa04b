"""3D fields on the GPU against the FP64 oracle (reading R20): the fused
ring-of-planes path (single and multi-slab, K up to 11 in passes, fp16 maps,
bf16 members, spacing, ddof 0), the unfused divergence and map steps, and the
256^3 workload of the bench on sampled crops."""

import numpy as np
import pytest
import torch

import oracle as O
from oracle import volume as V3
from paper_2510_01190_gb300 import synth

pytestmark = pytest.mark.gpu

LCP_TOL = 1e-5


def _np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def _guard(mu_d, iso, band=1e-5):
    """Cells none of whose 8 vertices lies within ``band`` of the isovalue."""
    out = []
    for c in iso:
        far = np.abs(mu_d - float(c)) > band
        g = np.ones(tuple(n - 1 for n in mu_d.shape), bool)
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    g &= far[dk:dk + g.shape[0], dj:dj + g.shape[1], di:di + g.shape[2]]
        out.append(g)
    return np.stack(out)


def _volume(seed, m, d, h, w, dtype=torch.float32, kmax=3):
    return synth.fourier_volume_torch(seed, d=d, h=h, w=w, m=m, k=1, kmax=kmax, device="cuda", dtype=dtype)


def _iso_from(mu_d, k):
    return np.quantile(mu_d, np.linspace(0.1, 0.9, k)).astype(np.float32)


def _check(lib, u, v, w, iso, dx=1.0, dy=1.0, dz=1.0, ddof=1, out_dtype=torch.float32, tol=LCP_TOL):
    lcp, mask = lib.lcp3d_fused_ws(u, v, w, iso, dx, dy, dz, ddof, out_dtype=out_dtype, mask=True)
    ref = V3.lcp_closed_form_3d(_np(u), _np(v), _np(w), dx, dy, dz, iso, ddof)
    got = _np(lcp)
    assert got.shape == ref["lcp"].shape
    err = float(np.max(np.abs(got - ref["lcp"])))
    assert err <= tol, err
    wd = u.shape[-1]
    gm = lib.unpack_mask(mask.reshape(-1, mask.shape[-2], mask.shape[-1]), wd).cpu().numpy().reshape(ref["mask"].shape)
    guard = _guard(ref["mu_d"], iso)
    assert np.array_equal(gm[guard], ref["mask"][guard])
    return lcp, ref


@pytest.mark.parametrize("m,d,h,w,k", [(6, 5, 7, 40, 3), (4, 2, 2, 2, 1), (10, 9, 33, 65, 4), (5, 3, 4, 97, 2)])
def test_fused_3d_matches_oracle(lib, m, d, h, w, k):
    vol = _volume(m + d, m, d, h, w)
    ref0 = V3.lcp_closed_form_3d(_np(vol["u"]), _np(vol["v"]), _np(vol["w"]), 1.0, 1.0, 1.0, [0.0])
    _check(lib, vol["u"], vol["v"], vol["w"], _iso_from(ref0["mu_d"], k))


def test_fused_3d_eight_and_eleven_isovalues_bf16_fp16(lib):
    vol = _volume(3, 8, 6, 10, 70, dtype=torch.bfloat16)
    ref0 = V3.lcp_closed_form_3d(_np(vol["u"]), _np(vol["v"]), _np(vol["w"]), 1.0, 1.0, 1.0, [0.0])
    _check(lib, vol["u"], vol["v"], vol["w"], _iso_from(ref0["mu_d"], 8))
    _check(lib, vol["u"], vol["v"], vol["w"], _iso_from(ref0["mu_d"], 11), out_dtype=torch.float16, tol=2.0 ** -11)


def test_fused_3d_spacing_ddof0_single_member(lib):
    vol = _volume(4, 7, 5, 9, 44)
    ref0 = V3.lcp_closed_form_3d(_np(vol["u"]), _np(vol["v"]), _np(vol["w"]), 0.5, 2.0, 1.5, [0.0])
    iso = _iso_from(ref0["mu_d"], 3)
    _check(lib, vol["u"], vol["v"], vol["w"], iso, 0.5, 2.0, 1.5, ddof=0)
    _check(lib, vol["u"][:1].contiguous(), vol["v"][:1].contiguous(), vol["w"][:1].contiguous(), iso, 0.5, 2.0, 1.5,
           ddof=0)


def test_fused_3d_ring_of_several_slabs(lib):
    """256 x 683 planes are 8 MB of records each: the ring holds a few planes
    (2B + 3 for B new planes per slab), so 9 planes run as several slabs that
    reuse the 3 older planes while the next slab's statistics are written."""
    vol = _volume(5, 3, 9, 256, 683)
    plane = 256 * 683 * 48
    ws = lib.lcp3d_workspace_bytes(3, 9, 256, 683)
    assert ws % plane == 0 and 5 <= ws // plane < 9 + 3 and (ws // plane - 3) % 2 == 0
    ref0 = V3.lcp_closed_form_3d(_np(vol["u"]), _np(vol["v"]), _np(vol["w"]), 1.0, 1.0, 1.0, [0.0])
    _check(lib, vol["u"], vol["v"], vol["w"], _iso_from(ref0["mu_d"], 2))


def test_unfused_divergence_and_map(lib):
    vol = _volume(6, 9, 6, 11, 37)
    u, v, w = vol["u"], vol["v"], vol["w"]
    m, d, h, wd = u.shape
    flat = lambda t: t.reshape(m, d * h, wd)  # noqa: E731
    mu_u, var_u, mu_v, var_v = lib.lcp_stats(flat(u), flat(v))
    mu_w, var_w, _, _ = lib.lcp_stats(flat(w), flat(w))
    st = [t.reshape(d, h, wd) for t in (mu_u, var_u, mu_v, var_v, mu_w, var_w)]
    mu_d, var_d = lib.lcp3d_divergence(*st, 0.5, 1.0, 2.0)
    ref = V3.lcp_closed_form_3d(_np(u), _np(v), _np(w), 0.5, 1.0, 2.0, [0.0])
    scale = float(np.max(np.abs(ref["mu_d"])))
    assert np.max(np.abs(_np(mu_d) - ref["mu_d"])) <= 1e-5 * max(1.0, scale)
    assert np.max(np.abs(_np(var_d) - ref["var_d"]) / np.maximum(ref["var_d"], 1e-30)) <= 1e-5
    iso = _iso_from(ref["mu_d"], 5)
    lcp, mask = lib.lcp3d_map(mu_d, var_d, iso, mask=True)
    ref = V3.lcp_closed_form_3d(_np(u), _np(v), _np(w), 0.5, 1.0, 2.0, iso)
    assert np.max(np.abs(_np(lcp) - ref["lcp"])) <= LCP_TOL
    gm = lib.unpack_mask(mask.reshape(-1, h - 1, mask.shape[-1]), wd).cpu().numpy().reshape(ref["mask"].shape)
    guard = _guard(ref["mu_d"], iso)
    assert np.array_equal(gm[guard], ref["mask"][guard])
    fused, _ = lib.lcp3d_fused_ws(u, v, w, iso, 0.5, 1.0, 2.0)
    assert torch.max(torch.abs(fused - lcp)).item() <= 2e-6


def test_fused_3d_256_cubed_sampled(lib):
    """The bench workload (256^3, 20 fp32 members of u, v, w, K = 4); the oracle
    evaluates crops and the cells whose stencils lie inside a crop are compared."""
    vol = synth.fourier_volume_torch(0)
    u, v, w, iso = vol["u"], vol["v"], vol["w"], vol["isovalues"]
    D, H, W = u.shape[1:]
    lcp, mask = lib.lcp3d_fused_ws(u, v, w, iso, mask=True)
    torch.cuda.synchronize()
    for (z0, y0, x0) in ((0, 0, 0), (120, 77, 131), (D - 8, H - 9, W - 40)):
        z1, y1, x1 = min(z0 + 8, D), min(y0 + 9, H), min(x0 + 40, W)
        crop = lambda t: _np(t[:, z0:z1, y0:y1, x0:x1])  # noqa: E731
        ref = V3.lcp_closed_form_3d(crop(u), crop(v), crop(w), 1.0, 1.0, 1.0, iso)
        valid = []
        for a0, a1, n in ((z0, z1, D), (y0, y1, H), (x0, x1, W)):
            ok = np.ones(a1 - a0, bool)
            ok[0], ok[-1] = a0 == 0, a1 == n  # crop faces that are not grid faces have one-sided stencils
            valid.append(ok[:-1] & ok[1:])
        sel = valid[0][:, None, None] & valid[1][None, :, None] & valid[2][None, None, :]
        got = _np(lcp[:, z0:z1 - 1, y0:y1 - 1, x0:x1 - 1])
        assert np.max(np.abs(got - ref["lcp"])[:, sel]) <= LCP_TOL
        words = mask[:, z0:z1 - 1, y0:y1 - 1]
        gm = lib.unpack_mask(words.reshape(-1, words.shape[-2], words.shape[-1]), W).cpu().numpy()
        gm = gm.reshape(len(iso), z1 - z0 - 1, y1 - y0 - 1, W - 1)[..., x0:x1 - 1]
        guard = _guard(ref["mu_d"], iso) & sel[None]
        assert np.array_equal(gm[guard], ref["mask"][guard])
    del u, v, w, lcp, mask, vol
    torch.cuda.empty_cache()
