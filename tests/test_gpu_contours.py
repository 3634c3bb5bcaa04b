"""Isocontour segments on the GPU against the oracle (reading R18): keys and
counts identical (the crossing and saddle decisions are taken in fp32 on both
sides), coordinates within a few fp32 ulps; single-pass compaction across many
tiles, capacity truncation, determinism, NaN cells, mean-field and spaghetti
contours."""

import numpy as np
import pytest
import torch

import oracle as O
from oracle import viz as V
from paper_2510_01190_gb300 import synth

pytestmark = pytest.mark.gpu


def _coord_tol(segs):
    return 1e-6 + 4.0 * 2.0 ** -23 * np.maximum(np.abs(segs), 1.0)


def _compare(seg, key, total, ref_keys, ref_segs):
    assert total == ref_keys.size
    got_k = key.cpu().numpy()
    assert np.array_equal(got_k, ref_keys)
    got_s = seg.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got_s - ref_segs) <= _coord_tol(ref_segs))


@pytest.mark.parametrize("h,w,k", [(17, 19, 3), (2, 2, 1), (33, 1100, 2), (300, 257, 4)])
def test_contours_random_fields(lib, h, w, k):
    g = np.random.Generator(np.random.PCG64(h * w + k))
    f = g.normal(0, 1, (h, w)).astype(np.float32)
    f[::7, ::5] = 0.25  # exact ties with an isovalue: not below
    iso = np.array([-0.7, 0.0, 0.25, 1.1][:k], np.float32)
    seg, key, total = lib.lcp_contours(torch.from_numpy(f).cuda(), iso)
    _compare(seg, key, total, *V.marching_squares(f, iso))


def test_contours_forty_isovalues_take_the_wide_masks(lib):
    g = np.random.Generator(np.random.PCG64(40))
    f = g.normal(0, 1, (45, 77)).astype(np.float32)
    iso = np.linspace(-2.0, 2.0, 40).astype(np.float32)[g.permutation(40)]  # unsorted on purpose
    seg, key, total = lib.lcp_contours(torch.from_numpy(f).cuda(), iso)
    _compare(seg, key, total, *V.marching_squares(f, iso))
    u = torch.from_numpy(g.normal(0, 1, (3, 20, 33)).astype(np.float32)).cuda()
    v = torch.from_numpy(g.normal(0, 1, (3, 20, 33)).astype(np.float32)).cuda()
    seg, key, total = lib.lcp_member_contours(u, v, iso[:35])
    _compare(seg, key, total, *V.spaghetti_contours(u.cpu().numpy(), v.cpu().numpy(), 1.0, 1.0, iso[:35]))


def test_contours_smooth_field_closed_loops_and_nan(lib):
    y, x = np.mgrid[0:90, 0:130].astype(np.float64)
    f = (np.sin(x / 9.0) * np.cos(y / 7.0) + 0.1 * np.sin(x / 3.1 + y / 4.3)).astype(np.float32)
    f[40:43, 60:62] = np.nan
    iso = np.array([-0.5, 0.0, 0.3], np.float32)
    seg, key, total = lib.lcp_contours(torch.from_numpy(f).cuda(), iso)
    _compare(seg, key, total, *V.marching_squares(f, iso))


def test_contours_capacity_and_determinism(lib):
    g = np.random.Generator(np.random.PCG64(5))
    f = torch.from_numpy(g.normal(0, 1, (200, 333)).astype(np.float32)).cuda()
    iso = [0.0, 0.5]
    seg, key, total = lib.lcp_contours(f, iso)
    s2, k2, t2 = lib.lcp_contours(f, iso)
    assert t2 == total and torch.equal(s2, seg) and torch.equal(k2, key)
    cap = total // 3
    s3, k3, t3 = lib.lcp_contours(f, iso, capacity=cap)
    assert t3 == total and s3.shape[0] == cap
    assert torch.equal(s3, seg[:cap]) and torch.equal(k3, key[:cap])
    s4, k4, t4 = lib.lcp_contours(f, iso, capacity=0)
    assert t4 == total and s4.shape[0] == 0
    flat = torch.full((40, 50), 2.0, device="cuda")
    assert lib.lcp_contours(flat, iso)[2] == 0


def test_contours_many_tiles(lib):
    """3.1 M cells in ~3000 tiles: the look-back chain over many tiles."""
    y, x = np.mgrid[0:1537, 0:2049].astype(np.float32)
    f = (np.sin(x / 37.0) + np.cos(y / 23.0) + 0.05 * np.sin(x * y / 5000.0)).astype(np.float32)
    iso = np.array([-0.2, 0.6], np.float32)
    seg, key, total = lib.lcp_contours(torch.from_numpy(f).cuda(), iso)
    _compare(seg, key, total, *V.marching_squares(f, iso))
    assert lib.lcp_device_status() == 0  # no bounded wait gave up


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_member_contours_spaghetti(lib, dtype):
    d = synth.fourier_ensemble(3, h=61, w=97, m=7, k=2)
    u = torch.from_numpy(d["u"]).cuda().to(dtype)
    v = torch.from_numpy(d["v"]).cuda().to(dtype)
    uf, vf = u.float().cpu().numpy(), v.float().cpu().numpy()
    for dx, dy in ((1.0, 1.0), (0.5, 2.0)):
        seg, key, total = lib.lcp_member_contours(u, v, d["isovalues"], dx, dy)
        _compare(seg, key, total, *V.spaghetti_contours(uf, vf, dx, dy, d["isovalues"]))


def test_mean_field_contours_of_the_divergence(lib):
    """lcp_stats -> lcp_divergence -> lcp_contours against the oracle's own
    mean divergence: identical segment keys on cells whose corners lie clear of
    the isovalue, and points within the propagated rounding of mu_d."""
    d = synth.fourier_ensemble(6, h=97, w=131, m=12, k=3)
    u, v = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()
    mu_d, _ = lib.lcp_divergence(*lib.lcp_stats(u, v))
    seg, key, total = lib.lcp_contours(mu_d, d["isovalues"])
    ref = O.lcp_closed_form(d["u"], d["v"], 1.0, 1.0, d["isovalues"])
    rk, rs = V.marching_squares(ref["mu_d"], d["isovalues"])
    k_iso = len(d["isovalues"])
    mu = ref["mu_d"]
    clear = []
    for c in d["isovalues"]:
        far = np.abs(mu - float(c)) > 1e-3
        clear.append((far[:-1, :-1] & far[:-1, 1:] & far[1:, :-1] & far[1:, 1:]).ravel())

    def keep(keys):
        cell, k = keys // 2 // k_iso, (keys // 2) % k_iso
        return np.array([clear[kk][cc] for cc, kk in zip(cell, k)], bool)

    gk = key.cpu().numpy()
    assert np.array_equal(gk[keep(gk)], rk[keep(rk)])
    gs = seg.cpu().numpy().astype(np.float64)[keep(gk)]
    assert np.max(np.abs(gs - rs[keep(rk)])) < 1e-2


def test_member_contours_latlon_full_sampled(lib):
    """The bench's workload (721 x 1440, 51 fp32 members, 8 isovalues: ~316 M
    segments) in one call; the segments of two members inside interior crops
    against the oracle's spaghetti contours of the crops (cells whose member
    divergences use no crop-edge stencil)."""
    d = synth.fourier_ensemble(0)
    u, v, iso = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda(), d["isovalues"]
    M_, H_, W_ = u.shape
    K_ = len(iso)
    seg, key, total = lib.lcp_member_contours(u, v, iso)
    assert total > 10 ** 8 and bool(torch.all(key[1:] > key[:-1]))
    Hc, Wc = H_ - 1, W_ - 1
    for m, (y0, x0) in ((0, (300, 600)), (37, (10, 1300))):
        y1, x1 = y0 + 24, x0 + 40
        ck, cs = V.spaghetti_contours(d["u"][m:m + 1, y0:y1, x0:x1], d["v"][m:m + 1, y0:y1, x0:x1], 1.0, 1.0, iso)
        # crop cells (il, jl) with 1 <= il <= w-3, 1 <= jl <= h-3 have interior-vertex stencils only
        wc, hc = x1 - x0 - 1, y1 - y0 - 1
        cell = ck // 2 // K_
        jl, il = cell // wc, cell % wc
        keep = (il >= 1) & (il <= wc - 2) & (jl >= 1) & (jl <= hc - 2)
        gkey = (((m * Hc + (y0 + jl)) * Wc + (x0 + il)) * K_ + (ck // 2) % K_) * 2 + ck % 2
        want_k, want_s = gkey[keep], cs[keep] + np.array([x0, y0, x0, y0], np.float64)
        idx = torch.nonzero(torch.isin(key, torch.from_numpy(want_k).cuda())).flatten()
        got_k = key[idx].cpu().numpy()
        assert np.array_equal(got_k, np.sort(want_k))
        got_s = seg[idx].cpu().numpy().astype(np.float64)
        order = np.argsort(want_k)
        assert np.all(np.abs(got_s - want_s[order]) <= _coord_tol(want_s[order]))
    del u, v, seg, key
    torch.cuda.empty_cache()
