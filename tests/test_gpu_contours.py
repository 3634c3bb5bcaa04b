"""Isocontour segments on the GPU against the FP64 oracle (reading R18).

The kernel takes two kinds of decision in fp32 that the oracle takes exactly:
whether a corner value lies below the isovalue, and, in a saddle cell, on
which side the centre value lies.  Guard bands (unit roundoff u = 2^-24):

* a field given as fp32 values (mean-field contours): the corner decisions are
  exact on both sides; the kernel's centre ((f0 + f1) + (f2 + f3)) * 0.25 is
  within 3u (|f0| + |f1| + |f2| + |f3|) / 4 of the exact one;
* member divergences (spaghetti plots): the kernel forms
  (u[i+] - u[i-]) sx + (v[j+] - v[j-]) sy with sx, sy rounded once, so each
  corner value is within 5u (|gx| + |gy|) of Eq. 1 in FP64 (gx, gy its two
  terms), and the centre within the mean of its corners' bounds plus the
  rounding above.

Outside the guard bands the segment keys are identical.  A saddle cell whose
centre lies inside its band has the same two keys either way, and the same
four crossing points paired one way or the other.  A cell-isovalue with a
corner inside its band is excluded from the key comparison and may hold at
most two segments.  Crossing points: the kernel divides with the approximate
division (2 ulp) and rounds the subtraction and the add, so a point is within
1e-6 + 4 fp32 ulps of the oracle's plus (d_a + d_b) / |f_b - f_a| from the
corner bounds d_a, d_b of its edge."""

import numpy as np
import pytest
import torch

import oracle as O
from oracle import viz as V
from paper_2510_01190_gb300 import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _coord_tol(segs):
    return 1e-6 + 4.0 * 2.0 ** -23 * np.maximum(np.abs(segs), 1.0)


def _member_bounds(u, v, dx, dy):
    """FP64 divergence of every member (Eq. 1) and the bound on the kernel's
    fp32 evaluation of it, 5u (|gx| + |gy|)."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    f = O.divergence_of_field(u, v, dx, dy)
    _, h, w = u.shape
    i = np.arange(w)
    il, ih = np.maximum(i - 1, 0), np.minimum(i + 1, w - 1)
    j = np.arange(h)
    jl, jh = np.maximum(j - 1, 0), np.minimum(j + 1, h - 1)
    gx = np.abs(u[:, :, ih] - u[:, :, il]) / ((ih - il) * dx)[None, None, :]
    gy = np.abs(v[:, jh, :] - v[:, jl, :]) / ((jh - jl) * dy)[None, :, None]
    return f, 5.0 * U32 * (gx + gy)


def _check_field(f, d, iso, got_k, got_s, min_clear=0.9, origin=(0.0, 0.0)):
    """Segments of one field f [H, W] (FP64) with corner bounds d [H, W]
    against the oracle's, per the guard bands above.  got_k: local keys;
    origin: the grid coordinates (x, y) of f's first vertex, whose magnitude
    sets the fp32 rounding of the kernel's coordinates."""
    org = np.array([origin[0], origin[1], origin[0], origin[1]], np.float64)
    iso = np.asarray(iso, np.float64)
    K = iso.size
    h, w = f.shape
    ref_k, ref_s = V.marching_squares(f, iso)
    f0, f1, f3, f2 = f[:-1, :-1], f[:-1, 1:], f[1:, :-1], f[1:, 1:]
    d0, d1, d3, d2 = d[:-1, :-1], d[:-1, 1:], d[1:, :-1], d[1:, 1:]
    with np.errstate(invalid="ignore"):
        cen = (f0 + f1 + f2 + f3) / 4.0
        dcen = (d0 + d1 + d2 + d3) / 4.0 + 3.0 * U32 * (np.abs(f0) + np.abs(f1) + np.abs(f2) + np.abs(f3)) / 4.0
    corner = np.zeros((K, h - 1, w - 1), bool)   # a corner decision may flip
    saddle = np.zeros((K, h - 1, w - 1), bool)   # only the saddle pairing may flip
    etol = np.zeros((K, h - 1, w - 1))           # coordinate bound from the corner values
    with np.errstate(invalid="ignore", divide="ignore"):
        for k, c in enumerate(iso):
            a = np.abs(f - c) <= d
            corner[k] = a[:-1, :-1] | a[:-1, 1:] | a[1:, :-1] | a[1:, 1:]
            b0, b1, b2, b3 = f0 < c, f1 < c, f2 < c, f3 < c
            sad = (b0 == b2) & (b1 == b3) & (b0 != b1)
            saddle[k] = sad & (np.abs(cen - c) <= dcen) & ~corner[k]
            t = np.zeros((h - 1, w - 1))
            for (fa, da), (fb, db), cr in (((f0, d0), (f1, d1), b0 != b1), ((f1, d1), (f2, d2), b1 != b2),
                                           ((f3, d3), (f2, d2), b3 != b2), ((f0, d0), (f3, d3), b0 != b3)):
                t = np.where(cr, np.maximum(t, (da + db) / np.abs(fb - fa)), t)
            etol[k] = np.nan_to_num(t, nan=0.0)

    def flags(keys):
        cell, k = (keys // 2) // K, (keys // 2) % K
        return corner.reshape(K, -1)[k, cell], saddle.reshape(K, -1)[k, cell], etol.reshape(K, -1)[k, cell]

    rc, rsad, _ = flags(ref_k)
    gc, gsad, gtol = flags(got_k)
    # keys: identical wherever no corner decision can flip
    assert np.array_equal(got_k[~gc], ref_k[~rc])
    # cells with an uncertain corner: at most two segments per cell and isovalue
    if np.any(gc):
        _, counts = np.unique(got_k[gc] // 2, return_counts=True)
        assert counts.max() <= 2
    # points of unambiguous cells
    sel_g, sel_r = ~gc & ~gsad, ~rc & ~rsad
    tol = _coord_tol(ref_s[sel_r] + org) + gtol[sel_g][:, None]
    assert np.all(np.abs(got_s[sel_g] - ref_s[sel_r]) <= tol)
    # uncertain saddles: the same four crossing points, paired either way
    for key in np.unique(got_k[gsad] // 2):
        g_pts = np.sort(got_s[got_k // 2 == key].reshape(-1, 2), axis=0)
        r_pts = np.sort(ref_s[ref_k // 2 == key].reshape(-1, 2), axis=0)
        assert np.all(np.abs(g_pts - r_pts) <= _coord_tol(r_pts + org[:2]) + flags(np.array([key * 2]))[2][0])
    n_cells = max(1, K * (h - 1) * (w - 1))
    assert 1.0 - np.count_nonzero(corner) / n_cells >= min_clear


def _compare(seg, key, total, f, d, iso):
    assert total == key.shape[0]
    _check_field(np.asarray(f, np.float64), d, iso, key.cpu().numpy(), seg.cpu().numpy().astype(np.float64))


def _compare_members(seg, key, total, u, v, dx, dy, iso):
    """Spaghetti contours of members u, v [M, H, W] member by member."""
    f, d = _member_bounds(u, v, dx, dy)
    m, h, w = f.shape
    K = len(iso)
    per = (h - 1) * (w - 1) * K * 2
    keys = key.cpu().numpy()
    segs = seg.cpu().numpy().astype(np.float64)
    assert total == keys.size and np.all(np.diff(keys) > 0)
    for mm in range(m):
        sel = (keys // per) == mm
        _check_field(f[mm], d[mm], iso, keys[sel] - mm * per, segs[sel])


@pytest.mark.parametrize("h,w,k", [(17, 19, 3), (2, 2, 1), (33, 1100, 2), (300, 257, 4)])
def test_contours_random_fields(lib, h, w, k):
    g = np.random.Generator(np.random.PCG64(h * w + k))
    f = g.normal(0, 1, (h, w)).astype(np.float32)
    f[::7, ::5] = 0.25  # exact ties with an isovalue: not below
    iso = np.array([-0.7, 0.0, 0.25, 1.1][:k], np.float32)
    seg, key, total = lib.lcp_contours(torch.from_numpy(f).cuda(), iso)
    _compare(seg, key, total, f, np.zeros(f.shape), iso)


def test_contours_forty_isovalues_take_the_wide_masks(lib):
    g = np.random.Generator(np.random.PCG64(40))
    f = g.normal(0, 1, (45, 77)).astype(np.float32)
    iso = np.linspace(-2.0, 2.0, 40).astype(np.float32)[g.permutation(40)]  # unsorted on purpose
    seg, key, total = lib.lcp_contours(torch.from_numpy(f).cuda(), iso)
    _compare(seg, key, total, f, np.zeros(f.shape), iso)
    u = torch.from_numpy(g.normal(0, 1, (3, 20, 33)).astype(np.float32)).cuda()
    v = torch.from_numpy(g.normal(0, 1, (3, 20, 33)).astype(np.float32)).cuda()
    seg, key, total = lib.lcp_member_contours(u, v, iso[:35])
    _compare_members(seg, key, total, u.cpu().numpy(), v.cpu().numpy(), 1.0, 1.0, iso[:35])


def test_contours_smooth_field_closed_loops_and_nan(lib):
    y, x = np.mgrid[0:90, 0:130].astype(np.float64)
    f = (np.sin(x / 9.0) * np.cos(y / 7.0) + 0.1 * np.sin(x / 3.1 + y / 4.3)).astype(np.float32)
    f[40:43, 60:62] = np.nan
    iso = np.array([-0.5, 0.0, 0.3], np.float32)
    seg, key, total = lib.lcp_contours(torch.from_numpy(f).cuda(), iso)
    _compare(seg, key, total, f, np.zeros(f.shape), iso)


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
    _compare(seg, key, total, f, np.zeros(f.shape), iso)
    assert lib.lcp_device_status() == 0  # no bounded wait gave up


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_member_contours_spaghetti(lib, dtype):
    d = synth.fourier_ensemble(3, h=61, w=97, m=7, k=2)
    u = torch.from_numpy(d["u"]).cuda().to(dtype)
    v = torch.from_numpy(d["v"]).cuda().to(dtype)
    uf, vf = u.float().cpu().numpy(), v.float().cpu().numpy()
    for dx, dy in ((1.0, 1.0), (0.5, 2.0)):
        seg, key, total = lib.lcp_member_contours(u, v, d["isovalues"], dx, dy)
        _compare_members(seg, key, total, uf, vf, dx, dy, d["isovalues"])


def test_mean_field_contours_of_the_divergence(lib):
    """lcp_stats -> lcp_divergence -> lcp_contours against the oracle's own
    mean divergence.  Each fp32 mean is x0 + S1 / M with S1 a recursive sum of
    M - 1 differences |x - x0| <= 2 max|x|, so it is within (2M + 3) u max|x|
    of the exact mean; the stencil takes two such differences (u and v) and
    rounds three times more, so mu_d is within (4M + 12) u max(|u|, |v|) /
    min(dx, dy) of the FP64 value, which serves as every corner's bound."""
    d = synth.fourier_ensemble(6, h=97, w=131, m=12, k=3)
    u, v = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()
    mu_d, _ = lib.lcp_divergence(*lib.lcp_stats(u, v))
    seg, key, total = lib.lcp_contours(mu_d, d["isovalues"])
    ref = O.lcp_closed_form(d["u"], d["v"], 1.0, 1.0, d["isovalues"])
    m = d["u"].shape[0]
    bound = (4 * m + 12) * U32 * max(np.abs(d["u"]).max(), np.abs(d["v"]).max())
    assert np.max(np.abs(mu_d.cpu().numpy() - ref["mu_d"])) <= bound
    _compare(seg, key, total, ref["mu_d"], np.full(ref["mu_d"].shape, bound), d["isovalues"])


def test_member_contours_latlon_full_sampled(lib):
    """The bench's workload (721 x 1440, 51 fp32 members, 8 isovalues: ~316 M
    segments) in one call; the segments of two members inside interior crops
    against the oracle's contours of those members' FP64 Eq. 1 divergence
    (computed on the crop plus a one-vertex margin, so every stencil is the
    full grid's)."""
    d = synth.fourier_ensemble(0)
    u, v, iso = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda(), d["isovalues"]
    M_, H_, W_ = u.shape
    K_ = len(iso)
    seg, key, total = lib.lcp_member_contours(u, v, iso)
    assert total > 10 ** 8 and bool(torch.all(key[1:] > key[:-1]))
    Hc, Wc = H_ - 1, W_ - 1
    per = Hc * Wc * K_ * 2
    for m, (y0, x0) in ((0, (300, 600)), (37, (10, 1300))):
        hh, ww = 24, 40
        f, db = _member_bounds(d["u"][m:m + 1, y0 - 1:y0 + hh + 1, x0 - 1:x0 + ww + 1],
                               d["v"][m:m + 1, y0 - 1:y0 + hh + 1, x0 - 1:x0 + ww + 1], 1.0, 1.0)
        f, db = f[0, 1:-1, 1:-1], db[0, 1:-1, 1:-1]
        mk = key // per
        rem = key - mk * per
        cell = rem // (2 * K_)
        jj, ii = cell // Wc, cell % Wc
        sel = (mk == m) & (jj >= y0) & (jj < y0 + hh - 1) & (ii >= x0) & (ii < x0 + ww - 1)
        ks, ss = key[sel], seg[sel]
        cell_s = (ks - m * per) // (2 * K_)
        lk = ((((cell_s // Wc) - y0) * (ww - 1) + (cell_s % Wc) - x0) * K_ + ((ks // 2) % K_)) * 2 + ks % 2
        got_k = lk.cpu().numpy()
        got_s = ss.cpu().numpy().astype(np.float64) - np.array([x0, y0, x0, y0], np.float64)
        assert np.all(np.diff(got_k) > 0)
        _check_field(f, db, iso, got_k, got_s, origin=(x0, y0))
        del mk, rem, cell, jj, ii, sel
    del u, v, seg, key
    torch.cuda.empty_cache()
