"""Visual outputs on the GPU against the FP64 oracle: the colour map byte for
byte outside the guard band where fp32 rounding can move a value across a
byte boundary (reading R17).

Guard band.  The kernel forms t = (x - vmin) R with R = 1 / (vmax - vmin)
rounded once, f = (t - t_s) r_s with r_s = 1 / (t_{s+1} - t_s) rounded once,
ch = c_s + f d_s and y = 255 ch + 1/2, each step one fp32 operation rounded to
nearest (unit roundoff u = 2^-24).  Then |t32 - t| <= 4u on [0, 1] (two
roundings in R, one in x - vmin, one in the product), |f32 - f| <= 4u r_s + 4u,
|ch32 - ch| <= |d_s| (4u r_s + 6u) + 2u and |y32 - y| <= 255 |ch32 - ch| + 512u
(the products by 255 and the add of 1/2 at magnitudes below 256).  Where t
lies within 8u of an interior stop the kernel may take the neighbouring
segment; the colour is continuous there, so the same bound holds with the
larger |d| r of the two segments.  A byte can differ from floor(y) only where
y lies within that bound of an integer, and then by one."""

import math

import numpy as np
import pytest
import torch

from oracle import viz as V
from paper_2510_01190_gb300 import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _f32(x):
    return float(np.float32(x))


def _guard(x, vmin, vmax, stops):
    """Per value and channel: True where fp32 rounding may change the byte."""
    st = np.asarray(stops, np.float64).reshape(-1, 5)
    y, s = V.colormap_levels(x, vmin, vmax, st)
    w = st[1:, 0] - st[:-1, 0]
    dr = np.abs(st[1:, 1:] - st[:-1, 1:]) / w[:, None]       # |d_s| r_s per segment and channel
    d = np.abs(st[1:, 1:] - st[:-1, 1:])
    drs, ds = dr[s], d[s]
    with np.errstate(invalid="ignore"):
        t = np.clip((np.asarray(x, np.float64) - vmin) / (vmax - vmin), 0.0, 1.0)
    for q in range(1, st.shape[0] - 1):                      # near an interior stop: either segment
        near = np.abs(t - st[q, 0]) <= 8 * U32
        drs = np.where(near[..., None], np.maximum(drs, np.maximum(dr[q - 1], dr[q])), drs)
        ds = np.where(near[..., None], np.maximum(ds, np.maximum(d[q - 1], d[q])), ds)
    eps = U32 * (255.0 * (4.0 * drs + 6.0 * ds + 2.0) + 512.0)
    with np.errstate(invalid="ignore"):
        dist = np.abs(y - np.round(y))
    return dist <= eps


def _assert_bytes(got, x, vmin, vmax, stops, max_diff_frac=1e-3, **kw):
    """Equal bytes outside the guard band, at most one apart inside it, and
    differing bytes rare (fp32 rounding moves a level across an integer only
    where it lies within a few ulps of it)."""
    want = V.colormap_rgba(x, vmin, vmax, stops, **kw)
    amb = _guard(x, vmin, vmax, stops)
    painted = np.isnan(np.asarray(x, np.float64))
    if kw.get("mask") is not None:
        painted = painted | np.asarray(kw["mask"], bool)
    amb = amb & ~painted[..., None]                      # NaN and mask colours are exact
    diff = np.abs(got.astype(np.int32) - want.astype(np.int32))
    assert np.all(diff[~amb] == 0), int(np.count_nonzero(diff[~amb]))
    assert np.all(diff[amb] <= 1)
    n_diff = int(np.count_nonzero(diff))
    assert n_diff <= max(1, max_diff_frac * diff.size), (n_diff, diff.size)
    return n_diff


def _random_stops(g, n):
    t = np.concatenate([[0.0], np.sort(g.uniform(0.02, 0.98, n - 2)), [1.0]]).astype(np.float32)
    while np.any(np.diff(t) <= 0):
        t = np.concatenate([[0.0], np.sort(g.uniform(0.02, 0.98, n - 2)), [1.0]]).astype(np.float32)
    c = g.uniform(0.0, 1.0, (n, 4)).astype(np.float32)
    return np.concatenate([t[:, None], c], axis=1)


def _values(g, shape):
    x = g.normal(0.3, 1.2, shape).astype(np.float32)
    flat = x.reshape(-1)
    idx = g.choice(flat.size, size=max(4, flat.size // 50), replace=False)
    flat[idx[0::4]] = np.nan
    flat[idx[1::4]] = np.inf
    flat[idx[2::4]] = -np.inf
    flat[idx[3::4]] = 0.3  # exactly on a stop-range boundary for some tables
    return x


@pytest.mark.parametrize("shape,n_stops", [((3, 37, 41), 7), ((1, 5, 3), 2), ((2, 129, 257), 16), ((4, 33, 32), 3)])
def test_colormap_bytes_against_the_fp64_oracle(lib, shape, n_stops):
    g = np.random.Generator(np.random.PCG64(sum(shape) + n_stops))
    x = _values(g, shape)
    stops = _random_stops(g, n_stops)
    planes, rows, cols = shape
    nw = (cols + 31) // 32
    words = g.integers(0, 2**32, size=(planes, rows, nw), dtype=np.uint64).astype(np.uint32).view(np.int32)
    words_t = torch.from_numpy(words.copy()).cuda()
    bits = lib.unpack_mask(words_t, cols + 1).cpu().numpy()
    nan_c, mask_c = V.pack_rgba(9, 8, 7, 6), V.pack_rgba(0, 255, 255, 255)
    xt = torch.from_numpy(x).cuda()
    for vmin, vmax in ((-1.5, 2.5), (0.0, 1.0), (-3e-3, 7e-3)):
        lo, hi = _f32(vmin), _f32(vmax)  # the fp32 range the kernel receives
        got = lib.lcp_colormap(xt, vmin, vmax, stops, nan_rgba=nan_c).cpu().numpy()
        _assert_bytes(got, x, lo, hi, stops, nan_rgba=nan_c)
        got = lib.lcp_colormap(xt, vmin, vmax, stops, nan_rgba=nan_c, mask=words_t, mask_rgba=mask_c).cpu().numpy()
        _assert_bytes(got, x, lo, hi, stops, nan_rgba=nan_c, mask=bits, mask_rgba=mask_c)


def test_colormap_unaligned_and_2d(lib):
    """A view that starts one float into its buffer takes the scalar path."""
    g = np.random.Generator(np.random.PCG64(3))
    rows, cols = 45, 67
    buf = torch.from_numpy(_values(g, (rows * cols + 1,))).cuda()
    xt = buf[1:].view(rows, cols)
    assert xt.data_ptr() % 16 != 0
    out = torch.empty(rows * cols * 4 + 4, dtype=torch.uint8, device="cuda")[4:]
    got = lib.lcp_colormap(xt, -2.0, 2.0, lib.DEFAULT_STOPS, out=out).view(rows, cols, 4).cpu().numpy()
    _assert_bytes(got, xt.cpu().numpy(), -2.0, 2.0, lib.DEFAULT_STOPS)


def test_colormap_of_an_lcp_map_with_its_contour_mask(lib):
    d = synth.fourier_ensemble(4, h=97, w=131, m=12, k=3)
    u, v = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()
    lcp, mask = lib.lcp_fused(u, v, d["isovalues"], mask=True)
    got = lib.lcp_colormap(lcp, 0.0, 1.0, mask=mask).cpu().numpy()
    bits = lib.unpack_mask(mask, 131).cpu().numpy()
    _assert_bytes(got, lcp.cpu().numpy(), 0.0, 1.0, lib.DEFAULT_STOPS, mask=bits, mask_rgba=0xFF000000)
    assert got.shape == (3, 96, 130, 4)


def test_colormap_large_grid_stride(lib):
    """More values than one sweep of the capped grid covers."""
    g = np.random.Generator(np.random.PCG64(11))
    x = g.uniform(-0.1, 1.1, (3, 1531, 1237)).astype(np.float32)
    x[0, 0, 0] = math.nan
    xt = torch.from_numpy(x).cuda()
    got = lib.lcp_colormap(xt, 0.0, 1.0).cpu().numpy()
    _assert_bytes(got, x, 0.0, 1.0, lib.DEFAULT_STOPS)


def test_colormap_dyadic_values_are_exact(lib):
    """Values k/256 on the range [0, 1] with a two-stop grey ramp: every fp32
    step is exact, so every byte equals floor((255 k + 128) / 256)."""
    k = np.arange(257)
    x = torch.from_numpy((k / 256.0).astype(np.float32)).reshape(1, 257).cuda()
    grey = [(0.0, 0.0, 0.0, 0.0, 0.0), (1.0, 1.0, 1.0, 1.0, 1.0)]
    got = lib.lcp_colormap(x, 0.0, 1.0, grey).cpu().numpy()[0]
    want = ((255 * k + 128) // 256).astype(np.uint8)
    for ch in range(4):
        assert np.array_equal(got[:, ch], want)


def test_colormap_infinities_and_a_range_that_overflows_fp32(lib):
    x = torch.tensor([[np.inf, -np.inf, 1.0, np.nan, 3e38]], dtype=torch.float32, device="cuda")
    got = lib.lcp_colormap(x, -1.0, 2.0, lib.DEFAULT_STOPS, nan_rgba=7).cpu().numpy()
    _assert_bytes(got, x.cpu().numpy(), -1.0, 2.0, lib.DEFAULT_STOPS, nan_rgba=7)
    # vmax - vmin beyond the fp32 range: the kernel cannot form 1 / (vmax - vmin), the call is refused
    with pytest.raises(RuntimeError):
        lib.lcp_colormap(x, -3e38, 3e38, lib.DEFAULT_STOPS)


def test_colormap_empty(lib):
    x = torch.empty((0, 5, 7), dtype=torch.float32, device="cuda")
    assert lib.lcp_colormap(x).shape == (0, 5, 7, 4)


def test_colormap_full_size_sampled(lib):
    """The bench's map: the 8192^2 eddy field's LCP (4 x 8191^2 fp32) with its
    mask, in the bench's launch; sampled rows of every plane checked byte for
    byte (outside the guard band) against the oracle on the same fp32 values."""
    if torch.cuda.get_device_properties(0).total_memory < 60e9:
        pytest.skip("needs the full-size device memory")
    d = synth.eddy_ensemble_torch(0)
    lcp, mask = lib.lcp_fused_ws(d["u"], d["v"], d["isovalues"], mask=True)
    del d
    torch.cuda.empty_cache()
    rgba = lib.lcp_colormap(lcp, 0.0, 1.0, mask=mask)
    K, Hc, Wc = lcp.shape
    for k in range(K):
        for r in (0, 1, 4095, Hc - 1):
            x = lcp[k, r].cpu().numpy()
            bits = lib.unpack_mask(mask[k:k + 1, r:r + 1], Wc + 1)[0, 0].cpu().numpy()
            _assert_bytes(rgba[k, r].cpu().numpy(), x, 0.0, 1.0, lib.DEFAULT_STOPS, mask=bits, mask_rgba=0xFF000000)
    del lcp, mask, rgba
    torch.cuda.empty_cache()
