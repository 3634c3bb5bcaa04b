"""Visual outputs on the GPU against the oracle: the colour map byte for byte
(reading R17 fixes every fp32 step, so the bytes must be identical)."""

import math

import numpy as np
import pytest
import torch

from oracle import viz as V
from paper_2510_01190_gb300 import synth

pytestmark = pytest.mark.gpu


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
def test_colormap_bit_exact(lib, shape, n_stops):
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
        got = lib.lcp_colormap(xt, vmin, vmax, stops, nan_rgba=nan_c).cpu().numpy()
        want = V.colormap_rgba(x, vmin, vmax, stops, nan_rgba=nan_c)
        assert np.array_equal(got, want), (vmin, vmax)
        got = lib.lcp_colormap(xt, vmin, vmax, stops, nan_rgba=nan_c, mask=words_t, mask_rgba=mask_c).cpu().numpy()
        want = V.colormap_rgba(x, vmin, vmax, stops, nan_rgba=nan_c, mask=bits, mask_rgba=mask_c)
        assert np.array_equal(got, want), (vmin, vmax, "mask")


def test_colormap_unaligned_and_2d(lib):
    """A view that starts one float into its buffer takes the scalar path."""
    g = np.random.Generator(np.random.PCG64(3))
    rows, cols = 45, 67
    buf = torch.from_numpy(_values(g, (rows * cols + 1,))).cuda()
    xt = buf[1:].view(rows, cols)
    assert xt.data_ptr() % 16 != 0
    out = torch.empty(rows * cols * 4 + 4, dtype=torch.uint8, device="cuda")[4:]
    got = lib.lcp_colormap(xt, -2.0, 2.0, lib.DEFAULT_STOPS, out=out).view(rows, cols, 4).cpu().numpy()
    want = V.colormap_rgba(xt.cpu().numpy(), -2.0, 2.0, lib.DEFAULT_STOPS)
    assert np.array_equal(got, want)


def test_colormap_of_an_lcp_map_with_its_contour_mask(lib):
    d = synth.fourier_ensemble(4, h=97, w=131, m=12, k=3)
    u, v = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()
    lcp, mask = lib.lcp_fused(u, v, d["isovalues"], mask=True)
    got = lib.lcp_colormap(lcp, 0.0, 1.0, mask=mask).cpu().numpy()
    bits = lib.unpack_mask(mask, 131).cpu().numpy()
    want = V.colormap_rgba(lcp.cpu().numpy(), 0.0, 1.0, lib.DEFAULT_STOPS, mask=bits, mask_rgba=0xFF000000)
    assert np.array_equal(got, want)
    assert got.shape == (3, 96, 130, 4)


def test_colormap_large_grid_stride(lib):
    """More values than one sweep of the capped grid covers."""
    g = np.random.Generator(np.random.PCG64(11))
    x = g.uniform(-0.1, 1.1, (3, 1531, 1237)).astype(np.float32)
    x[0, 0, 0] = math.nan
    xt = torch.from_numpy(x).cuda()
    got = lib.lcp_colormap(xt, 0.0, 1.0).cpu().numpy()
    want = V.colormap_rgba(x, 0.0, 1.0, lib.DEFAULT_STOPS)
    assert np.array_equal(got, want)


def test_colormap_overflowing_range(lib):
    x = torch.tensor([[np.inf, -np.inf, 1.0, np.nan, 3e38]], dtype=torch.float32, device="cuda")
    got = lib.lcp_colormap(x, -3e38, 3e38, lib.DEFAULT_STOPS, nan_rgba=7).cpu().numpy()
    want = V.colormap_rgba(x.cpu().numpy(), -3e38, 3e38, lib.DEFAULT_STOPS, nan_rgba=7)
    assert np.array_equal(got, want)


def test_colormap_empty(lib):
    x = torch.empty((0, 5, 7), dtype=torch.float32, device="cuda")
    assert lib.lcp_colormap(x).shape == (0, 5, 7, 4)


def test_colormap_full_size_sampled(lib):
    """The bench's map: the 8192^2 eddy field's LCP (4 x 8191^2 fp32) with its
    mask, in the bench's launch; sampled rows of every plane checked byte for
    byte against the oracle on the same fp32 values."""
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
            want = V.colormap_rgba(x, 0.0, 1.0, lib.DEFAULT_STOPS, mask=bits, mask_rgba=0xFF000000)
            assert np.array_equal(rgba[k, r].cpu().numpy(), want), (k, r)
    del lcp, mask, rgba
    torch.cuda.empty_cache()
