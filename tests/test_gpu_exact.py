"""The exact empirical LCP on the GPU (sorted pairwise differences, counted
with two pointers) against the FP64 oracle's meet-in-the-middle judge."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2510_01190_gb300 import synth

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def test_exact_empirical_integer_members_bit_exact(lib):
    """Integer members with dx = dy = 1/2: every pairwise difference and sum is
    an exact fp32 integer, so the counts, hence p, equal the oracle's exactly."""
    g = np.random.Generator(np.random.PCG64(5))
    u = g.integers(-9, 10, size=(7, 9, 11)).astype(np.float32)
    v = g.integers(-9, 10, size=(7, 9, 11)).astype(np.float32)
    iso = np.array([-3.5, 0.0, 2.25, 7.0], np.float32)
    out, below = lib.lcp_exact_empirical(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), iso, 0.5, 0.5)
    for k, c in enumerate(iso):
        ref_p = O.exact_empirical_below(u, v, 0.5, 0.5, float(c))
        assert np.array_equal(_np(below[k, 1:-1, 1:-1]), ref_p.astype(np.float32).astype(np.float64))
    ref = O.exact_empirical_lcp(u, v, 0.5, 0.5, iso)
    got = _np(out)
    assert np.max(np.abs(got[:, 1:-1, 1:-1] - ref)) <= 1e-6
    assert np.isnan(got[:, 0]).all() and np.isnan(got[:, -1]).all() and np.isnan(got[:, :, 0]).all()


@pytest.mark.parametrize("m,dtype", [(20, torch.float32), (50, torch.float32), (12, torch.bfloat16)])
def test_exact_empirical_matches_oracle(lib, m, dtype):
    d = synth.non_gaussian_ensemble(7 + m, h=18, w=23, m=m, k=4)
    u = torch.from_numpy(d["u"]).cuda().to(dtype)
    v = torch.from_numpy(d["v"]).cuda().to(dtype)
    out, _ = lib.lcp_exact_empirical(u, v, d["isovalues"], 1.0, 2.0)
    ref = O.exact_empirical_lcp(_np(u), _np(v), 1.0, 2.0, d["isovalues"])  # the same (bf16-rounded) members
    err = np.abs(_np(out)[:, 1:-1, 1:-1] - ref)
    assert np.max(err) <= 1e-5, float(np.max(err))


def test_empirical_mc_converges_to_gpu_exact(lib):
    d = synth.non_gaussian_ensemble(3, h=40, w=40, m=30, k=4)
    u, v = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()
    exact, _ = lib.lcp_exact_empirical(u, v, d["isovalues"])
    est, _ = lib.lcp_mc(d["isovalues"], 40000, 11, mode="empirical", members=(u, v))
    e = (_np(est) - _np(exact))[:, 1:-1, 1:-1]
    # binomial standard error at S = 4e4 is at most 2.5e-3; 5 SE over ~5800 cells
    assert np.max(np.abs(e)) <= 5 * 0.0025
    assert np.sqrt(np.mean(e * e)) <= 0.0025


def test_exact_empirical_full_size_crop(lib):
    """The bench's judge call (1024^2, 50 fp32 members, 8 isovalues) against the
    oracle's exact LCP of a 12 x 12 crop (cells with interior-vertex stencils)."""
    d = synth.non_gaussian_ensemble(0)
    u, v = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()
    out, _ = lib.lcp_exact_empirical(u, v, d["isovalues"], 1.0, 1.0)
    y0, x0 = 517, 203
    ref = O.exact_empirical_lcp(d["u"][:, y0:y0 + 12, x0:x0 + 12], d["v"][:, y0:y0 + 12, x0:x0 + 12], 1.0, 1.0,
                                d["isovalues"])
    got = _np(out[:, y0 + 1:y0 + 10, x0 + 1:x0 + 10])
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= 1e-5
