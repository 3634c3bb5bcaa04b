"""lcp_fused_static_ws, the entry point that allocates nothing (its scratch is a
fixed device array of the library), called through the C ABI: two calls in a
row must each agree with lcp_fused_ws on its own workspace.  Collected last so
that it also runs after every other test in one process."""

import ctypes

import pytest
import torch

from paper_2510_01190_gb300 import synth

LCP_TOL = 1e-5

CASES = [
    # (h, w, m, k, member dtype)
    (97, 203, 9, 5, torch.float32),
    (64, 130, 12, 3, torch.bfloat16),
    (721, 1440, 51, 8, torch.float32),
    # 600 x 8192: 157 MB of records; the 64 MiB scratch runs 248-row bands
    (600, 8192, 3, 2, torch.float32),
]


def _call_static(clib, u, v, iso, out, mask):
    m, h, w = u.shape
    code = {torch.float32: 0, torch.bfloat16: 1}[u.dtype]
    iso_c = (ctypes.c_float * len(iso))(*[float(c) for c in iso])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return clib.lcp_fused_static_ws(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()), code, m, h, w,
                                    h * w, 1, 1.0, 1.0, iso_c, len(iso), ctypes.c_void_p(out.data_ptr()), 0,
                                    ctypes.c_void_p(mask.data_ptr()), stream)


@pytest.mark.gpu
@pytest.mark.parametrize("h,w,m,k,dt", CASES)
def test_static_scratch_matches_workspace_path_twice(lib, h, w, m, k, dt):
    f = synth.fourier_ensemble(seed=11, h=h, w=w, m=m, k=k)
    u = torch.from_numpy(f["u"]).cuda().to(dt).contiguous()
    v = torch.from_numpy(f["v"]).cuda().to(dt).contiguous()
    iso = f["isovalues"]
    ref, ref_mask = lib.lcp_fused_ws(u, v, iso, 1.0, 1.0, 1, mask=True)
    clib = lib.load()
    nw = lib.mask_words_per_row(w)
    for _ in range(2):
        out = torch.full((k, h - 1, w - 1), float("nan"), device="cuda")
        mask = torch.full((k, h - 1, nw), -1, dtype=torch.int32, device="cuda")
        assert _call_static(clib, u, v, iso, out, mask) == 0, clib.lcp_last_error()
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item()
        assert err <= LCP_TOL, err
        # the same kernels on the same per-vertex records: identical bits, whatever the bands
        assert torch.equal(out, ref)
        assert torch.equal(mask, ref_mask)
    assert lib.lcp_device_status(reset=True) == 0


def test_static_scratch_bands_differ_from_the_workspace_layout():
    """The 600 x 8192 case really runs other bands than lcp_fused_ws with its
    full workspace: 248 rows in the 64 MiB scratch against 376 (host arithmetic
    of the library; no GPU needed)."""
    from paper_2510_01190_gb300 import _binding

    try:
        clib = _binding.load()
    except RuntimeError as e:
        pytest.skip(f"library not buildable here: {e}")
    full = clib.lcp_fused_workspace_bytes(3, 600, 8192, 0)
    assert clib.lcp_fused_band_rows(600, 8192, full) == 376
    assert clib.lcp_fused_band_rows(600, 8192, 64 << 20) == 248
    assert clib.lcp_fused_band_rows(721, 1440, 64 << 20) == 720  # one band


@pytest.mark.gpu
def test_static_scratch_rejects_grids_above_its_maximum(lib):
    clib = lib.load()
    iso_c = (ctypes.c_float * 1)(0.0)
    # 100 x 400000: even the smallest band (8 cell rows + halo) needs about 140 MB
    # of scratch, more than the 64 MiB array (stand-in pointers: nothing is read)
    fake = ctypes.c_void_p(256)
    s = clib.lcp_fused_static_ws(fake, fake, 0, 2, 100, 400000, 100 * 400000, 1, 1.0, 1.0, iso_c, 1, fake, 0, None,
                                 None)
    assert s == -1
    assert b"smallest band" in clib.lcp_last_error()
