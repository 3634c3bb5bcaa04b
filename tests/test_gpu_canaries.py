"""Guard canaries around outputs (the stand-in for a memory sanitizer, which is
not available here): every output is a view into a larger buffer whose margins
before and after hold a fixed bit pattern, on small odd shapes (2 x 2, 3 x 17,
one member, widths that end mid mask word); after the call the margins must be
unchanged bit for bit, so no kernel writes outside the output it was given."""

import math

import numpy as np
import pytest
import torch

from paper_2510_01190_gb300 import synth

pytestmark = pytest.mark.gpu

PAD = 96  # elements of canary on each side (more than any vector store or mask word)
_PATTERN = {torch.float32: (torch.int32, 0x7FC0DEAD), torch.int32: (torch.int32, 0x5A5AA5A5),
            torch.float16: (torch.int16, 0x7E5A), torch.uint8: (torch.uint8, 0xA5)}


class Guarded:
    """A contiguous output view of `shape` inside a buffer with canary margins."""

    def __init__(self, shape, dtype):
        self.n = math.prod(shape)
        raw_t, bits = _PATTERN[dtype]
        if raw_t == torch.uint8:
            raw = torch.full((self.n + 2 * PAD,), bits, dtype=torch.uint8, device="cuda")
        else:
            signed = bits - (1 << (8 * torch.tensor([], dtype=raw_t).element_size())) \
                if bits >= 1 << (8 * torch.tensor([], dtype=raw_t).element_size() - 1) else bits
            raw = torch.full((self.n + 2 * PAD,), signed, dtype=raw_t, device="cuda")
        self.raw = raw
        self.ref = raw[:PAD].clone()
        self.view = raw.view(dtype)[PAD:PAD + self.n].view(shape)

    def intact(self):
        torch.cuda.synchronize()
        return torch.equal(self.raw[:PAD], self.ref) and torch.equal(self.raw[PAD + self.n:], self.ref)


def _fields(h, w, m, seed, k=3):
    d = synth.fourier_ensemble(seed=seed, h=h, w=w, m=m, k=k)
    return (torch.from_numpy(d["u"]).cuda().contiguous(), torch.from_numpy(d["v"]).cuda().contiguous(),
            list(d["isovalues"]))


SHAPES = [(2, 2, 2), (3, 17, 5), (2, 33, 1), (17, 3, 4), (9, 65, 3), (40, 97, 7)]


@pytest.mark.parametrize("h,w,m", SHAPES)
def test_fused_paths_write_only_their_outputs(lib, h, w, m):
    u, v, iso = _fields(h, w, m, seed=h * 31 + w)
    k, nw = len(iso), lib.mask_words_per_row(w)
    ddof = 0 if m == 1 else 1
    for entry in ("lcp_fused_ws", "lcp_fused", "lcp_fused_static_ws"):
        for dt in (torch.float32, torch.float16):
            g = Guarded((k, h - 1, w - 1), dt)
            gm = Guarded((k, h - 1, nw), torch.int32)
            getattr(lib, entry)(u, v, iso, 1.0, 1.0, ddof, out_dtype=dt, mask=True, out=g.view, mask_out=gm.view)
            assert g.intact() and gm.intact(), (entry, dt)
            assert torch.isfinite(g.view.float()).all(), (entry, dt)


def test_fused_ws_bands_write_only_their_outputs(lib):
    """Several row bands (a small workspace), bf16 members."""
    h, w, m = 70, 131, 6
    u, v, iso = _fields(h, w, m, seed=5)
    u16, v16 = u.to(torch.bfloat16), v.to(torch.bfloat16)
    k, nw = len(iso), lib.mask_words_per_row(w)
    ws = torch.empty(2 * w * 16 * 20 + 2048, dtype=torch.uint8, device="cuda")
    ws = ws[(256 - ws.data_ptr() % 256) % 256:]
    assert lib.lcp_fused_band_rows(h, w, ws.numel()) < h - 1
    g = Guarded((k, h - 1, w - 1), torch.float32)
    gm = Guarded((k, h - 1, nw), torch.int32)
    lib.lcp_fused_ws(u16, v16, iso, mask=True, out=g.view, mask_out=gm.view, workspace=ws)
    assert g.intact() and gm.intact()


@pytest.mark.parametrize("h,w,m", SHAPES)
def test_unfused_calls_write_only_their_outputs(lib, h, w, m):
    u, v, iso = _fields(h, w, m, seed=h + 7 * w)
    ddof = 0 if m == 1 else 1
    gs = [Guarded((h, w), torch.float32) for _ in range(4)]
    mu_u, var_u, mu_v, var_v = lib.lcp_stats(u, v, ddof, out=tuple(x.view for x in gs))
    assert all(x.intact() for x in gs)
    mu_d, var_d = lib.lcp_divergence(mu_u, var_u, mu_v, var_v)
    k, nw = len(iso), lib.mask_words_per_row(w)
    g = Guarded((k, h - 1, w - 1), torch.float32)
    gm = Guarded((k, h - 1, nw), torch.int32)
    lib.lcp_map(mu_d, var_d, iso, mask=True, out=g.view, mask_out=gm.view)
    assert g.intact() and gm.intact()


@pytest.mark.parametrize("h,w,m", [(3, 18, 4), (10, 64, 5), (33, 130, 3)])
def test_speed_gradient_writes_only_its_outputs(lib, h, w, m):
    u, v, iso = _fields(h, w, m, seed=3 * h + w)
    k, nw = len(iso), lib.mask_words_per_row(w)
    g = Guarded((k, h - 1, w - 1), torch.float32)
    gm = Guarded((k, h - 1, nw), torch.int32)
    lib.lcp_speed_gradient_ws(u, v, iso, mask=True, out=g.view, mask_out=gm.view)
    assert g.intact() and gm.intact()


def test_volume_writes_only_its_outputs(lib):
    rng = np.random.default_rng(3)
    m, d, h, w = 3, 5, 6, 37
    u, v, ww = (torch.from_numpy(rng.standard_normal((m, d, h, w)).astype(np.float32)).cuda() for _ in range(3))
    iso = [-0.2, 0.1]
    nw = lib.mask_words_per_row(w)
    g = Guarded((2, d - 1, h - 1, w - 1), torch.float32)
    gm = Guarded((2, d - 1, h - 1, nw), torch.int32)
    lib.lcp3d_fused_ws(u, v, ww, iso, mask=True, out=g.view, mask_out=gm.view)
    assert g.intact() and gm.intact()


def test_colormap_and_exact_write_only_their_outputs(lib):
    rng = np.random.default_rng(4)
    vals = torch.from_numpy(rng.random((2, 5, 37), dtype=np.float32)).cuda()
    g = Guarded((2, 5, 37, 4), torch.uint8)
    lib.lcp_colormap(vals, out=g.view)
    assert g.intact()
    u, v, iso = _fields(7, 11, 5, seed=9)
    ge = Guarded((len(iso), 6, 10), torch.float32)
    lib.lcp_exact_empirical(u, v, iso, out=ge.view)
    assert ge.intact()
