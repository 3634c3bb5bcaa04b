"""Failure detection on the GPU without a fault: each probe launches one of the
library's waiting kernels against a flag that nothing sets, with a wait budget
of about a millisecond, and checks that the kernel gives up, reports it in the
device status word, leaves its outputs recognisably invalid, and that the next
ordinary call on the same context is correct and clean."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2510_01190_gb300 import synth

pytestmark = pytest.mark.gpu

BUDGET = 2_000_000  # clock cycles, ~1 ms at 2 GHz


class _budget:
    def __init__(self, lib, cycles):
        self.lib, self.cycles = lib, cycles

    def __enter__(self):
        self.prev = self.lib.lcp_set_wait_budget(self.cycles)

    def __exit__(self, *exc):
        self.lib.lcp_set_wait_budget(0)


def test_wait_budget_setter_round_trips(lib):
    default = lib.lcp_set_wait_budget(0)
    assert default == 4_000_000_000
    assert lib.lcp_set_wait_budget(12345) == default
    assert lib.lcp_set_wait_budget(0) == 12345
    assert lib.lcp_set_wait_budget(0) == default


@pytest.mark.parametrize("k", [3, 8, 20])
def test_stalled_lcp_wait_gives_up_and_leaves_nan(lib, k):
    """The LCP kernels (the warp kernel for K <= 8 in passes 2 + 1 and 8, the
    shared-memory kernel for 20 = 16 + 4) wait on statistics counters no
    statistics grid will release."""
    h, w = 97, 131
    iso = np.linspace(-0.5, 0.5, k).astype(np.float32)
    assert lib.lcp_device_status(reset=True) == 0
    out = torch.zeros((k, h - 1, w - 1), dtype=torch.float32, device="cuda")
    nw = lib.mask_words_per_row(w)
    mask = torch.full((k, h - 1, nw), -1, dtype=torch.int32, device="cuda")
    with _budget(lib, BUDGET):
        lib.lcp_test_stalled_lcp_wait(h, w, iso, out, mask)
        torch.cuda.synchronize()
    flags = lib.lcp_device_status(reset=True)
    assert flags & 1, flags
    assert bool(torch.isnan(out).all())
    assert bool((mask == 0).all())
    # the context is intact and the status clean for the next ordinary call
    d = synth.fourier_ensemble(7, h=h, w=w, m=9, k=k)
    u, v = torch.from_numpy(d["u"]).cuda(), torch.from_numpy(d["v"]).cuda()
    lcp, _ = lib.lcp_fused_ws(u, v, d["isovalues"])
    ref = O.lcp_closed_form(d["u"], d["v"], 1.0, 1.0, d["isovalues"])["lcp"]
    assert np.max(np.abs(lcp.cpu().numpy() - ref)) <= 1e-5
    assert lib.lcp_device_status() == 0


def test_stalled_lcp_wait_fp16_output(lib):
    h, w, k = 40, 300, 4
    out = torch.zeros((k, h - 1, w - 1), dtype=torch.float16, device="cuda")
    with _budget(lib, BUDGET):
        lib.lcp_test_stalled_lcp_wait(h, w, [0.0, 0.1, 0.2, 0.3], out)
        torch.cuda.synchronize()
    assert lib.lcp_device_status(reset=True) & 1
    assert bool(torch.isnan(out).all())


def test_stalled_lookback_gives_up_and_the_next_call_is_clean(lib):
    """Tile 0 of the contour compaction never runs, so the tile after it waits
    for a look-back flag nothing writes; it gives up, counts tile 0 as empty
    and sets bit 2.  Every segment outside tile 0's cells is still produced,
    in key order, shifted down by tile 0's count."""
    g = np.random.Generator(np.random.PCG64(17))
    f = torch.from_numpy(g.normal(0, 1, (120, 150)).astype(np.float32)).cuda()
    iso = [0.0, 0.4]
    assert lib.lcp_device_status(reset=True) == 0
    seg_ok, key_ok, total_ok = lib.lcp_contours(f, iso)
    assert lib.lcp_device_status() == 0
    tile_items = 8 * 4 * 31  # cells per tile of the compaction kernel
    in_tile0 = (key_ok // 2 // len(iso)) < tile_items
    with _budget(lib, BUDGET):
        seg, key, total = lib.lcp_test_stalled_lookback(f, iso, capacity=total_ok)
        torch.cuda.synchronize()
    flags = lib.lcp_device_status(reset=True)
    assert flags & 4, flags
    n_rest = int((~in_tile0).sum())
    assert total == n_rest
    assert torch.equal(key[:n_rest], key_ok[~in_tile0])
    assert torch.equal(seg[:n_rest], seg_ok[~in_tile0])
    seg2, key2, total2 = lib.lcp_contours(f, iso)
    assert total2 == total_ok and torch.equal(key2, key_ok) and torch.equal(seg2, seg_ok)
    assert lib.lcp_device_status() == 0
