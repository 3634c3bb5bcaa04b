"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every symbol declared in include/lcp.h, and rejects bad arguments on the host
(before any CUDA call, so these run without a GPU).  Also checks that the
product package never reaches the oracle."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lcp.h")

FAKE = ctypes.c_void_p(256)  # never dereferenced: validation fails first


@pytest.fixture(scope="module")
def clib():
    from paper_2510_01190_gb300 import _binding

    try:
        return _binding.load()
    except RuntimeError as e:  # no nvcc at all: nothing to check
        pytest.skip(f"library not buildable here: {e}")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lcp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_hot_path_entry_points():
    names = declared_functions()
    for want in ("lcp_stats", "lcp_divergence", "lcp_map", "lcp_fused", "lcp_mc"):
        assert want in names


def test_every_declared_symbol_is_exported(clib):
    for name in declared_functions():
        assert hasattr(clib, name), name


def test_status_strings_and_version(clib):
    for code in (0, -1, -2, -3, -4, -5):
        assert clib.lcp_status_string(code)
    assert clib.lcp_version() >= 10000


def _err(clib):
    return clib.lcp_last_error().decode()


def test_stats_rejects_bad_arguments(clib):
    f = clib.lcp_stats
    outs = [FAKE] * 4
    assert f(None, FAKE, 0, 4, 8, 8, 64, 1, *outs, None) == -1 and "non-NULL" in _err(clib)
    assert f(FAKE, FAKE, 0, 4, 1, 8, 64, 1, *outs, None) == -1 and "H >= 2" in _err(clib)
    assert f(FAKE, FAKE, 0, 1, 8, 8, 64, 1, *outs, None) == -1 and "M - ddof" in _err(clib)
    assert f(FAKE, FAKE, 0, 4, 8, 8, 63, 1, *outs, None) == -1 and "member_stride" in _err(clib)
    assert f(FAKE, FAKE, 2, 4, 8, 8, 64, 1, *outs, None) == -1 and "dtype" in _err(clib)
    assert f(FAKE, FAKE, 0, 4, 8, 8, 64, 2, *outs, None) == -1 and "ddof" in _err(clib)


def test_fused_map_mc_reject_bad_arguments(clib):
    iso = (ctypes.c_float * 2)(0.0, 1.0)
    fused = clib.lcp_fused
    assert fused(FAKE, FAKE, 0, 4, 8, 8, 64, 1, 1.0, 0.0, iso, 2, FAKE, 0, None, None) == -1
    assert "dx and dy" in _err(clib)
    assert fused(FAKE, FAKE, 0, 4, 8, 8, 64, 1, 1.0, 1.0, iso, 0, FAKE, 0, None, None) == -1
    assert fused(FAKE, FAKE, 0, 4, 8, 8, 64, 1, 1.0, 1.0, iso, 2, FAKE, 1, None, None) == -1  # bf16 output
    assert fused(FAKE, FAKE, 0, 4, 8, 8, 64, 1, 1.0, 1.0, None, 2, FAKE, 0, None, None) == -1
    assert clib.lcp_map(FAKE, FAKE, 8, 8, iso, 300, FAKE, 0, None, None) == -1
    assert clib.lcp_divergence(FAKE, FAKE, FAKE, FAKE, 8, 8, -1.0, 1.0, FAKE, FAKE, None) == -1
    mc = clib.lcp_mc
    assert mc(0, FAKE, FAKE, FAKE, FAKE, None, None, 0, 0, 0, 8, 8, 1.0, 1.0, iso, 2, 0, 1, 0, FAKE, None, None) == -1
    assert "n_samples" in _err(clib)
    assert mc(0, FAKE, FAKE, FAKE, FAKE, None, None, 0, 0, 0, 8, 8, 1.0, 1.0, iso, 2, 10, 1, 0, None, None, None) == -1
    assert mc(5, FAKE, FAKE, FAKE, FAKE, None, None, 0, 0, 0, 8, 8, 1.0, 1.0, iso, 2, 10, 1, 0, FAKE, None, None) == -1
    assert mc(1, None, None, None, None, None, FAKE, 0, 4, 64, 8, 8, 1.0, 1.0, iso, 2, 10, 1, 0, FAKE, None, None) == -1
    assert clib.lcp_philox_fill(0, 0, 0, 0, None, None) == 0  # empty request: nothing to do
    assert clib.lcp_philox_fill(0, 0, 0, 10, None, None) == -1


def test_product_package_never_reaches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2510_01190_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
                assert "lcp_oracle" not in src, f


def test_oracle_never_reaches_the_product_package():
    """The oracle shares no code with the CUDA path: its modules import only the
    standard library, numpy, scipy and each other, never the product package."""
    allowed = {"__future__", "math", "numpy", "scipy"}
    odir = os.path.join(ROOT, "oracle")
    for f in sorted(os.listdir(odir)):
        if not f.endswith(".py"):
            continue
        src = open(os.path.join(odir, f)).read()
        for m in re.finditer(r"^\s*(?:import|from)\s+([A-Za-z_.][A-Za-z0-9_.]*)", src, flags=re.M):
            mod = m.group(1)
            assert mod.startswith(".") or mod.split(".")[0] in allowed, (f, mod)


def test_input_generators_stand_apart_from_both_sides():
    """The seeded input generators, the one module that the oracle's tests and
    the CUDA path's tests share, import neither the library binding nor the
    oracle."""
    src = open(os.path.join(ROOT, "paper_2510_01190_gb300", "synth.py")).read()
    mods = {m.group(1).split(".")[0]
            for m in re.finditer(r"^\s*(?:import|from)\s+([A-Za-z_.][A-Za-z0-9_.]*)", src, flags=re.M)}
    assert mods <= {"__future__", "math", "numpy", "torch", "statistics"}, mods


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2510_01190_gb300 import _binding

    monkeypatch.setattr(_binding, "_LIB", None)
    monkeypatch.setattr(_binding, "library_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(_binding.LcpError):
        _binding.load(build_if_stale=False)


def test_colormap_rejects_bad_arguments(clib):
    f = clib.lcp_colormap
    good = (ctypes.c_float * 10)(0.0, 0, 0, 0, 1, 1.0, 1, 1, 1, 1)
    assert f(FAKE, 1, 4, 4, 1.0, 1.0, good, 2, 0, None, 0, FAKE, None) == -1 and "vmin < vmax" in _err(clib)
    assert f(FAKE, 1, 4, 4, 0.0, float("nan"), good, 2, 0, None, 0, FAKE, None) == -1
    assert f(FAKE, 1, 4, 4, 0.0, 1.0, good, 1, 0, None, 0, FAKE, None) == -1 and "stops" in _err(clib)
    assert f(FAKE, 1, 4, 4, 0.0, 1.0, None, 2, 0, None, 0, FAKE, None) == -1
    back = (ctypes.c_float * 10)(1.0, 0, 0, 0, 1, 0.0, 1, 1, 1, 1)
    assert f(FAKE, 1, 4, 4, 0.0, 1.0, back, 2, 0, None, 0, FAKE, None) == -1 and "increase" in _err(clib)
    short = (ctypes.c_float * 10)(0.0, 0, 0, 0, 1, 0.5, 1, 1, 1, 1)
    assert f(FAKE, 1, 4, 4, 0.0, 1.0, short, 2, 0, None, 0, FAKE, None) == -1 and "last at 1" in _err(clib)
    bright = (ctypes.c_float * 10)(0.0, 0, 0, 0, 1, 1.0, 2, 1, 1, 1)
    assert f(FAKE, 1, 4, 4, 0.0, 1.0, bright, 2, 0, None, 0, FAKE, None) == -1 and "outside" in _err(clib)
    assert f(FAKE, -1, 4, 4, 0.0, 1.0, good, 2, 0, None, 0, FAKE, None) == -1
    assert f(None, 1, 4, 4, 0.0, 1.0, good, 2, 0, None, 0, FAKE, None) == -1 and "NULL" in _err(clib)
    assert f(ctypes.c_void_p(258), 1, 4, 4, 0.0, 1.0, good, 2, 0, None, 0, FAKE, None) == -1
    assert f(None, 0, 4, 4, 0.0, 1.0, good, 2, 0, None, 0, None, None) == 0  # empty: nothing to do


def test_speed_gradient_rejects_bad_arguments(clib):
    iso = (ctypes.c_float * 2)(0.0, 1.0)
    g = clib.lcp_speed_gradient
    assert g(FAKE, FAKE, 0, 4, 8, 8, 64, 1.0, 1.0, FAKE, None, None) == -1 and "NULL" in _err(clib)
    assert g(FAKE, FAKE, 0, 4, 8, 8, 64, 0.0, 1.0, FAKE, FAKE, None) == -1 and "dx and dy" in _err(clib)
    assert g(FAKE, FAKE, 0, 4, 8, 8, 63, 1.0, 1.0, FAKE, FAKE, None) == -1 and "member_stride" in _err(clib)
    f = clib.lcp_speed_gradient_ws
    args = [FAKE, FAKE, 0, 4, 8, 8, 64, 1, 1.0, 1.0, iso, 2, FAKE, 0, None]
    assert f(*args, None, 0, None) == -1 and "workspace" in _err(clib)
    assert f(*args, ctypes.c_void_p(512), 16, None) == -1 and "too small" in _err(clib)
    assert f(*args, ctypes.c_void_p(520), 1 << 30, None) == -1 and "aligned" in _err(clib)
    big = [FAKE, FAKE, 0, 2, 65536, 32768, 65536 * 32768, 1, 1.0, 1.0, iso, 2, FAKE, 0, None]
    assert f(*big, ctypes.c_void_p(512), 1 << 40, None) == -3 and "2^31" in _err(clib)


def test_volume_calls_reject_bad_arguments(clib):
    iso = (ctypes.c_float * 2)(0.0, 1.0)
    f = clib.lcp3d_fused_ws
    ws = ctypes.c_void_p(512)
    ok = [FAKE, FAKE, FAKE, 0, 4, 5, 6, 7, 5 * 6 * 7, 1, 1.0, 1.0, 1.0, iso, 2, FAKE, 0, None]
    assert clib.lcp3d_workspace_bytes(4, 5, 6, 7, 0) > 0 and clib.lcp3d_workspace_bytes(4, 1, 6, 7, 0) == 0
    bad = list(ok)
    bad[2] = None
    assert f(*bad, ws, 1 << 30, None) == -1 and "non-NULL" in _err(clib)
    bad = list(ok)
    bad[5] = 1
    assert f(*bad, ws, 1 << 30, None) == -1 and "D, H, W >= 2" in _err(clib)
    bad = list(ok)
    bad[12] = 0.0
    assert f(*bad, ws, 1 << 30, None) == -1 and "dz" in _err(clib)
    bad = list(ok)
    bad[8] = 5 * 6 * 7 - 1
    assert f(*bad, ws, 1 << 30, None) == -1 and "member_stride" in _err(clib)
    assert f(*ok, None, 1 << 30, None) == -1 and "workspace" in _err(clib)
    assert f(*ok, ws, 64, None) == -1 and "too small" in _err(clib)
    assert clib.lcp3d_divergence(FAKE, FAKE, FAKE, FAKE, FAKE, None, 4, 4, 4, 1.0, 1.0, 1.0, FAKE, FAKE, None) == -1
    assert clib.lcp3d_divergence(*([FAKE] * 6), 4, 4, 4, 1.0, 1.0, -1.0, FAKE, FAKE, None) == -1
    assert clib.lcp3d_map(FAKE, FAKE, 4, 4, 4, iso, 65, FAKE, 0, None, None) == -3
    assert clib.lcp3d_map(FAKE, FAKE, 4, 4, 4, iso, 2, FAKE, 1, None, None) == -1


def test_contour_calls_reject_bad_arguments(clib):
    iso = (ctypes.c_float * 2)(0.0, 1.0)
    ws, cnt = ctypes.c_void_p(512), ctypes.c_void_p(1024)
    f = clib.lcp_contours
    assert clib.lcp_contours_workspace_bytes(1, 4, 4) == 256 + 8 and clib.lcp_contours_workspace_bytes(1, 1, 4) == 0
    assert f(None, 4, 4, iso, 2, FAKE, None, 10, cnt, ws, 1 << 20, None) == -1 and "field" in _err(clib)
    assert f(FAKE, 1, 4, iso, 2, FAKE, None, 10, cnt, ws, 1 << 20, None) == -1
    assert f(FAKE, 4, 4, iso, 65, FAKE, None, 10, cnt, ws, 1 << 20, None) == -3
    assert f(FAKE, 4, 4, iso, 2, None, None, 10, cnt, ws, 1 << 20, None) == -1 and "capacity" in _err(clib)
    assert f(FAKE, 4, 4, iso, 2, ctypes.c_void_p(264), None, 10, cnt, ws, 1 << 20, None) == -1 and "16-byte" in _err(clib)
    assert f(FAKE, 4, 4, iso, 2, FAKE, None, 10, None, ws, 1 << 20, None) == -1 and "count" in _err(clib)
    assert f(FAKE, 4, 4, iso, 2, FAKE, None, 10, cnt, None, 1 << 20, None) == -1 and "workspace" in _err(clib)
    assert f(FAKE, 4, 4, iso, 2, FAKE, None, 10, cnt, ws, 8, None) == -1 and "too small" in _err(clib)
    g = clib.lcp_member_contours
    assert g(FAKE, FAKE, 0, 3, 4, 4, 15, 1.0, 1.0, iso, 2, FAKE, None, 10, cnt, ws, 1 << 20, None) == -1
    assert g(FAKE, FAKE, 0, 3, 4, 4, 16, 1.0, 0.0, iso, 2, FAKE, None, 10, cnt, ws, 1 << 20, None) == -1


def test_fused_band_rows_keep_one_band_when_the_workspace_is_exact(clib):
    """lcp_fused_band_rows is host arithmetic: a workspace of exactly
    lcp_fused_workspace_bytes keeps the budget's bands (one band whenever the
    grid fits the 96 MB budget), a smaller one gives smaller bands in whole
    8-row tiles, and one below the smallest band gives 0."""
    rows = clib.lcp_fused_band_rows
    need = clib.lcp_fused_workspace_bytes
    for h, w in ((721, 1440), (2, 2), (9, 2), (60, 64), (601, 4096), (2185, 2), (3000, 1)):
        if w < 2:
            assert rows(h, w, 1 << 30) == 0
            continue
        assert rows(h, w, need(1, h, w, 0)) == h - 1, (h, w)
        assert rows(h, w, need(1, h, w, 0) + 12345) == h - 1
    assert rows(1001, 4096, need(1, 1001, 4096, 0)) == 760  # 131 MB of records: 766 rows in 96 MB
    # 8192 columns: 512 KiB of records per row, 382 rows in 96 MB -> bands of 376
    full = need(20, 8192, 8192, 1)
    assert rows(8192, 8192, full) == 376
    last = 376
    for cap in (full - 1, 80 << 20, 64 << 20, 20 << 20, 6 << 20):
        r = rows(8192, 8192, cap)
        assert 8 <= r < 376 and r % 8 == 0 and r <= last, (cap, r)
        assert (r + 3) * 8192 * 32 <= cap < (r + 8 + 3) * 8192 * 32 + 4096, (cap, r)
        last = r
    assert rows(8192, 8192, 64 << 20) == 248  # the static 64 MiB scratch of lcp_fused_static_ws
    assert rows(8192, 8192, 11 * 8192 * 32 - 1) == 0  # below 8 rows plus 3 halo/record rows
    assert rows(1, 8192, full) == 0 and rows(8192, 8192, 0) == 0


def test_volume_ring_and_contour_workspace_sizes(clib):
    """Host arithmetic of the 3D ring and the contour scratch.  The ring holds
    2B + 3 z-planes of 48-byte records (u, v, w per vertex): B new planes per
    slab (as many as fit a 96 MB budget, at least 1, at most D) plus the 3
    planes the next slab re-reads."""
    ws3 = clib.lcp3d_workspace_bytes
    plane = lambda h, w: h * w * 48  # noqa: E731
    # 256^2 planes: 3.1 MB each, 32 fit in 96 MB -> B = 14, a 31-plane ring
    assert ws3(20, 256, 256, 256, 0) == 31 * plane(256, 256)
    # 256 x 683: 8.4 MB planes, 11 fit -> B = 4, an 11-plane ring
    assert ws3(3, 9, 256, 683, 0) == 11 * plane(256, 683)
    # tiny volumes: B is capped at D
    assert ws3(1, 2, 2, 2, 0) == (2 * 2 + 3) * plane(2, 2)
    assert ws3(4, 5, 7, 40, 1) == (2 * 5 + 3) * plane(7, 40)
    # planes too large for 5 in the budget still get B = 1 (a 5-plane ring)
    assert ws3(2, 64, 1024, 1024, 0) == 5 * plane(1024, 1024)
    for bad in ((1, 1, 4, 4), (1, 4, 1, 4), (1, 4, 4, 1)):
        assert ws3(*bad, 0) == 0
    wsc = clib.lcp_contours_workspace_bytes
    assert wsc(0, 4, 4) == 0 and wsc(1, 1, 4) == 0 and wsc(1, 4, 1) == 0
    prev = 0
    for m, h, w in ((1, 2, 2), (1, 97, 131), (51, 721, 1440)):
        n = wsc(m, h, w)
        assert n >= 264 and (n - 256) % 8 == 0 and n > prev  # header + one 8-byte descriptor per tile
        prev = n


def test_fused_host_rejects_bad_arguments_and_sizes_its_workspace(clib):
    """lcp_fused_host: host-side checks before any device work, and its
    workspace = the map and mask staging (each rounded up to 256 bytes) plus
    lcp_fused_ws's records (host arithmetic only)."""
    iso = (ctypes.c_float * 2)(0.0, 1.0)
    f = clib.lcp_fused_host
    head = [FAKE, FAKE, 0, 4, 8, 8, 64, 1, 1.0, 1.0, iso, 2]
    ws = ctypes.c_void_p(512)
    assert f(*head, None, 0, None, ws, 1 << 30, None) == -1 and "NULL output" in _err(clib)
    assert f(*head, FAKE, 3, None, ws, 1 << 30, None) == -1 and "out dtype" in _err(clib)  # F64
    assert f(*head, FAKE, 0, None, None, 1 << 30, None) == -1 and "workspace" in _err(clib)
    assert f(*head, FAKE, 0, None, ctypes.c_void_p(520), 1 << 30, None) == -1 and "aligned" in _err(clib)
    bad = list(head)
    bad[6] = 63  # member stride below H * W
    assert f(*bad, FAKE, 0, None, ws, 1 << 30, None) == -1 and "member_stride" in _err(clib)
    size = clib.lcp_fused_host_workspace_bytes
    records = clib.lcp_fused_workspace_bytes(4, 8, 8, 0)
    # K = 2 maps of 7 x 7 fp32 cells = 392 B -> 512; mask words 2 x 7 x 1 x 4 = 56 B -> 256
    assert size(4, 8, 8, 2, 0, 0) == 512 + records
    assert size(4, 8, 8, 2, 0, 1) == 512 + 256 + records
    assert size(4, 8, 8, 2, 2, 0) == 256 + records  # fp16 maps: 196 B -> 256
    assert size(4, 1, 8, 2, 0, 0) == 0 and size(4, 8, 8, 0, 0, 0) == 0
