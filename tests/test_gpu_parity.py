"""GPU parity: every C-ABI entry point against the FP64 oracle on the same inputs.

Tolerances (each derived from the arithmetic of the two sides):
* LCP in fp32: max |gpu - oracle| <= 1e-5 (the target), observed ~1e-6.
* LCP in fp16: |gpu - fp16(oracle)| <= 1 fp16 ulp of the value.
* Mean-field masks: bit-exact on dyadic data (exact arithmetic on both sides);
  on general data bit-exact outside a guard band |mu_d - c| <= 1e-5 (|mu_d| + 1).
* Statistics / divergence: FP32 rounding bounds (relative 2e-6 / 2e-5).
* Monte Carlo: same Philox streams on both sides, so crossing counts agree
  except where a divergence sample lies within FP32 rounding of c.
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2510_01190_gb300 import synth

pytestmark = pytest.mark.gpu

LCP_TOL = 1e-5


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


def _np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def _fields(h, w, m, seed, kind="fourier", k=4):
    if kind == "fourier":
        d = synth.fourier_ensemble(seed, h=h, w=w, m=m, k=k)
    elif kind == "sources":
        d = synth.point_sources_ensemble(seed, h=h, w=w, m=m)
    else:
        raise ValueError(kind)
    return d


def _oracle_mask_guard(mu_d, iso):
    """cells whose vertices are all clear of the FP32 rounding band around c"""
    out = []
    for c in iso:
        clear = np.abs(mu_d - c) > 1e-5 * (np.abs(mu_d) + 1.0)
        out.append(clear[:-1, :-1] & clear[:-1, 1:] & clear[1:, :-1] & clear[1:, 1:])
    return np.stack(out)


# ---------------------------------------------------------------------------
# statistics, divergence, map (unfused path)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("h,w,m,ddof", [(64, 64, 20, 1), (37, 53, 7, 0), (5, 3, 1, 0), (2, 2, 2, 1), (181, 360, 51, 1)])
def test_stats_parity(lib, h, w, m, ddof):
    d = _fields(h, w, m, seed=h * 7 + w)
    mu_u, var_u, mu_v, var_v = lib.lcp_stats(_dev(d["u"]), _dev(d["v"]), ddof)
    for x, mu, var in ((d["u"], mu_u, var_u), (d["v"], mu_v, var_v)):
        om, ov = O.ensemble_stats(x, ddof)
        scale = np.abs(om) + np.sqrt(ov) + 1e-30
        assert np.max(np.abs(_np(mu) - om) / scale) < 2e-6
        assert np.max(np.abs(_np(var) - ov) / (ov + 1e-12)) < 2e-5


def test_stats_bf16_and_strided_members(lib):
    d = _fields(40, 72, 12, seed=3)
    u16 = _dev(d["u"], torch.bfloat16)
    v16 = _dev(d["v"], torch.bfloat16)
    # members embedded in a larger buffer: member stride > H*W
    big_u = torch.zeros((12, 40 * 72 + 64), device="cuda", dtype=torch.bfloat16)
    big_v = torch.zeros_like(big_u)
    big_u[:, : 40 * 72] = u16.reshape(12, -1)
    big_v[:, : 40 * 72] = v16.reshape(12, -1)
    su = big_u.as_strided((12, 40, 72), (40 * 72 + 64, 72, 1))
    sv = big_v.as_strided((12, 40, 72), (40 * 72 + 64, 72, 1))
    for uu, vv in ((u16, v16), (su, sv)):
        mu_u, var_u, mu_v, var_v = lib.lcp_stats(uu, vv, 1)
        om, ov = O.ensemble_stats(_np(u16), 1)
        assert np.max(np.abs(_np(mu_u) - om) / (np.abs(om) + np.sqrt(ov))) < 2e-6
        assert np.max(np.abs(_np(var_u) - ov) / (ov + 1e-12)) < 2e-5


@pytest.mark.parametrize("m", [1, 2, 9, 10, 11, 20, 23, 31])
def test_stats_bf16_member_batches(lib, m):
    """bf16 lcp_stats over member counts that give every batch shape of its 8-byte
    loads (below one batch, exactly one, one plus a remainder, two, two plus a
    remainder), on a plane whose vertex count leaves a ragged tail (37 x 53 = 1961)."""
    ddof = 0 if m == 1 else 1
    d = _fields(37, 53, m, seed=70 + m)
    u16, v16 = _dev(d["u"], torch.bfloat16), _dev(d["v"], torch.bfloat16)
    mu_u, var_u, mu_v, var_v = lib.lcp_stats(u16, v16, ddof)
    for x, mu, var in ((u16, mu_u, var_u), (v16, mu_v, var_v)):
        om, ov = O.ensemble_stats(_np(x), ddof)  # the same bf16-rounded values
        assert np.max(np.abs(_np(mu) - om) / (np.abs(om) + np.sqrt(ov) + 1e-30)) < 2e-6
        assert np.max(np.abs(_np(var) - ov) / (ov + 1e-12)) < 2e-5


@pytest.mark.parametrize("h,w,dx,dy", [(64, 64, 1.0, 1.0), (9, 130, 0.5, 2.0), (2, 2, 1.0, 3.0), (300, 7, 0.1, 0.1)])
def test_divergence_parity(lib, h, w, dx, dy):
    st = synth.random_stats(h * w, h, w, zero_fraction=0.05)
    mu_d, var_d = lib.lcp_divergence(*map(_dev, st), dx, dy)
    om, ov = O.divergence_gaussian(*[s.astype(np.float64) for s in st], dx, dy)
    scale = np.abs(om) + np.sqrt(ov) + 1e-30
    assert np.max(np.abs(_np(mu_d) - om) / scale) < 2e-6
    assert np.max(np.abs(_np(var_d) - ov) / (ov + 1e-30)) < 2e-6


@pytest.mark.parametrize("h,w,k", [(64, 64, 1), (33, 517, 5), (2, 2, 3), (130, 33, 70)])
def test_map_parity(lib, h, w, k):
    st = synth.random_stats(7 + h, h, w, zero_fraction=0.1)
    om, ov = O.divergence_gaussian(*[s.astype(np.float64) for s in st], 1.0, 1.0)
    mu32, var32 = om.astype(np.float32), ov.astype(np.float32)
    var32[::5, ::3] = 0.0
    iso = np.quantile(mu32, np.linspace(0.1, 0.9, k)).astype(np.float32)
    lcp, mask = lib.lcp_map(_dev(mu32), _dev(var32), iso, mask=True)
    ref = O.level_crossing_probability(mu32, var32, iso)
    assert np.max(np.abs(_np(lcp) - ref)) <= LCP_TOL
    got_mask = lib.unpack_mask(mask, w).cpu().numpy()
    want_mask = O.mean_field_crossing(mu32, iso)
    assert np.array_equal(got_mask, want_mask)  # exact: same fp32 mu_d on both sides


# ---------------------------------------------------------------------------
# fused path
# ---------------------------------------------------------------------------
FUSED_CASES = [
    # h, w, m, k, generator      (vector path needs W % 4 == 0; others take the scalar path)
    (64, 64, 20, 1, "sources"),
    (181, 360, 51, 8, "fourier"),
    (2, 2, 1, 1, "fourier"),
    (3, 5, 2, 2, "fourier"),
    (45, 1028, 9, 3, "fourier"),   # 3 column tiles, ragged last tile
    (70, 1031, 6, 2, "fourier"),   # odd W: scalar loads, 9 column tiles
    (97, 64, 40, 33, "fourier"),   # K > 32: two isovalue passes
    (300, 16, 3, 4, "fourier"),    # tall and narrow: many bands
]


@pytest.mark.parametrize("entry", ["lcp_fused", "lcp_fused_ws"])
@pytest.mark.parametrize("h,w,m,k,kind", FUSED_CASES)
def test_fused_parity(lib, h, w, m, k, kind, entry):
    d = _fields(h, w, m, seed=h + 3 * w, kind=kind, k=k) if kind == "fourier" else _fields(h, w, m, 0, kind)
    iso = d["isovalues"][:k] if len(d["isovalues"]) >= k else np.linspace(-0.5, 0.5, k).astype(np.float32)
    ddof = 1 if m > 1 else 0
    fn = getattr(lib, entry)
    lcp, mask = fn(_dev(d["u"]), _dev(d["v"]), iso, d["dx"], d["dy"], ddof=ddof, mask=True)
    ref = O.lcp_closed_form(d["u"], d["v"], d["dx"], d["dy"], iso, ddof)
    err = np.abs(_np(lcp) - ref["lcp"])
    assert np.max(err) <= LCP_TOL, np.max(err)
    guard = _oracle_mask_guard(ref["mu_d"], iso)
    got = lib.unpack_mask(mask, w).cpu().numpy()
    assert np.array_equal(got[guard], ref["mask"][guard])


def test_fused_equals_unfused_chain(lib):
    d = _fields(90, 200, 17, seed=5, k=5)
    u, v = _dev(d["u"]), _dev(d["v"])
    iso = d["isovalues"]
    fused, fm = lib.lcp_fused(u, v, iso, mask=True)
    st = lib.lcp_stats(u, v, 1)
    mu_d, var_d = lib.lcp_divergence(*st)
    chain, cm = lib.lcp_map(mu_d, var_d, iso, mask=True)
    assert torch.max(torch.abs(fused - chain)).item() <= 2e-6


@pytest.mark.parametrize("entry", ["lcp_fused", "lcp_fused_ws"])
def test_fused_fp16_output_within_one_ulp(lib, entry):
    d = _fields(61, 256, 10, seed=9, k=4)
    lcp, _ = getattr(lib, entry)(_dev(d["u"]), _dev(d["v"]), d["isovalues"], out_dtype=torch.float16)
    ref = O.lcp_closed_form(d["u"], d["v"], 1.0, 1.0, d["isovalues"])["lcp"]
    ref16 = ref.astype(np.float16).astype(np.float64)
    ulp = np.spacing(np.abs(ref16).astype(np.float16)).astype(np.float64)
    assert np.all(np.abs(_np(lcp) - ref16) <= ulp + 1e-12)


@pytest.mark.parametrize("entry", ["lcp_fused", "lcp_fused_ws"])
def test_fused_bf16_members(lib, entry):
    fn = getattr(lib, entry)
    d = _fields(64, 512, 20, seed=11, k=4)
    u16, v16 = _dev(d["u"], torch.bfloat16), _dev(d["v"], torch.bfloat16)
    lcp, _ = fn(u16, v16, d["isovalues"])
    ref = O.lcp_closed_form(_np(u16), _np(v16), 1.0, 1.0, d["isovalues"])["lcp"]  # same bf16-rounded values
    assert np.max(np.abs(_np(lcp) - ref)) <= LCP_TOL
    # odd width: scalar bf16 path
    d = _fields(33, 99, 5, seed=12, k=2)
    u16, v16 = _dev(d["u"], torch.bfloat16), _dev(d["v"], torch.bfloat16)
    lcp, _ = fn(u16, v16, d["isovalues"])
    ref = O.lcp_closed_form(_np(u16), _np(v16), 1.0, 1.0, d["isovalues"])["lcp"]
    assert np.max(np.abs(_np(lcp) - ref)) <= LCP_TOL


@pytest.mark.parametrize("entry", ["lcp_fused", "lcp_fused_ws"])
def test_fused_large_offset_keeps_accuracy(lib, entry):
    """|mean| / sigma ~ 2e5: the member-0 shift cancels the offset exactly."""
    d = _fields(48, 128, 20, seed=13, k=3)
    u = (d["u"] * 0.05 + 1e4).astype(np.float32)
    v = (d["v"] * 0.05 + 1e4).astype(np.float32)
    iso = (d["isovalues"] * 0.05).astype(np.float32)
    lcp, _ = getattr(lib, entry)(_dev(u), _dev(v), iso)
    ref = O.lcp_closed_form(u, v, 1.0, 1.0, iso)["lcp"]
    assert np.max(np.abs(_np(lcp) - ref)) <= LCP_TOL


@pytest.mark.parametrize("entry", ["lcp_fused", "lcp_fused_ws"])
def test_fused_dyadic_zero_variance_is_bit_exact(lib, entry):
    for (h, w, dx) in ((33, 68, 1.0), (20, 77, 0.5)):
        d = synth.dyadic_ensemble(h * w, h, w, m=4, k=3)
        lcp, mask = getattr(lib, entry)(_dev(d["u"]), _dev(d["v"]), d["isovalues"], dx, dx, mask=True)
        ref = O.lcp_closed_form(d["u"], d["v"], dx, dx, d["isovalues"])
        assert np.array_equal(lib.unpack_mask(mask, w).cpu().numpy(), ref["mask"])
        assert np.array_equal(_np(lcp), ref["lcp"])  # var = 0: LCP is the mask exactly


@pytest.mark.parametrize("entry", ["lcp_fused", "lcp_fused_ws"])
def test_fused_nan_member_propagates(lib, entry):
    d = _fields(20, 40, 6, seed=14, k=2)
    u = d["u"].copy()
    u[3, 10, 17] = np.nan
    lcp, _ = getattr(lib, entry)(_dev(u), _dev(d["v"]), d["isovalues"])
    ref = O.lcp_closed_form(u, d["v"], 1.0, 1.0, d["isovalues"])["lcp"]
    got = _np(lcp)
    assert np.array_equal(np.isnan(got), np.isnan(ref)) and np.isnan(ref).any()
    ok = ~np.isnan(ref)
    assert np.max(np.abs(got[ok] - ref[ok])) <= LCP_TOL


@pytest.mark.slow
@pytest.mark.parametrize("entry", ["lcp_fused", "lcp_fused_ws"])
def test_fused_full_size_latlon(lib, entry):
    """The 721 x 1440 x 51, K = 8 workload in the bench's launch configuration,
    compared with the oracle on every cell."""
    d = synth.fourier_ensemble(0)
    u, v = _dev(d["u"]), _dev(d["v"])
    lcp, mask = getattr(lib, entry)(u, v, d["isovalues"], mask=True)
    ref = O.lcp_closed_form(d["u"], d["v"], 1.0, 1.0, d["isovalues"])
    assert np.max(np.abs(_np(lcp) - ref["lcp"])) <= LCP_TOL
    guard = _oracle_mask_guard(ref["mu_d"], d["isovalues"])
    assert np.array_equal(lib.unpack_mask(mask, 1440).cpu().numpy()[guard], ref["mask"][guard])


# ---------------------------------------------------------------------------
# Monte Carlo
# ---------------------------------------------------------------------------
def test_philox_fill_bit_exact(lib):
    for seed, c1, off in ((0, 0, 0), (2**40 + 7, 12345, 2**33 + 5), (2**64 - 1, 2**32 - 1, 2**64 - 1)):
        got = lib.lcp_philox_fill(seed, c1, off, 5000).cpu().numpy().view(np.uint32)
        ctr = np.zeros((5000, 4), np.uint64)
        ctr[:, 0] = np.arange(5000)
        ctr[:, 1] = c1
        ctr[:, 2] = off & 0xFFFFFFFF
        ctr[:, 3] = off >> 32
        want = O.philox4x32_10(ctr, (seed & 0xFFFFFFFF, seed >> 32))
        assert np.array_equal(got, want)


def _count_agreement(got, want, n_samples):
    diff = np.abs(got.astype(np.int64) - want)
    assert diff.max() <= 2, diff.max()
    assert np.mean(diff > 0) < 2e-3


@pytest.mark.parametrize("h,w,k,s", [(40, 70, 2, 64), (9, 33, 17, 31), (2, 2, 1, 5)])
def test_mc_gauss_counts_match_oracle(lib, h, w, k, s):
    st = synth.random_stats(h + w, h, w, sd_scale=0.4)
    om, _ = O.divergence_gaussian(*[x.astype(np.float64) for x in st], 1.0, 1.0)
    iso = np.quantile(om, np.linspace(0.2, 0.8, k)).astype(np.float32)
    est, counts = lib.lcp_mc(iso, s, seed=77, dx=1.0, dy=1.0, stats=tuple(map(_dev, st)), offset=3)
    _, want = O.mc_lcp(iso, s, seed=77, dx=1.0, dy=1.0, stats=st, offset=3)
    got = counts.cpu().numpy().view(np.uint32)
    _count_agreement(got, want, s)
    assert np.max(np.abs(_np(est) - got / s)) < 1e-6


def test_mc_empirical_counts_match_oracle(lib):
    d = _fields(30, 44, 9, seed=21, k=3)
    iso = d["isovalues"]
    est, counts = lib.lcp_mc(iso, 40, seed=5, mode="empirical", members=(_dev(d["u"]), _dev(d["v"])))
    _, want = O.mc_lcp(iso, 40, seed=5, dx=1.0, dy=1.0, mode="empirical", members=(d["u"], d["v"]))
    _count_agreement(counts.cpu().numpy().view(np.uint32), want, 40)


def test_mc_converges_to_closed_form(lib):
    d = synth.point_sources_ensemble(1)
    u, v = _dev(d["u"]), _dev(d["v"])
    st = lib.lcp_stats(u, v, 1)
    iso = np.array([0.0, -0.02], np.float32)
    closed, _ = lib.lcp_fused(u, v, iso)
    s = 20000
    est, _ = lib.lcp_mc(iso, s, seed=1, stats=st)
    c, e = _np(closed)[:, 1:-1, 1:-1], _np(est)[:, 1:-1, 1:-1]  # interior cells (independent vertices)
    se = np.sqrt(c * (1 - c) / s) + 1e-9
    assert np.abs((e - c) / se).max() < 5.5


# ---------------------------------------------------------------------------
# both fused variants (TMA pipeline and register streaming) on the same input
# ---------------------------------------------------------------------------
_VARIANT_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_2510_01190_gb300 as lib
from paper_2510_01190_gb300 import synth
d = synth.fourier_ensemble(31, h=150, w=516, m=23, k=5)
u = torch.from_numpy(d["u"]).cuda(); v = torch.from_numpy(d["v"]).cuda()
lcp, mask = lib.lcp_fused(u, v, d["isovalues"], mask=True)
np.save(sys.argv[2], lcp.cpu().numpy()); np.save(sys.argv[3], mask.cpu().numpy())
"""


def test_register_streaming_variant_matches_oracle(tmp_path):
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "variant.py"
    script.write_text(_VARIANT_SCRIPT)
    outs = {}
    for tma in ("0", "1"):
        env = dict(os.environ, LCP_FUSED_TMA=tma)
        a, b = tmp_path / f"lcp{tma}.npy", tmp_path / f"mask{tma}.npy"
        subprocess.run([sys.executable, str(script), root, str(a), str(b)], check=True, env=env, timeout=600)
        outs[tma] = (np.load(a), np.load(b))
    d = synth.fourier_ensemble(31, h=150, w=516, m=23, k=5)
    ref = O.lcp_closed_form(d["u"], d["v"], 1.0, 1.0, d["isovalues"])
    for tma in ("0", "1"):
        assert np.max(np.abs(outs[tma][0] - ref["lcp"])) <= LCP_TOL
    assert np.max(np.abs(outs["0"][0] - outs["1"][0])) <= 2e-6
    assert np.array_equal(outs["0"][1], outs["1"][1])


def test_device_status_clear_after_runs(lib):
    torch.cuda.synchronize()
    assert lib.lcp_device_status() == 0


def test_fused_ws_small_workspace_runs_smaller_bands(lib):
    """A workspace below lcp_fused_workspace_bytes runs the grid in smaller row
    bands with identical results; one below the smallest band is rejected."""
    d = _fields(60, 64, 4, seed=15, k=2)
    u, v = _dev(d["u"]), _dev(d["v"])
    need = lib.lcp_fused_workspace_bytes(4, 60, 64)
    ref, ref_mask = lib.lcp_fused_ws(u, v, d["isovalues"], mask=True)
    ws = torch.empty(need // 2 + 512, dtype=torch.uint8, device="cuda")
    base = ws.data_ptr() % 256
    ws = ws[(256 - base) % 256:]
    got, got_mask = lib.lcp_fused_ws(u, v, d["isovalues"], mask=True, workspace=ws)
    assert torch.equal(got, ref) and torch.equal(got_mask, ref_mask)
    tiny = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.LcpError) as e:
        lib.lcp_fused_ws(u, v, d["isovalues"], workspace=tiny)
    assert e.value.status == -1


def test_fused_ws_bands_finish_on_the_callers_stream(lib):
    """A grid run in several bands on a caller's (non-default) stream: a copy
    queued right after the call on that stream, with no device synchronisation
    in between, sees the finished map of every band."""
    d = _fields(60, 64, 4, seed=17, k=3)
    u, v = _dev(d["u"]), _dev(d["v"])
    ref, ref_mask = lib.lcp_fused_ws(u, v, d["isovalues"], mask=True)
    need = lib.lcp_fused_workspace_bytes(4, 60, 64)
    ws = torch.empty(need // 2 + 512, dtype=torch.uint8, device="cuda")
    ws = ws[(256 - ws.data_ptr() % 256) % 256:]
    assert 8 <= lib.lcp_fused_band_rows(60, 64, ws.numel()) < 59
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(3):
            out = torch.full_like(ref, float("nan"))
            mask = torch.full_like(ref_mask, -1)
            lib.lcp_fused_ws(u, v, d["isovalues"], mask=True, out=out, mask_out=mask, workspace=ws)
            seen, seen_mask = out.clone(), mask.clone()
            assert torch.equal(seen, ref) and torch.equal(seen_mask, ref_mask)


def test_fused_ws_repeated_calls_reuse_workspace(lib):
    """Counters are reset by every call: back-to-back calls on one workspace agree."""
    d = _fields(50, 300, 9, seed=16, k=3)
    u, v = _dev(d["u"]), _dev(d["v"])
    a, _ = lib.lcp_fused_ws(u, v, d["isovalues"])
    b, _ = lib.lcp_fused_ws(u, v, d["isovalues"])
    c, _ = lib.lcp_fused_ws(u, v, d["isovalues"][:2])
    assert torch.equal(a, b) and torch.equal(a[:2], c)
    assert lib.lcp_device_status() == 0


def test_map_single_gaussian_vertex_tracks_the_normal_tail(lib):
    """Cells with three deterministic vertices below c and one Gaussian vertex:
    LCP = P(D >= c) = erfc((c - mu)/(sigma sqrt 2))/2 exactly, so this pins the
    kernels' erfc over z in [-9, 9] against the oracle's FP64 erfc."""
    n = 2001
    z = np.linspace(-9.0, 9.0, n)
    w = 2 * n + 1
    mu = np.full((2, w), -1e3, np.float32)
    var = np.zeros((2, w), np.float32)
    sd = 0.37
    mu[1, 1::2] = (-z * sd).astype(np.float32)  # c = 0: (c - mu)/sd = z
    var[1, 1::2] = sd * sd
    lcp, _ = lib.lcp_map(_dev(mu), _dev(var), [0.0])
    ref = O.level_crossing_probability(mu, var, [0.0])
    err = np.abs(_np(lcp) - ref)
    assert err.max() <= 3e-7, err.max()


def test_fused_ws_row_bands_match_oracle(lib):
    """A grid of >= 2^18 vertices runs in bands of rows (48-row bands here), one
    halo row each side, alternating two workspace buffers, each band's cells
    on the auxiliary stream beside the next band's statistics."""
    h, w, m = 250, 16384, 3
    rng = np.random.default_rng(17)
    base = np.cumsum(rng.normal(size=(h, w)) * 0.05, axis=1).astype(np.float32)
    u = (base[None] + 0.3 * rng.standard_normal((m, h, w))).astype(np.float32)
    v = (base[None] * 0.5 + 0.3 * rng.standard_normal((m, h, w))).astype(np.float32)
    iso = np.array([-0.05, 0.02], np.float32)
    lcp, mask = lib.lcp_fused_ws(_dev(u), _dev(v), iso, mask=True)
    ref = O.lcp_closed_form(u, v, 1.0, 1.0, iso)
    assert np.max(np.abs(_np(lcp) - ref["lcp"])) <= LCP_TOL
    guard = _oracle_mask_guard(ref["mu_d"], iso)
    assert np.array_equal(lib.unpack_mask(mask, w).cpu().numpy()[guard], ref["mask"][guard])


@pytest.mark.parametrize("m", [2, 9, 10, 11, 20, 23, 31])
def test_fused_ws_bf16_banded_member_batches(lib, m):
    """bf16 members run in several row bands (a small workspace), so the statistics
    grid is the persistent one, with member counts that give every batch shape of the
    8-byte loads: fewer members than a batch, exactly one batch, a batch plus a
    remainder, two batches, two plus a remainder.  Against the oracle on the same
    bf16-rounded values, masks outside the guard band, and bit for bit against the
    single-band call (the per-vertex records do not depend on the bands)."""
    h, w = 120, 256
    d = _fields(h, w, m, seed=40 + m, k=4)
    u16, v16 = _dev(d["u"], torch.bfloat16), _dev(d["v"], torch.bfloat16)
    iso = d["isovalues"]
    row_bytes = 2 * w * 16
    ws = torch.empty(40 * row_bytes + 1024, dtype=torch.uint8, device="cuda")
    ws = ws[(256 - ws.data_ptr() % 256) % 256:]
    assert lib.lcp_fused_band_rows(h, w, ws.numel()) < h - 1  # several bands
    got, got_mask = lib.lcp_fused_ws(u16, v16, iso, mask=True, workspace=ws)
    one, one_mask = lib.lcp_fused_ws(u16, v16, iso, mask=True)
    assert torch.equal(got, one) and torch.equal(got_mask, one_mask)
    ref = O.lcp_closed_form(_np(u16), _np(v16), 1.0, 1.0, iso)
    assert np.max(np.abs(_np(got) - ref["lcp"])) <= LCP_TOL
    guard = _oracle_mask_guard(ref["mu_d"], iso)
    assert np.array_equal(lib.unpack_mask(got_mask, w).cpu().numpy()[guard], ref["mask"][guard])


@pytest.mark.slow
def test_fused_ws_ocean_8192_bf16_sampled(lib):
    """The 8192 x 8192 ocean-shaped workload (20 bf16 members, K = 4: 5.4 GB of
    members) in the bench's launch configuration; the oracle evaluates vertex
    crops (corner, interior, far edge) on the same bf16-rounded values, and the
    cells whose stencils lie inside a crop are compared."""
    if torch.cuda.get_device_properties(0).total_memory < 60e9:
        pytest.skip("needs the full-size device memory")
    d = synth.eddy_ensemble_torch(0)
    u, v, iso = d["u"], d["v"], d["isovalues"]
    H, W = u.shape[1:]
    lcp, mask = lib.lcp_fused_ws(u, v, iso, 1.0, 1.0, 1, mask=True)
    torch.cuda.synchronize()
    for (y0, x0) in ((0, 0), (4000, 3001), (H - 70, W - 110)):
        y1, x1 = min(y0 + 70, H), min(x0 + 110, W)
        uc, vc = _np(u[:, y0:y1, x0:x1]), _np(v[:, y0:y1, x0:x1])
        ref = O.lcp_closed_form(uc, vc, 1.0, 1.0, iso)
        vy = np.ones(y1 - y0, bool)
        vx = np.ones(x1 - x0, bool)
        vy[0], vy[-1] = y0 == 0, y1 == H
        vx[0], vx[-1] = x0 == 0, x1 == W
        sel = (vy[:-1] & vy[1:])[:, None] & (vx[:-1] & vx[1:])[None, :]
        got = _np(lcp[:, y0:y1 - 1, x0:x1 - 1])
        assert np.max(np.abs(got - ref["lcp"])[:, sel]) <= LCP_TOL
        guard = _oracle_mask_guard(ref["mu_d"], iso) & sel[None]
        gm = lib.unpack_mask(mask[:, y0:y1 - 1], W).cpu().numpy()[:, :, x0:x1 - 1]
        assert np.array_equal(gm[guard], ref["mask"][guard])
    del u, v, lcp, mask, d
    torch.cuda.empty_cache()


def test_fused_host_c_abi_host_and_device_outputs(lib):
    """lcp_fused_host called through the C ABI: pinned members read in place,
    the map copied into pageable host memory and into device memory, fp16
    maps, a workspace below the largest bands (smaller bands), all equal to
    lcp_fused_ws bit for bit; pageable members are rejected before any work."""
    import ctypes

    clib = lib.load()
    h, w, m = 61, 97, 7
    d = _fields(h, w, m, seed=23, k=3)
    iso = d["isovalues"]
    k = len(iso)
    u, v = torch.from_numpy(d["u"]), torch.from_numpy(d["v"])
    ref, ref_mask = lib.lcp_fused_ws(u.cuda(), v.cuda(), iso, mask=True)
    ref16, _ = lib.lcp_fused_ws(u.cuda(), v.cuda(), iso, out_dtype=torch.float16)
    uh, vh = u.pin_memory(), v.pin_memory()
    iso_c = (ctypes.c_float * k)(*[float(c) for c in iso])
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(uu, vv, out, out_code, mask, ws_bytes):
        ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device="cuda")
        p = ws.data_ptr() + (-ws.data_ptr()) % 256
        r = clib.lcp_fused_host(ctypes.c_void_p(uu.data_ptr()), ctypes.c_void_p(vv.data_ptr()), 0, m, h, w, h * w, 1,
                                1.0, 1.0, iso_c, k, ctypes.c_void_p(out.data_ptr()), out_code,
                                ctypes.c_void_p(mask.data_ptr()) if mask is not None else None, ctypes.c_void_p(p),
                                ws_bytes, st)
        torch.cuda.synchronize()
        return r

    need = clib.lcp_fused_host_workspace_bytes(m, h, w, k, 0, 1)
    out = torch.full((k, h - 1, w - 1), float("nan"))  # pageable host output
    mask = torch.full(tuple(ref_mask.shape), -1, dtype=torch.int32)
    assert call(uh, vh, out, 0, mask, need) == 0, clib.lcp_last_error()
    assert torch.equal(out, ref.cpu()) and torch.equal(mask, ref_mask.cpu())
    outd = torch.full_like(ref, float("nan"))  # device output
    assert call(uh, vh, outd, 0, None, clib.lcp_fused_host_workspace_bytes(m, h, w, k, 0, 0)) == 0
    assert torch.equal(outd, ref)
    out16 = torch.empty((k, h - 1, w - 1), dtype=torch.float16).pin_memory()
    assert call(uh, vh, out16, 2, None, clib.lcp_fused_host_workspace_bytes(m, h, w, k, 2, 0)) == 0
    assert torch.equal(out16, ref16.cpu())
    small = need - clib.lcp_fused_workspace_bytes(m, h, w, 0) + lib.lcp_fused_workspace_bytes(m, h, w) // 2 + 512
    assert 8 <= lib.lcp_fused_band_rows(h, w, small - (need - clib.lcp_fused_workspace_bytes(m, h, w, 0))) < h - 1
    out.fill_(float("nan"))
    assert call(uh, vh, out, 0, mask, small) == 0
    assert torch.equal(out, ref.cpu()) and torch.equal(mask, ref_mask.cpu())
    assert call(u, v, out, 0, None, need) == -1 and "pinned" in clib.lcp_last_error().decode()
    assert lib.lcp_device_status(reset=True) == 0


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_fused_host_pinned_in_place_and_pageable_staged(lib, dtype):
    """lcp_fused_host: pinned members read in place by the statistics kernel,
    pageable members through a device staging copy; both give the device-resident
    result bit for bit, with and without the mask, and again after the shape
    changes (the staging buffers are rebuilt)."""
    for h, w, m in ((61, 97, 7), (40, 33, 3)):
        d = _fields(h, w, m, seed=h + m, k=3)
        u = torch.from_numpy(d["u"]).to(dtype)
        v = torch.from_numpy(d["v"]).to(dtype)
        ref, ref_mask = lib.lcp_fused_ws(u.cuda(), v.cuda(), d["isovalues"], mask=True)
        ref, ref_mask = ref.cpu(), ref_mask.cpu()
        for pinned in (True, False):
            uh, vh = (u.pin_memory(), v.pin_memory()) if pinned else (u.clone(), v.clone())
            assert uh.is_pinned() == pinned
            mh = torch.empty(ref_mask.shape, dtype=torch.int32).pin_memory()
            out, mask = lib.lcp_fused_host(uh, vh, d["isovalues"], mask_host=mh)
            torch.cuda.synchronize()
            assert torch.equal(out, ref) and torch.equal(mask, ref_mask)
            out2, none = lib.lcp_fused_host(uh, vh, d["isovalues"])
            torch.cuda.synchronize()
            assert none is None and torch.equal(out2, ref)
    assert lib.lcp_device_status(reset=True) == 0


@pytest.mark.parametrize("n", [1, 2, 3, 7])
def test_row_strips_reassemble_the_whole_map(lib, n):
    """The multi-GPU partition run on one GPU: every strip's kept rows of
    lcp_fused_ws on its vertex rows (with the halo) equal the whole-grid map and
    mask bit for bit (the same per-vertex records and stencils)."""
    d = synth.fourier_ensemble(9, h=203, w=311, m=7, k=3)
    u, v, iso = _dev(d["u"]), _dev(d["v"]), d["isovalues"]
    whole, wmask = lib.lcp_fused_ws(u, v, iso, mask=True)
    parts = [lib.lcp_fused_strip(u, v, iso, n, r, mask=True) for r in range(n)]
    assert [p[0] for p in parts] == [lib.lcp_strip_plan(203, n, r)[2] for r in range(n)]
    assert torch.equal(torch.cat([p[1] for p in parts], dim=1), whole)
    assert torch.equal(torch.cat([p[2] for p in parts], dim=1), wmask)


def _sign_changing_field(h, w, m, seed, amp=1e4, sigma=0.05):
    """Means of magnitude amp whose sign flips across every central stencil
    (columns +, +, -, - repeating for u, rows for v; |mean| / sigma = 2e5) with
    a gentle smooth part, and Gaussian member noise sigma."""
    g = np.random.Generator(np.random.PCG64(seed))
    sx = np.array([1.0, 1.0, -1.0, -1.0])[np.arange(w) % 4]
    sy = np.array([1.0, -1.0, -1.0, 1.0])[np.arange(h) % 4]
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    mu_u = amp * sx[None, :] + 0.3 * np.sin(x / 5.0 + y / 7.0)
    mu_v = amp * sy[:, None] + 0.3 * np.cos(x / 6.0 - y / 4.0)
    u = (mu_u[None] + sigma * g.standard_normal((m, h, w))).astype(np.float32)
    v = (mu_v[None] + sigma * g.standard_normal((m, h, w))).astype(np.float32)
    return u, v


@pytest.mark.parametrize("dx,dy", [(1.0, 1.0), (0.7, 1.3)])
@pytest.mark.parametrize("k", [1, 5, 12])
def test_fused_ws_sign_changing_large_means(lib, dx, dy, k):
    """Means of 1e4 whose sign changes across the stencil (sigma = 0.05) and
    isovalues placed within a few sigma of chosen vertices' mu_d: the fp32
    difference of member-0 values would move z-scores by ~1e-2 here; the
    flagged FP64 stencil keeps the map within 1e-5 of the FP64 oracle and the
    mask exact outside the rounding guard band."""
    h, w, m = 45, 70, 12
    u, v = _sign_changing_field(h, w, m, seed=17)
    ref0 = O.lcp_closed_form(u, v, dx, dy, [0.0])
    g = np.random.Generator(np.random.PCG64(k))
    picks = g.integers(0, h * w, size=k)
    sd = np.sqrt(ref0["var_d"].reshape(-1)[picks])
    iso = (ref0["mu_d"].reshape(-1)[picks] + g.uniform(-2.0, 2.0, size=k) * sd).astype(np.float32)
    lcp, mask = lib.lcp_fused_ws(_dev(u), _dev(v), iso, dx, dy, mask=True)
    ref = O.lcp_closed_form(u, v, dx, dy, iso)
    err = np.abs(_np(lcp) - ref["lcp"])
    assert np.max(err) <= LCP_TOL, float(np.max(err))
    assert np.count_nonzero((ref["lcp"] > 1e-3) & (ref["lcp"] < 1 - 1e-3)) > 10  # the isovalues are really near mu_d
    guard = _oracle_mask_guard(ref["mu_d"], iso)
    assert np.array_equal(lib.unpack_mask(mask, w).cpu().numpy()[guard], ref["mask"][guard])
