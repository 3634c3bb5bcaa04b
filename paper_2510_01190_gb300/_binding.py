"""ctypes binding of ``include/lcp.h``: argument marshalling only.

Every function here checks tensor shapes / dtypes / devices, allocates the
outputs with torch (device memory is plumbing), and calls the C entry point of
the same name on the current torch CUDA stream.  All arithmetic runs in the
CUDA kernels of ``liblcp_gb300.so``.  If that library cannot be loaded the call
raises; nothing falls back to the CPU.
"""

from __future__ import annotations

import ctypes
import os
import threading

import torch

__all__ = [
    "LcpError",
    "load",
    "library_path",
    "lcp_stats",
    "lcp_divergence",
    "lcp_map",
    "lcp_fused",
    "lcp_fused_ws",
    "lcp_fused_static_ws",
    "lcp_fused_workspace_bytes",
    "lcp_fused_band_rows",
    "lcp_fused_host",
    "lcp_field_desc",
    "lcp_tune",
    "lcp_batch_plan",
    "TILE_SHAPES",
    "lcp_batch_workspace_bytes",
    "lcp_batch_prepare",
    "lcp_batch",
    "lcp_batch_autotune",
    "lcp_batch_autotune_cached",
    "lcp_batch_tune_key",
    "lcp_tune_cache_lookup",
    "lcp_tune_cache_store",
    "Batch",
    "lcp_mc",
    "lcp_philox_fill",
    "lcp_exact_empirical",
    "lcp_colormap",
    "lcp_contours",
    "lcp_member_contours",
    "lcp_contours_workspace_bytes",
    "lcp3d_fused_ws",
    "lcp3d_workspace_bytes",
    "lcp3d_divergence",
    "lcp3d_map",
    "lcp_speed_gradient",
    "lcp_speed_gradient_ws",
    "DEFAULT_STOPS",
    "pack_rgba",
    "lcp_device_status",
    "lcp_set_wait_budget",
    "lcp_test_stalled_lcp_wait",
    "lcp_test_stalled_lookback",
    "lcp_strip_plan",
    "lcp_lpt_assign",
    "lcp_fused_strip",
    "mask_words_per_row",
    "unpack_mask",
    "LCP_F32",
    "LCP_BF16",
    "LCP_F16",
    "LCP_MC_GAUSS",
    "LCP_MC_EMPIRICAL",
]

LCP_F32, LCP_BF16, LCP_F16, LCP_F64 = 0, 1, 2, 3
LCP_MC_GAUSS, LCP_MC_EMPIRICAL = 0, 1

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()

c_int, c_i64, c_u64, c_u32, c_double = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
c_vp, c_fp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)


class lcp_field_desc(ctypes.Structure):
    """One field of a batch (the C struct of the same name)."""

    _fields_ = [("u", c_vp), ("v", c_vp), ("member_stride", c_i64), ("M", c_int), ("H", c_int), ("W", c_int),
                ("ddof", c_int), ("dx", c_double), ("dy", c_double), ("iso_begin", c_int), ("K", c_int),
                ("lcp_out", c_vp), ("mask", c_vp)]


class lcp_tune(ctypes.Structure):
    """Tile shape of the batch kernel (the C struct of the same name)."""

    _fields_ = [("tile_rows", c_int), ("tile_cols", c_int), ("ctas_per_sm", c_int)]


class lcp_batch_plan(ctypes.Structure):
    """A prepared batch (the C struct of the same name)."""

    _fields_ = [("workspace", c_vp), ("workspace_bytes", ctypes.c_size_t), ("n_fields", c_int), ("n_iso", c_int),
                ("in_dtype", c_int), ("out_dtype", c_int), ("cells", c_i64), ("cell_isovalues", c_i64),
                ("member_bytes", c_i64), ("out_bytes", c_i64)]


TILE_SHAPES = [(64, 64), (32, 128), (32, 64), (16, 128)]

_SIGNATURES = {
    "lcp_status_string": (ctypes.c_char_p, [c_int]),
    "lcp_last_error": (ctypes.c_char_p, []),
    "lcp_version": (c_int, []),
    "lcp_stats": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int, c_i64, c_int, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "lcp_divergence": (c_int, [c_vp, c_vp, c_vp, c_vp, c_int, c_int, c_double, c_double, c_vp, c_vp, c_vp]),
    "lcp_map": (c_int, [c_vp, c_vp, c_int, c_int, c_fp, c_int, c_vp, c_int, c_vp, c_vp]),
    "lcp_fused": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int, c_i64, c_int, c_double, c_double, c_fp, c_int,
                          c_vp, c_int, c_vp, c_vp]),
    "lcp_mc": (c_int, [c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_int, c_int, c_i64, c_int, c_int, c_double,
                       c_double, c_fp, c_int, c_i64, c_u64, c_u64, c_vp, c_vp, c_vp]),
    "lcp_philox_fill": (c_int, [c_u64, c_u32, c_u64, c_i64, c_vp, c_vp]),
    "lcp_device_status": (c_int, [ctypes.POINTER(c_u32), c_int]),
    "lcp_fused_workspace_bytes": (ctypes.c_size_t, [c_int, c_int, c_int, c_int]),
    "lcp_fused_band_rows": (c_int, [c_int, c_int, ctypes.c_size_t]),
    "lcp_fused_ws": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int, c_i64, c_int, c_double, c_double, c_fp, c_int,
                             c_vp, c_int, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "lcp_batch_workspace_bytes": (ctypes.c_size_t, [c_int, c_int]),
    "lcp_batch_prepare": (c_int, [ctypes.POINTER(lcp_field_desc), c_int, c_fp, c_int, c_int, c_int, c_vp,
                                  ctypes.c_size_t, c_vp, ctypes.POINTER(lcp_batch_plan)]),
    "lcp_batch": (c_int, [ctypes.POINTER(lcp_batch_plan), ctypes.POINTER(lcp_tune), c_vp]),
    "lcp_batch_autotune": (c_int, [ctypes.POINTER(lcp_batch_plan), c_int, ctypes.POINTER(lcp_tune), c_fp, c_vp]),
    "lcp_tune_cache_lookup": (c_int, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(lcp_tune), c_fp]),
    "lcp_tune_cache_store": (c_int, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(lcp_tune), c_fp]),
    "lcp_batch_tune_key": (c_int, [ctypes.POINTER(lcp_batch_plan), ctypes.c_char_p, ctypes.c_size_t]),
    "lcp_batch_autotune_cached": (c_int, [ctypes.POINTER(lcp_batch_plan), c_int, ctypes.c_char_p,
                                          ctypes.POINTER(lcp_tune), c_fp, ctypes.POINTER(c_int), c_vp]),
    "lcp_exact_empirical": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int, c_i64, c_double, c_double, c_fp, c_int,
                                    c_vp, c_vp, c_vp]),
    "lcp_contours_workspace_bytes": (ctypes.c_size_t, [c_int, c_int, c_int]),
    "lcp_contours": (c_int, [c_vp, c_int, c_int, c_fp, c_int, c_vp, c_vp, c_i64, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "lcp_member_contours": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int, c_i64, c_double, c_double, c_fp, c_int,
                                    c_vp, c_vp, c_i64, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "lcp3d_workspace_bytes": (ctypes.c_size_t, [c_int, c_int, c_int, c_int, c_int]),
    "lcp3d_fused_ws": (c_int, [c_vp, c_vp, c_vp, c_int, c_int, c_int, c_int, c_int, c_i64, c_int, c_double, c_double,
                               c_double, c_fp, c_int, c_vp, c_int, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "lcp3d_divergence": (c_int, [c_vp] * 6 + [c_int, c_int, c_int, c_double, c_double, c_double, c_vp, c_vp, c_vp]),
    "lcp3d_map": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_fp, c_int, c_vp, c_int, c_vp, c_vp]),
    "lcp_speed_gradient": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int, c_i64, c_double, c_double, c_vp, c_vp,
                                   c_vp]),
    "lcp_speed_gradient_ws": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int, c_i64, c_int, c_double, c_double,
                                      c_fp, c_int, c_vp, c_int, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "lcp_colormap": (c_int, [c_vp, c_int, c_int, c_int, ctypes.c_float, ctypes.c_float, c_fp, c_int, c_u32, c_vp,
                             c_u32, c_vp, c_vp]),
    "lcp_fused_static_ws": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int, c_i64, c_int, c_double, c_double, c_fp,
                                    c_int, c_vp, c_int, c_vp, c_vp]),
    "lcp_fused_host_workspace_bytes": (ctypes.c_size_t, [c_int, c_int, c_int, c_int, c_int, c_int]),
    "lcp_fused_host": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int, c_i64, c_int, c_double, c_double, c_fp, c_int,
                               c_vp, c_int, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "lcp_set_wait_budget": (ctypes.c_longlong, [ctypes.c_longlong]),
    "lcp_strip_plan": (c_int, [c_int, c_int, c_int] + [ctypes.POINTER(c_int)] * 4),
    "lcp_lpt_assign": (c_int, [ctypes.POINTER(c_i64), c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_i64)]),
    "lcp_test_stalled_lcp_wait": (c_int, [c_int, c_int, c_fp, c_int, c_vp, c_int, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "lcp_test_stalled_lookback": (c_int, [c_vp, c_int, c_int, c_fp, c_int, c_vp, c_vp, c_i64, c_vp, c_vp,
                                          ctypes.c_size_t, c_vp]),
}


class LcpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


def library_path() -> str:
    return os.path.join(_PKG, "_lib", "liblcp_gb300.so")


def load(build_if_stale: bool = True):
    """Load (building first if missing or older than its sources) the CUDA library."""
    global _LIB
    if _LIB is not None:
        return _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        from . import build as _build

        if build_if_stale and _build.is_stale():
            _build.build()
        path = library_path()
        if not os.path.exists(path):
            raise LcpError(-2, f"CUDA library missing: {path} (run paper_2510_01190_gb300.build.build())")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def _check(status: int):
    if status != 0:
        lib = load()
        msg = lib.lcp_last_error().decode() or lib.lcp_status_string(status).decode()
        raise LcpError(status, msg)


def _stream():
    return c_vp(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else c_vp(t.data_ptr())


def _dtype_code(dt) -> int:
    if dt == torch.float32:
        return LCP_F32
    if dt == torch.bfloat16:
        return LCP_BF16
    if dt == torch.float16:
        return LCP_F16
    raise ValueError(f"unsupported dtype {dt}")


def _members(u, v):
    if u.dim() != 3 or u.shape != v.shape or u.dtype != v.dtype:
        raise ValueError("u and v must be [M, H, W] tensors of one shape and dtype")
    if not (u.is_cuda and v.is_cuda):
        raise ValueError("members must be CUDA tensors")
    m, h, w = u.shape
    for t in (u, v):
        if t.stride(2) != 1 or t.stride(1) != w:
            raise ValueError("each member plane must be row-major contiguous [H][W]")
    if u.stride(0) != v.stride(0):
        raise ValueError("u and v must share one member stride")
    return m, h, w, u.stride(0) if m > 1 else h * w


def _iso(isovalues):
    iso = torch.as_tensor(isovalues, dtype=torch.float32).reshape(-1).contiguous().cpu()
    return iso, iso.numel(), ctypes.cast(iso.data_ptr(), c_fp)


def mask_words_per_row(w: int) -> int:
    return (w - 1 + 31) // 32


def _plane(t, h, w, name):
    if t.dtype != torch.float32 or not t.is_cuda or t.shape != (h, w) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor [{h}, {w}]")


def lcp_stats(u, v, ddof: int = 1, out=None):
    """Per-vertex (mean, variance) of u and v over the members (Sec. 3.1):
    (mu_u, var_u, mu_v, var_v), written into `out` (four fp32 [H][W] planes) when given."""
    m, h, w, stride = _members(u, v)
    if out is None:
        outs = [torch.empty((h, w), dtype=torch.float32, device=u.device) for _ in range(4)]
    else:
        outs = list(out)
        if len(outs) != 4:
            raise ValueError("lcp_stats: out must hold four planes (mu_u, var_u, mu_v, var_v)")
        for t, n in zip(outs, ("mu_u", "var_u", "mu_v", "var_v")):
            _plane(t, h, w, n)
    lib = load()
    _check(lib.lcp_stats(_ptr(u), _ptr(v), _dtype_code(u.dtype), m, h, w, stride, ddof, *map(_ptr, outs), _stream()))
    return tuple(outs)


def lcp_divergence(mu_u, var_u, mu_v, var_v, dx: float = 1.0, dy: float = 1.0):
    """Divergence Gaussian (Eqs. 2, 3) at every vertex: returns (mu_d, var_d)."""
    h, w = mu_u.shape
    for t, n in ((mu_u, "mu_u"), (var_u, "var_u"), (mu_v, "mu_v"), (var_v, "var_v")):
        _plane(t, h, w, n)
    mu_d = torch.empty_like(mu_u)
    var_d = torch.empty_like(mu_u)
    lib = load()
    _check(lib.lcp_divergence(_ptr(mu_u), _ptr(var_u), _ptr(mu_v), _ptr(var_v), h, w, float(dx), float(dy),
                              _ptr(mu_d), _ptr(var_d), _stream()))
    return mu_d, var_d


def _outputs(k, h, w, device, out_dtype, mask, out, mask_out):
    if out is None:
        out = torch.empty((k, h - 1, w - 1), dtype=out_dtype, device=device)
    if mask and mask_out is None:
        mask_out = torch.empty((k, h - 1, mask_words_per_row(w)), dtype=torch.int32, device=device)
    return out, (mask_out if mask else None)


def lcp_map(mu_d, var_d, isovalues, out_dtype=torch.float32, mask: bool = False, out=None, mask_out=None):
    """LCP of every cell and isovalue from the divergence Gaussians: returns (lcp, mask_words|None)."""
    h, w = mu_d.shape
    _plane(mu_d, h, w, "mu_d")
    _plane(var_d, h, w, "var_d")
    iso, k, iso_p = _iso(isovalues)
    out, mask_out = _outputs(k, h, w, mu_d.device, out_dtype, mask, out, mask_out)
    lib = load()
    _check(lib.lcp_map(_ptr(mu_d), _ptr(var_d), h, w, iso_p, k, _ptr(out), _dtype_code(out.dtype),
                       _ptr(mask_out), _stream()))
    return out, mask_out


def lcp_fused(u, v, isovalues, dx: float = 1.0, dy: float = 1.0, ddof: int = 1, out_dtype=torch.float32,
              mask: bool = False, out=None, mask_out=None):
    """Members -> LCP map in one pass (stats, Eqs. 2/3 and LCP fused): returns (lcp, mask_words|None)."""
    m, h, w, stride = _members(u, v)
    iso, k, iso_p = _iso(isovalues)
    out, mask_out = _outputs(k, h, w, u.device, out_dtype, mask, out, mask_out)
    lib = load()
    _check(lib.lcp_fused(_ptr(u), _ptr(v), _dtype_code(u.dtype), m, h, w, stride, ddof, float(dx), float(dy),
                         iso_p, k, _ptr(out), _dtype_code(out.dtype), _ptr(mask_out), _stream()))
    return out, mask_out


def lcp_fused_workspace_bytes(m: int, h: int, w: int, dtype=torch.float32) -> int:
    return int(load().lcp_fused_workspace_bytes(m, h, w, _dtype_code(dtype)))


def lcp_fused_band_rows(h: int, w: int, workspace_bytes: int) -> int:
    """Cell rows per band of ``lcp_fused_ws`` for an h x w grid and that many
    workspace bytes (h - 1: one band); 0 when the workspace is too small.
    Host arithmetic only."""
    return int(load().lcp_fused_band_rows(h, w, workspace_bytes))


_WS = {}


def _workspace(nbytes: int, device):
    key = (str(device), torch.cuda.current_stream(device).cuda_stream)
    buf = _WS.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        _WS[key] = buf
    off = (-buf.data_ptr()) % 256
    return buf, buf.data_ptr() + off


def lcp_fused_ws(u, v, isovalues, dx: float = 1.0, dy: float = 1.0, ddof: int = 1, out_dtype=torch.float32,
                 mask: bool = False, out=None, mask_out=None, workspace=None):
    """``lcp_fused`` through the persistent dataflow kernel, with a device
    workspace (a uint8 CUDA tensor, 256-byte aligned, ideally of
    ``lcp_fused_workspace_bytes``: a smaller one runs smaller row bands; by
    default one cached per device and stream).  Returns (lcp, mask_words|None)."""
    m, h, w, stride = _members(u, v)
    iso, k, iso_p = _iso(isovalues)
    out, mask_out = _outputs(k, h, w, u.device, out_dtype, mask, out, mask_out)
    lib = load()
    need = int(lib.lcp_fused_workspace_bytes(m, h, w, _dtype_code(u.dtype)))
    if workspace is None:
        _, ws_ptr = _workspace(need, u.device)
        ws_bytes = need
    else:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    _check(lib.lcp_fused_ws(_ptr(u), _ptr(v), _dtype_code(u.dtype), m, h, w, stride, ddof, float(dx), float(dy),
                            iso_p, k, _ptr(out), _dtype_code(out.dtype), _ptr(mask_out), c_vp(ws_ptr), ws_bytes,
                            _stream()))
    return out, mask_out


def lcp_fused_static_ws(u, v, isovalues, dx: float = 1.0, dy: float = 1.0, ddof: int = 1, out_dtype=torch.float32,
                        mask: bool = False, out=None, mask_out=None):
    """``lcp_fused_ws`` with the library's fixed 64 MiB device scratch: the C
    call allocates nothing (pass ``out``/``mask_out`` to keep this wrapper from
    allocating them).  Calls on one device must not overlap in time.
    Returns (lcp, mask_words|None)."""
    m, h, w, stride = _members(u, v)
    iso, k, iso_p = _iso(isovalues)
    out, mask_out = _outputs(k, h, w, u.device, out_dtype, mask, out, mask_out)
    _check(load().lcp_fused_static_ws(_ptr(u), _ptr(v), _dtype_code(u.dtype), m, h, w, stride, ddof, float(dx),
                                      float(dy), iso_p, k, _ptr(out), _dtype_code(out.dtype), _ptr(mask_out),
                                      _stream()))
    return out, mask_out


def lcp_speed_gradient(u, v, dx: float = 1.0, dy: float = 1.0):
    """Gradient of every member's velocity magnitude (Sec. 4.2 preprocessing):
    returns (gx, gy), float32 [M, H, W]."""
    m, h, w, stride = _members(u, v)
    gx = torch.empty((m, h, w), dtype=torch.float32, device=u.device)
    gy = torch.empty_like(gx)
    _check(load().lcp_speed_gradient(_ptr(u), _ptr(v), _dtype_code(u.dtype), m, h, w, stride, float(dx), float(dy),
                                     _ptr(gx), _ptr(gy), _stream()))
    return gx, gy


def lcp_speed_gradient_ws(u, v, isovalues, dx: float = 1.0, dy: float = 1.0, ddof: int = 1,
                          out_dtype=torch.float32, mask: bool = False, out=None, mask_out=None, workspace=None):
    """LCP map of the divergence of the members' speed gradients, the
    preprocessing fused into the statistics pass (Sec. 4.2, Fig. 3d).
    Returns (lcp, mask_words|None)."""
    m, h, w, stride = _members(u, v)
    iso, k, iso_p = _iso(isovalues)
    out, mask_out = _outputs(k, h, w, u.device, out_dtype, mask, out, mask_out)
    lib = load()
    need = int(lib.lcp_fused_workspace_bytes(m, h, w, _dtype_code(u.dtype)))
    if workspace is None:
        _, ws_ptr = _workspace(need, u.device)
        ws_bytes = need
    else:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    _check(lib.lcp_speed_gradient_ws(_ptr(u), _ptr(v), _dtype_code(u.dtype), m, h, w, stride, ddof, float(dx),
                                     float(dy), iso_p, k, _ptr(out), _dtype_code(out.dtype), _ptr(mask_out),
                                     c_vp(ws_ptr), ws_bytes, _stream()))
    return out, mask_out


def _members3(u, v, w):
    if u.dim() != 4 or u.shape != v.shape or u.shape != w.shape or u.dtype != v.dtype or u.dtype != w.dtype:
        raise ValueError("u, v and w must be [M, D, H, W] tensors of one shape and dtype")
    if not (u.is_cuda and v.is_cuda and w.is_cuda):
        raise ValueError("members must be CUDA tensors")
    m, d, h, wd = u.shape
    for t in (u, v, w):
        if t.stride(3) != 1 or t.stride(2) != wd or t.stride(1) != h * wd:
            raise ValueError("each member volume must be contiguous [D][H][W]")
    if u.stride(0) != v.stride(0) or u.stride(0) != w.stride(0):
        raise ValueError("u, v and w must share one member stride")
    return m, d, h, wd, u.stride(0) if m > 1 else d * h * wd


def lcp3d_workspace_bytes(m: int, d: int, h: int, w: int, dtype=torch.float32) -> int:
    return int(load().lcp3d_workspace_bytes(m, d, h, w, _dtype_code(dtype)))


def lcp3d_fused_ws(u, v, w, isovalues, dx: float = 1.0, dy: float = 1.0, dz: float = 1.0, ddof: int = 1,
                   out_dtype=torch.float32, mask: bool = False, out=None, mask_out=None, workspace=None):
    """3D members [M, D, H, W] of (u, v, w) -> LCP map [K, D-1, H-1, W-1] of the
    hexahedral cells (and mean-field mask words [K, D-1, H-1, ceil((W-1)/32)]).
    Returns (lcp, mask_words|None)."""
    m, d, h, wd, stride = _members3(u, v, w)
    iso, k, iso_p = _iso(isovalues)
    if out is None:
        out = torch.empty((k, d - 1, h - 1, wd - 1), dtype=out_dtype, device=u.device)
    if mask and mask_out is None:
        mask_out = torch.empty((k, d - 1, h - 1, mask_words_per_row(wd)), dtype=torch.int32, device=u.device)
    mask_out = mask_out if mask else None
    lib = load()
    need = int(lib.lcp3d_workspace_bytes(m, d, h, wd, _dtype_code(u.dtype)))
    if workspace is None:
        _, ws_ptr = _workspace(need, u.device)
        ws_bytes = need
    else:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    _check(lib.lcp3d_fused_ws(_ptr(u), _ptr(v), _ptr(w), _dtype_code(u.dtype), m, d, h, wd, stride, ddof,
                              float(dx), float(dy), float(dz), iso_p, k, _ptr(out), _dtype_code(out.dtype),
                              _ptr(mask_out), c_vp(ws_ptr), ws_bytes, _stream()))
    return out, mask_out


def lcp3d_divergence(mu_u, var_u, mu_v, var_v, mu_w, var_w, dx: float = 1.0, dy: float = 1.0, dz: float = 1.0):
    """3D divergence Gaussian at every vertex from fp32 [D, H, W] statistics: returns (mu_d, var_d)."""
    shape = mu_u.shape
    for t in (mu_u, var_u, mu_v, var_v, mu_w, var_w):
        if t.dtype != torch.float32 or not t.is_cuda or t.shape != shape or not t.is_contiguous() or t.dim() != 3:
            raise ValueError("statistics must be contiguous float32 CUDA tensors [D, H, W] of one shape")
    mu_d, var_d = torch.empty_like(mu_u), torch.empty_like(mu_u)
    d, h, w = shape
    _check(load().lcp3d_divergence(*map(_ptr, (mu_u, var_u, mu_v, var_v, mu_w, var_w)), d, h, w, float(dx),
                                   float(dy), float(dz), _ptr(mu_d), _ptr(var_d), _stream()))
    return mu_d, var_d


def lcp3d_map(mu_d, var_d, isovalues, out_dtype=torch.float32, mask: bool = False):
    """LCP of every hexahedral cell from the divergence Gaussians [D, H, W]:
    returns (lcp [K, D-1, H-1, W-1], mask_words|None)."""
    for t in (mu_d, var_d):
        if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 3 or not t.is_contiguous() or t.shape != mu_d.shape:
            raise ValueError("mu_d and var_d must be contiguous float32 CUDA tensors [D, H, W]")
    d, h, w = mu_d.shape
    iso, k, iso_p = _iso(isovalues)
    out = torch.empty((k, d - 1, h - 1, w - 1), dtype=out_dtype, device=mu_d.device)
    mask_out = torch.empty((k, d - 1, h - 1, mask_words_per_row(w)), dtype=torch.int32, device=mu_d.device) \
        if mask else None
    _check(load().lcp3d_map(_ptr(mu_d), _ptr(var_d), d, h, w, iso_p, k, _ptr(out), _dtype_code(out.dtype),
                            _ptr(mask_out), _stream()))
    return out, mask_out


def lcp_contours_workspace_bytes(m: int, h: int, w: int) -> int:
    return int(load().lcp_contours_workspace_bytes(m, h, w))


def _contour_call(launch, m, h, w, k, device, capacity, keys, out):
    """Run a contour call; with capacity None, estimate, then re-run once if short."""
    lib = load()
    need = int(lib.lcp_contours_workspace_bytes(m, h, w))
    ws, ws_ptr = _workspace(need, device)
    count = torch.zeros(1, dtype=torch.int64, device=device)
    cap = capacity if capacity is not None else max(1024, m * (h - 1) * (w - 1) * k // 8)
    while True:
        if out is not None and capacity is not None:
            seg, key = out
        else:
            seg = torch.empty((cap, 4), dtype=torch.float32, device=device)
            key = torch.empty(cap, dtype=torch.int64, device=device) if keys else None
        _check(launch(_ptr(seg), _ptr(key), cap, _ptr(count), c_vp(ws_ptr), need))
        total = int(count.item())
        if capacity is not None or total <= cap:
            n = min(total, cap)
            return seg[:n], (key[:n] if key is not None else None), total
        cap = total


def lcp_contours(field, isovalues, capacity=None, keys: bool = True, out=None):
    """Isocontour segments of a scalar field (float32 CUDA [H, W], e.g. mu_d)
    in key order: returns (seg [n, 4] float32 (x0, y0, x1, y1), key [n] int64 or
    None, total).  With ``capacity`` given, at most that many are stored (and
    ``out`` = (seg, key) may supply the buffers); total is always the full count."""
    if field.dtype != torch.float32 or not field.is_cuda or field.dim() != 2 or not field.is_contiguous():
        raise ValueError("field must be a contiguous float32 CUDA tensor [H, W]")
    h, w = field.shape
    iso, k, iso_p = _iso(isovalues)

    def launch(seg, key, cap, count, ws, nbytes):
        return load().lcp_contours(_ptr(field), h, w, iso_p, k, seg, key, cap, count, ws, nbytes, _stream())

    return _contour_call(launch, 1, h, w, k, field.device, capacity, keys, out)


def lcp_member_contours(u, v, isovalues, dx: float = 1.0, dy: float = 1.0, capacity=None, keys: bool = True,
                        out=None):
    """Spaghetti plot: isocontour segments of every member's divergence (fp32,
    fixed operation order), in key order.  Returns (seg, key|None, total)."""
    m, h, w, stride = _members(u, v)
    iso, k, iso_p = _iso(isovalues)

    def launch(seg, key, cap, count, ws, nbytes):
        return load().lcp_member_contours(_ptr(u), _ptr(v), _dtype_code(u.dtype), m, h, w, stride, float(dx),
                                          float(dy), iso_p, k, seg, key, cap, count, ws, nbytes, _stream())

    return _contour_call(launch, m, h, w, k, u.device, capacity, keys, out)


# Device buffers of ``lcp_fused_host``, one set per (device, stream), reused
# while the shape, dtype, isovalue count, mask flag and input mode stay the same:
# calls on one stream are ordered, so they may share them; other streams get
# their own.
_STAGING = {}


def lcp_fused_host(u_host, v_host, isovalues, dx: float = 1.0, dy: float = 1.0, ddof: int = 1,
                   out_host=None, mask_host=None, device="cuda"):
    """End-to-end call for host-resident ensembles [M, H, W] (fp32 or bf16),
    through the C entry point ``lcp_fused_host``: pinned members are read in
    place by the statistics kernel over the CPU-GPU link, each byte once, and
    the LCP map (and the mask words, if ``mask_host`` is given) is copied by the
    library into the host outputs, all on the current stream.  Pageable members
    (which the device cannot address) are first copied into device buffers
    here.  Returns (out_host, mask_host); the results are complete, and the
    members may be changed again, once the stream is synchronised."""
    if u_host.is_cuda or v_host.is_cuda:
        raise ValueError("lcp_fused_host takes host tensors")
    if u_host.dim() != 3 or u_host.shape != v_host.shape or u_host.dtype != v_host.dtype:
        raise ValueError("u and v must be [M, H, W] host tensors of one shape and dtype")
    if not (u_host.is_contiguous() and v_host.is_contiguous()):
        raise ValueError("host members must be contiguous [M][H][W]")
    m, h, w = u_host.shape
    iso, k, iso_p = _iso(isovalues)
    dev = torch.device(device)
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    in_place = u_host.is_pinned() and v_host.is_pinned()
    if out_host is None:
        out_host = torch.empty((k, h - 1, w - 1), dtype=torch.float32, pin_memory=True)
    if tuple(out_host.shape) != (k, h - 1, w - 1) or out_host.dtype != torch.float32 or not out_host.is_contiguous():
        raise ValueError("out_host must be a contiguous fp32 [K, H-1, W-1] tensor")
    if mask_host is not None and (tuple(mask_host.shape) != (k, h - 1, mask_words_per_row(w))
                                  or mask_host.dtype != torch.int32 or not mask_host.is_contiguous()):
        raise ValueError("mask_host must be a contiguous int32 [K, H-1, ceil((W-1)/32)] tensor")
    if in_place:
        ud, vd = u_host, v_host
    else:  # device staging of pageable members, kept per device and stream
        slot = (str(dev), torch.cuda.current_stream(dev).cuda_stream)
        key = (tuple(u_host.shape), u_host.dtype)
        cached = _STAGING.get(slot)
        if cached is None or cached[0] != key:
            cached = (key, (torch.empty_like(u_host, device=dev), torch.empty_like(v_host, device=dev)))
            _STAGING[slot] = cached
        ud, vd = cached[1]
        ud.copy_(u_host, non_blocking=True)
        vd.copy_(v_host, non_blocking=True)
    lib = load()
    code = _dtype_code(u_host.dtype)
    need = int(lib.lcp_fused_host_workspace_bytes(m, h, w, k, LCP_F32, int(mask_host is not None)))
    with torch.cuda.device(dev):
        _, ws_ptr = _workspace(need, dev)
        _check(lib.lcp_fused_host(c_vp(ud.data_ptr()), c_vp(vd.data_ptr()), code, m, h, w, h * w, ddof, float(dx),
                                  float(dy), iso_p, k, c_vp(out_host.data_ptr()), LCP_F32,
                                  c_vp(mask_host.data_ptr()) if mask_host is not None else None, c_vp(ws_ptr), need,
                                  _stream()))
    return out_host, mask_host


def lcp_mc(isovalues, n_samples: int, seed: int, dx: float = 1.0, dy: float = 1.0, mode: str = "gauss",
           stats=None, members=None, offset: int = 0, estimate: bool = True, counts=None):
    """Monte Carlo LCP (Sec. 3.2, Sec. 4): returns (estimate|None, counts uint32-as-int32)."""
    iso, k, iso_p = _iso(isovalues)
    if mode == "gauss":
        mu_u, var_u, mu_v, var_v = stats
        h, w = mu_u.shape
        for t, n in ((mu_u, "mu_u"), (var_u, "var_u"), (mu_v, "mu_v"), (var_v, "var_v")):
            _plane(t, h, w, n)
        dev = mu_u.device
        args = (LCP_MC_GAUSS, _ptr(mu_u), _ptr(var_u), _ptr(mu_v), _ptr(var_v), None, None, LCP_F32, 0, 0)
    elif mode == "empirical":
        u, v = members
        m, h, w, stride = _members(u, v)
        dev = u.device
        args = (LCP_MC_EMPIRICAL, None, None, None, None, _ptr(u), _ptr(v), _dtype_code(u.dtype), m, stride)
    else:
        raise ValueError(mode)
    if counts is None:
        counts = torch.empty((k, h - 1, w - 1), dtype=torch.int32, device=dev)
    est = torch.empty((k, h - 1, w - 1), dtype=torch.float32, device=dev) if estimate else None
    lib = load()
    _check(lib.lcp_mc(*args, h, w, float(dx), float(dy), iso_p, k, int(n_samples), int(seed) & (2**64 - 1),
                      int(offset) & (2**64 - 1), _ptr(counts), _ptr(est), _stream()))
    return est, counts


def lcp_exact_empirical(u, v, isovalues, dx: float = 1.0, dy: float = 1.0, out=None, below=None):
    """Exact LCP under the empirical model (cells with four interior vertices;
    NaN elsewhere): fp32 [K, H-1, W-1]; also returns P(D < c) [K, H, W]."""
    m, h, w, stride = _members(u, v)
    iso, k, iso_p = _iso(isovalues)
    if out is None:
        out = torch.empty((k, h - 1, w - 1), dtype=torch.float32, device=u.device)
    if below is None:
        below = torch.empty((k, h, w), dtype=torch.float32, device=u.device)
    _check(load().lcp_exact_empirical(_ptr(u), _ptr(v), _dtype_code(u.dtype), m, h, w, stride, float(dx), float(dy),
                                      iso_p, k, _ptr(below), _ptr(out), _stream()))
    return out, below


def lcp_philox_fill(seed: int, c1: int, offset: int, count: int, device="cuda"):
    """Raw Philox-4x32-10 words of the Monte Carlo generator: uint32-as-int32 [count, 4]."""
    out = torch.empty((count, 4), dtype=torch.int32, device=device)
    lib = load()
    _check(lib.lcp_philox_fill(int(seed) & (2**64 - 1), int(c1) & 0xFFFFFFFF, int(offset) & (2**64 - 1), int(count),
                               _ptr(out), _stream()))
    return out


def lcp_device_status(reset: bool = False) -> int:
    """The library's device status word (bit 0: a bounded device wait gave up).  Synchronising."""
    flags = c_u32(0)
    status = load().lcp_device_status(ctypes.byref(flags), int(reset))
    if status not in (0, -4):
        _check(status)
    return int(flags.value)


def lcp_set_wait_budget(cycles: int) -> int:
    """Clock-cycle budget of the bounded device waits that take it (0 restores
    the default, ~2 s); returns the previous budget."""
    return int(load().lcp_set_wait_budget(int(cycles)))


def lcp_test_stalled_lcp_wait(h: int, w: int, isovalues, out, mask_out=None, workspace=None):
    """Failure-path probe: the LCP kernels of the workspace path waiting on
    statistics counters that nothing releases (``out`` float32/float16
    [K, H-1, W-1], ``mask_out`` int32 words or None)."""
    iso, k, iso_p = _iso(isovalues)
    lib = load()
    need = int(lib.lcp_fused_workspace_bytes(1, h, w, LCP_F32))
    if workspace is None:
        _, ws_ptr = _workspace(need, out.device)
        ws_bytes = need
    else:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    _check(lib.lcp_test_stalled_lcp_wait(h, w, iso_p, k, _ptr(out), _dtype_code(out.dtype), _ptr(mask_out),
                                         c_vp(ws_ptr), ws_bytes, _stream()))
    return out, mask_out


def lcp_test_stalled_lookback(field, isovalues, capacity: int):
    """Failure-path probe: lcp_contours with tile 0 never run, so the next
    tile's look-back waits for a flag nothing sets.  Returns (seg, key, total)."""
    h, w = field.shape
    iso, k, iso_p = _iso(isovalues)

    def launch(seg, key, cap, count, ws, nbytes):
        return load().lcp_test_stalled_lookback(_ptr(field), h, w, iso_p, k, seg, key, cap, count, ws, nbytes,
                                                _stream())

    return _contour_call(launch, 1, h, w, k, field.device, capacity, True, None)


def lcp_strip_plan(h: int, nranks: int, rank: int):
    """Row strip of one rank (host arithmetic, no GPU needed): returns
    (vrow_begin, vrow_end, cell_begin, cell_end); the rank evaluates vertex rows
    [vrow_begin, vrow_end) as a grid of their own and keeps its cell rows
    [cell_begin - vrow_begin, cell_end - vrow_begin)."""
    out = [c_int(0) for _ in range(4)]
    _check(load(build_if_stale=False).lcp_strip_plan(int(h), int(nranks), int(rank), *[ctypes.byref(o) for o in out]))
    return tuple(int(o.value) for o in out)


def lcp_lpt_assign(costs, nranks: int):
    """Whole fields to ranks, largest first to the least-loaded rank (host
    arithmetic): returns (owner list, per-rank load list)."""
    n = len(costs)
    c = (c_i64 * max(n, 1))(*[int(x) for x in costs])
    owner = (c_int * max(n, 1))()
    ld = (c_i64 * nranks)()
    _check(load(build_if_stale=False).lcp_lpt_assign(c, n, int(nranks), owner, ld))
    return [int(owner[i]) for i in range(n)], [int(ld[r]) for r in range(nranks)]


def lcp_fused_strip(u, v, isovalues, nranks: int, rank: int, dx: float = 1.0, dy: float = 1.0, ddof: int = 1,
                    mask: bool = False):
    """This rank's strip of the LCP map of the field (u, v) [M, H, W]: the
    kept cell rows [cell_begin, cell_end) of lcp_fused_ws run on the strip's
    vertex rows (a view: no copy).  Returns (cell_begin, lcp [K, rows, W-1],
    mask words or None)."""
    m, h, w, stride = _members(u, v)
    vb, ve, cb, ce = lcp_strip_plan(h, nranks, rank)
    k = len(_iso(isovalues)[0])
    if cb == ce:
        empty = torch.empty((k, 0, w - 1), dtype=torch.float32, device=u.device)
        return cb, empty, (torch.empty((k, 0, mask_words_per_row(w)), dtype=torch.int32, device=u.device) if mask else None)
    lcp, words = lcp_fused_ws(u[:, vb:ve], v[:, vb:ve], isovalues, dx, dy, ddof, mask=mask)
    keep = slice(cb - vb, ce - vb)
    return cb, lcp[:, keep], (words[:, keep] if mask else None)


def lcp_batch_workspace_bytes(n_fields: int, n_iso: int) -> int:
    return int(load().lcp_batch_workspace_bytes(n_fields, n_iso))


def lcp_batch_prepare(descs, iso, in_dtype, out_dtype, workspace, stream=None) -> lcp_batch_plan:
    """Validate a list of ``lcp_field_desc`` and write the work table into
    ``workspace`` (a uint8 CUDA tensor); returns the plan.  Synchronising."""
    arr = (lcp_field_desc * len(descs))(*descs)
    iso_t = torch.as_tensor(iso, dtype=torch.float32).reshape(-1).contiguous().cpu()
    plan = lcp_batch_plan()
    off = (-workspace.data_ptr()) % 256
    _check(load().lcp_batch_prepare(arr, len(descs), ctypes.cast(iso_t.data_ptr(), c_fp), iso_t.numel(),
                                    _dtype_code(in_dtype), _dtype_code(out_dtype), c_vp(workspace.data_ptr() + off),
                                    workspace.numel() - off, stream if stream is not None else _stream(),
                                    ctypes.byref(plan)))
    return plan


def lcp_batch(plan: lcp_batch_plan, tune=None, stream=None):
    """One persistent launch over every field of ``plan`` (``tune`` = (rows, cols) or lcp_tune)."""
    t = None
    if tune is not None:
        t = tune if isinstance(tune, lcp_tune) else lcp_tune(int(tune[0]), int(tune[1]), 0)
    _check(load().lcp_batch(ctypes.byref(plan), ctypes.byref(t) if t is not None else None,
                            stream if stream is not None else _stream()))


def lcp_batch_autotune(plan: lcp_batch_plan, reps: int = 3, stream=None):
    """Time every tile shape on the plan; returns ((rows, cols), [ms per shape])."""
    best = lcp_tune()
    ms = (ctypes.c_float * len(TILE_SHAPES))()
    _check(load().lcp_batch_autotune(ctypes.byref(plan), int(reps), ctypes.byref(best),
                                     ctypes.cast(ms, c_fp), stream if stream is not None else _stream()))
    return (best.tile_rows, best.tile_cols), [float(x) for x in ms]


def _path_bytes(path):
    return None if path is None else os.fsencode(path)


def lcp_tune_cache_lookup(path, key: str):
    """The cached (tile, ms) of ``key`` in the JSON tune cache at ``path``, or None."""
    best = lcp_tune()
    ms = (ctypes.c_float * len(TILE_SHAPES))()
    r = load().lcp_tune_cache_lookup(_path_bytes(path), key.encode(), ctypes.byref(best), ctypes.cast(ms, c_fp))
    if r < 0:
        _check(r)
    return ((best.tile_rows, best.tile_cols), [float(x) for x in ms]) if r == 1 else None


def lcp_tune_cache_store(path, key: str, tile, ms=None):
    """Add or replace ``key``'s entry (tile (rows, cols), optional 4 times) in the tune cache."""
    best = lcp_tune(int(tile[0]), int(tile[1]), 0)
    arr = None
    if ms is not None:
        if len(ms) != len(TILE_SHAPES):
            raise ValueError(f"ms must hold {len(TILE_SHAPES)} times")
        arr = ctypes.cast((ctypes.c_float * len(TILE_SHAPES))(*[float(x) for x in ms]), c_fp)
    _check(load().lcp_tune_cache_store(_path_bytes(path), key.encode(), ctypes.byref(best), arr))


def lcp_batch_tune_key(plan: lcp_batch_plan) -> str:
    """The tune-cache key of ``plan`` on the current device."""
    buf = ctypes.create_string_buffer(512)
    n = load().lcp_batch_tune_key(ctypes.byref(plan), buf, len(buf))
    if n < 0:
        _check(n)
    return buf.value.decode()


def lcp_batch_autotune_cached(plan: lcp_batch_plan, reps: int = 3, cache_path=None, stream=None):
    """lcp_batch_autotune through the JSON tune cache at ``cache_path`` (None: $LCP_TUNE_CACHE,
    else no cache).  Returns ((rows, cols), [ms per shape], from_cache)."""
    best = lcp_tune()
    ms = (ctypes.c_float * len(TILE_SHAPES))()
    hit = c_int(0)
    _check(load().lcp_batch_autotune_cached(ctypes.byref(plan), int(reps), _path_bytes(cache_path), ctypes.byref(best),
                                            ctypes.cast(ms, c_fp), ctypes.byref(hit),
                                            stream if stream is not None else _stream()))
    return (best.tile_rows, best.tile_cols), [float(x) for x in ms], bool(hit.value)


class Batch:
    """Many fields evaluated by one persistent launch.

    ``fields``: list of dict(u, v, isovalues[, dx, dy]) with u, v CUDA tensors
    [M, H, W] of one dtype (fp32 or bf16).  Allocates each field's outputs
    (``lcp[f]`` [K, H-1, W-1] of ``out_dtype``; ``mask[f]`` words or None) and
    the device workspace, and prepares the plan.  ``run()`` is capturable into
    a CUDA graph once it has run outside capture.
    """

    def __init__(self, fields, out_dtype=torch.float32, mask: bool = False, ddof: int = 1):
        if not fields:
            raise ValueError("a batch needs at least one field")
        dt = fields[0]["u"].dtype
        dev = fields[0]["u"].device
        self.fields = fields
        self.lcp, self.mask, descs, iso = [], [], [], []
        for f in fields:
            u, v = f["u"], f["v"]
            if u.dtype != dt:
                raise ValueError("all fields of a batch share one member dtype")
            m, h, w, stride = _members(u, v)
            k = len(f["isovalues"])
            out = torch.empty((k, h - 1, w - 1), dtype=out_dtype, device=dev)
            mw = torch.zeros((k, h - 1, mask_words_per_row(w)), dtype=torch.int32, device=dev) if mask else None
            descs.append(lcp_field_desc(u.data_ptr(), v.data_ptr(), stride, m, h, w, ddof, float(f.get("dx", 1.0)),
                                        float(f.get("dy", 1.0)), len(iso), k, out.data_ptr(),
                                        mw.data_ptr() if mw is not None else None))
            iso.extend(float(c) for c in f["isovalues"])
            self.lcp.append(out)
            self.mask.append(mw)
        nbytes = lcp_batch_workspace_bytes(len(descs), len(iso))
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        self.plan = lcp_batch_prepare(descs, iso, dt, out_dtype, self.workspace)

    def run(self, tune=None):
        lcp_batch(self.plan, tune)
        return self.lcp, self.mask

    def autotune(self, reps: int = 3, cache_path=None):
        """The fastest tile shape and every shape's time; with ``cache_path`` (or
        $LCP_TUNE_CACHE) through the JSON tune cache (a hit times nothing)."""
        if cache_path is None and not os.environ.get("LCP_TUNE_CACHE"):
            return lcp_batch_autotune(self.plan, reps)
        tile, ms, _ = lcp_batch_autotune_cached(self.plan, reps, cache_path)
        return tile, ms


def unpack_mask(mask_words, w: int):
    """Expand mask words [K, H-1, ceil((W-1)/32)] to bool [K, H-1, W-1] (bit i % 32 of word i / 32)."""
    words = mask_words.to(torch.int64) & 0xFFFFFFFF
    shifts = torch.arange(32, device=words.device, dtype=torch.int64)
    bits = (words[..., None] >> shifts) & 1
    return bits.reshape(*words.shape[:-1], -1)[..., : w - 1].to(torch.bool)


# ---------------------------------------------------------------------------
# Colour mapping into a headless RGBA8 buffer
# ---------------------------------------------------------------------------
# (t, r, g, b, a): dark blue -> blue -> cyan -> yellow -> red -> dark red, the
# usual rainbow ramp for divergence and probability maps (sinks blue, sources red)
DEFAULT_STOPS = [
    (0.0, 0.0, 0.0, 0.5, 1.0),
    (0.125, 0.0, 0.0, 1.0, 1.0),
    (0.375, 0.0, 1.0, 1.0, 1.0),
    (0.625, 1.0, 1.0, 0.0, 1.0),
    (0.875, 1.0, 0.0, 0.0, 1.0),
    (1.0, 0.5, 0.0, 0.0, 1.0),
]


def pack_rgba(r: int, g: int, b: int, a: int = 255) -> int:
    """Packed colour word r | g << 8 | b << 16 | a << 24 of ``lcp_colormap``."""
    return (int(r) & 255) | ((int(g) & 255) << 8) | ((int(b) & 255) << 16) | ((int(a) & 255) << 24)


def lcp_colormap(values, vmin: float = 0.0, vmax: float = 1.0, stops=None, nan_rgba: int = 0, mask=None,
                 mask_rgba: int = 0xFF000000, out=None):
    """RGBA8 image of a scalar map (``[rows, cols]`` or ``[planes, rows, cols]``
    float32 CUDA tensor, e.g. an LCP map): returns uint8 ``[..., rows, cols, 4]``.
    ``mask`` is the library's crossing-mask words for those cells (as returned by
    ``lcp_fused(..., mask=True)``); set bits paint ``mask_rgba``."""
    if values.dtype != torch.float32 or not values.is_cuda or not values.is_contiguous() or values.dim() not in (2, 3):
        raise ValueError("values must be a contiguous float32 CUDA tensor [rows, cols] or [planes, rows, cols]")
    planes, rows, cols = (1, *values.shape) if values.dim() == 2 else tuple(values.shape)
    st = torch.as_tensor(stops if stops is not None else DEFAULT_STOPS, dtype=torch.float32).reshape(-1).contiguous()
    if st.numel() % 5:
        raise ValueError("stops must be rows of (t, r, g, b, a)")
    if mask is not None:
        nw = (cols + 31) // 32
        if mask.dtype != torch.int32 or not mask.is_cuda or not mask.is_contiguous() or mask.numel() != planes * rows * nw:
            raise ValueError(f"mask must be contiguous int32 CUDA words [{planes}, {rows}, {nw}]")
    if out is None:
        out = torch.empty(tuple(values.shape) + (4,), dtype=torch.uint8, device=values.device)
    elif out.dtype != torch.uint8 or out.numel() != values.numel() * 4 or not out.is_contiguous():
        raise ValueError("out must be a contiguous uint8 tensor with 4 bytes per value")
    _check(load().lcp_colormap(_ptr(values), planes, rows, cols, float(vmin), float(vmax),
                               ctypes.cast(st.data_ptr(), c_fp), st.numel() // 5, int(nan_rgba) & 0xFFFFFFFF,
                               _ptr(mask), int(mask_rgba) & 0xFFFFFFFF, _ptr(out), _stream()))
    return out
