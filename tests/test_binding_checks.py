"""The Python wrappers of the NEXT-row calls reject malformed tensors before any
CUDA call (so these run without a GPU), and the product package keeps every
such call behind the library: no CPU fallback."""

import pytest
import torch

from paper_2510_01190_gb300 import _binding as B


def cpu(*shape, dtype=torch.float32):
    return torch.zeros(shape, dtype=dtype)


def test_colormap_wrapper_checks():
    with pytest.raises(ValueError):
        B.lcp_colormap(cpu(4, 4))  # not on a CUDA device
    with pytest.raises(ValueError):
        B.lcp_colormap(cpu(4, 4, dtype=torch.float64))
    with pytest.raises(ValueError):
        B.lcp_colormap(cpu(2, 3, 4, 5))


def test_volume_wrapper_checks():
    u = cpu(2, 3, 4, 5)
    with pytest.raises(ValueError):
        B.lcp3d_fused_ws(u, u, cpu(2, 3, 4, 6), [0.0])
    with pytest.raises(ValueError):
        B.lcp3d_fused_ws(u, u, u, [0.0])  # CPU tensors
    with pytest.raises(ValueError):
        B.lcp3d_divergence(*(cpu(3, 4, 5),) * 6)
    with pytest.raises(ValueError):
        B.lcp3d_map(cpu(3, 4, 5), cpu(3, 4, 5), [0.0])


def test_gradient_and_contour_wrapper_checks():
    u = cpu(2, 4, 5)
    with pytest.raises(ValueError):
        B.lcp_speed_gradient(u, u)
    with pytest.raises(ValueError):
        B.lcp_speed_gradient_ws(u, cpu(2, 4, 6), [0.0])
    with pytest.raises(ValueError):
        B.lcp_contours(cpu(4, 5), [0.0])
    with pytest.raises(ValueError):
        B.lcp_member_contours(u, u, [0.0])


def test_pack_rgba_and_default_stops():
    assert B.pack_rgba(1, 2, 3, 4) == 0x04030201
    assert B.pack_rgba(255, 0, 0) == 0xFF0000FF
    t = [s[0] for s in B.DEFAULT_STOPS]
    assert t[0] == 0.0 and t[-1] == 1.0 and all(a < b for a, b in zip(t, t[1:]))
    assert all(0.0 <= c <= 1.0 for s in B.DEFAULT_STOPS for c in s)


def test_fused_host_wrapper_checks():
    """lcp_fused_host takes host tensors [M, H, W] of one shape and dtype,
    contiguous, and checks them before any CUDA call."""
    u = cpu(3, 4, 5)
    with pytest.raises(ValueError):
        B.lcp_fused_host(u, cpu(3, 4, 6), [0.0])  # shapes differ
    with pytest.raises(ValueError):
        B.lcp_fused_host(u, cpu(3, 4, 5, dtype=torch.bfloat16), [0.0])  # dtypes differ
    with pytest.raises(ValueError):
        B.lcp_fused_host(cpu(4, 5), cpu(4, 5), [0.0])  # not [M, H, W]
    with pytest.raises(ValueError):
        B.lcp_fused_host(u.transpose(1, 2), u.transpose(1, 2), [0.0])  # not contiguous
