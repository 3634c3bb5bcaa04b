"""CPU checks behind the precision design of the fused path: where the fp32
stencil is exact and where it is not."""

import numpy as np

import oracle as O


def test_sign_changing_large_means_defeat_the_plain_fp32_stencil():
    """Positive control for the GPU test of sign-changing 1e4 means: rounding
    the difference of two member-0 values of opposite sign to fp32 moves mu_d
    by up to ~5e-4, i.e. 1e-2 of sigma_d = 0.05, which is why the kernels form
    such stencils again in FP64."""
    g = np.random.Generator(np.random.PCG64(17))
    a = (1e4 + 0.3 * g.standard_normal(4096)).astype(np.float32)
    b = (-1e4 + 0.3 * g.standard_normal(4096)).astype(np.float32)
    diff32 = (a - b).astype(np.float32)
    exact = a.astype(np.float64) - b.astype(np.float64)
    err = np.max(np.abs(diff32.astype(np.float64) - exact)) * 0.5  # the central difference's 1 / (2 dx)
    assert err > 1e-4
    # ... while members within a factor of 2 (a uniform offset) subtract exactly (Sterbenz)
    c = (1e4 + 0.3 * g.standard_normal(4096)).astype(np.float32)
    assert np.array_equal((a - c).astype(np.float64), a.astype(np.float64) - c.astype(np.float64))


def test_oracle_mu_d_of_the_sign_changing_field_is_large():
    """The field of the GPU test: |mu_d| reaches 2e4 while sigma_d ~ 0.05."""
    h, w = 16, 20
    sx = np.array([1.0, 1.0, -1.0, -1.0])[np.arange(w) % 4]
    sy = np.array([1.0, -1.0, -1.0, 1.0])[np.arange(h) % 4]
    g = np.random.Generator(np.random.PCG64(3))
    u = (1e4 * sx[None, None, :] + 0.05 * g.standard_normal((8, h, w))).astype(np.float32)
    v = (1e4 * sy[None, :, None] + 0.05 * g.standard_normal((8, h, w))).astype(np.float32)
    ref = O.lcp_closed_form(u, v, 1.0, 1.0, [0.0])
    inner = ref["mu_d"][1:-1, 1:-1]
    assert np.max(np.abs(inner)) > 1.9e4
    assert np.max(np.sqrt(ref["var_d"][1:-1, 1:-1])) < 0.1
