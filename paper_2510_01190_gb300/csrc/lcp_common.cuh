// Device-side helpers shared by the kernels of liblcp_gb300 (sm_103a); the
// host-side checks and cross-file entry points are in lcp_host.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lcp.h"
#include "lcp_host.h"

namespace lcp {


// Isovalues travel by value in the launch parameters (no device copy, safe to
// capture in a CUDA graph).  Kernels take them as __grid_constant__ so that a
// runtime index reads parameter space directly.
constexpr int kMaxIsoPerLaunch = 64;
struct IsoParams {
    int K;  // isovalues in this launch
    float c[kMaxIsoPerLaunch];
};

// ---------------------------------------------------------------------------
// Element loads: VEC consecutive elements of one member row as floats
// ---------------------------------------------------------------------------
template <typename T, int VEC>
struct Loader;

template <>
struct Loader<float, 1> {
    using raw_t = float;
    static __device__ __forceinline__ raw_t load(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void cvt(const raw_t& r, float* x) { x[0] = r; }
};

template <>
struct Loader<float, 4> {
    using raw_t = float4;
    static __device__ __forceinline__ raw_t load(const float* p) {
        float4 r;
        asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                     : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                     : "l"(p));
        return r;
    }
    static __device__ __forceinline__ void cvt(const raw_t& r, float* x) {
        x[0] = r.x; x[1] = r.y; x[2] = r.z; x[3] = r.w;
    }
};

template <>
struct Loader<__nv_bfloat16, 1> {
    using raw_t = unsigned short;
    static __device__ __forceinline__ raw_t load(const __nv_bfloat16* p) {
        return __ldg(reinterpret_cast<const unsigned short*>(p));
    }
    static __device__ __forceinline__ void cvt(const raw_t& r, float* x) {
        x[0] = __uint_as_float(static_cast<uint32_t>(r) << 16);
    }
};

template <>
struct Loader<__nv_bfloat16, 8> {
    using raw_t = uint4;
    static __device__ __forceinline__ raw_t load(const __nv_bfloat16* p) {
        uint4 r;
        asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                     : "l"(p));
        return r;
    }
    static __device__ __forceinline__ void cvt(const raw_t& r, float* x) {
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            x[2 * i] = __uint_as_float(w[i] << 16);          // low half = lower address
            x[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
        }
    }
};

template <typename OutT>
__device__ __forceinline__ OutT to_out(float x);
template <>
__device__ __forceinline__ float to_out<float>(float x) { return x; }
template <>
__device__ __forceinline__ __half to_out<__half>(float x) { return __float2half_rn(x); }

// ---------------------------------------------------------------------------
// P(D < c) and P(D >= c) for D ~ N(mu, var), complementary erfc form
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// erfc(x) / 2 for x >= 0, from the Chebyshev-fitted form of Press, Teukolsky,
// Vetterling and Flannery (Numerical Recipes, 2nd ed., Sec. 6.2, "erfcc"):
//   erfc(x) ~= t exp(-x^2 + P(t)),  t = 1 / (1 + x/2),
// with P a degree-9 polynomial whose fractional error is below 1.2e-7 for all
// x >= 0, so the far tail keeps its relative accuracy.  Here the factor 1/2 is
// folded into P's constant (-1.26551223 - ln 2) and log2(e) into every
// coefficient, so that the exponential is one hardware ex2 and the reciprocal
// one hardware rcp: 2 MUFU + 13 FMA-pipe instructions.  Error budget in FP32:
// fit 1.2e-7 + ex2/rcp approximations ~3e-7 relative, plus |exponent| x 6e-8
// from rounding the exponent (which only matters where the result is tiny);
// results below 2^-126 flush to 0.  Tested against the FP64 oracle's erfc.
__device__ __forceinline__ float half_erfc_nonneg(float x) {
    constexpr float L = 1.4426950408889634f;  // log2(e)
    const float t = rcp_approx(fmaf(0.5f, x, 1.0f));
    float r = 0.17087277f * L;
    r = fmaf(r, t, -0.82215223f * L);
    r = fmaf(r, t, 1.48851587f * L);
    r = fmaf(r, t, -1.13520398f * L);
    r = fmaf(r, t, 0.27886807f * L);
    r = fmaf(r, t, -0.18628806f * L);
    r = fmaf(r, t, 0.09678418f * L);
    r = fmaf(r, t, 0.37409196f * L);
    r = fmaf(r, t, 1.00002368f * L);
    r = fmaf(r, t, -1.95865941f * L);  // (-1.26551223 - ln 2) log2(e)
    return t * ex2_approx(fmaf(-x * L, x, r));
}

// Two evaluations of half_erfc_nonneg at once with Blackwell's paired FP32
// instructions (FFMA2 / FMUL2 on float2): the same polynomial and constants,
// half the FMA-pipe instructions; the reciprocals and exponentials stay scalar.
__device__ __forceinline__ float2 half_erfc_nonneg2(float2 x) {
    constexpr float L = 1.4426950408889634f;  // log2(e)
    const float2 den = __ffma2_rn(make_float2(0.5f, 0.5f), x, make_float2(1.0f, 1.0f));
    const float2 t = make_float2(rcp_approx(den.x), rcp_approx(den.y));
    float2 r = make_float2(0.17087277f * L, 0.17087277f * L);
    r = __ffma2_rn(r, t, make_float2(-0.82215223f * L, -0.82215223f * L));
    r = __ffma2_rn(r, t, make_float2(1.48851587f * L, 1.48851587f * L));
    r = __ffma2_rn(r, t, make_float2(-1.13520398f * L, -1.13520398f * L));
    r = __ffma2_rn(r, t, make_float2(0.27886807f * L, 0.27886807f * L));
    r = __ffma2_rn(r, t, make_float2(-0.18628806f * L, -0.18628806f * L));
    r = __ffma2_rn(r, t, make_float2(0.09678418f * L, 0.09678418f * L));
    r = __ffma2_rn(r, t, make_float2(0.37409196f * L, 0.37409196f * L));
    r = __ffma2_rn(r, t, make_float2(1.00002368f * L, 1.00002368f * L));
    r = __ffma2_rn(r, t, make_float2(-1.95865941f * L, -1.95865941f * L));
    const float2 ex = __ffma2_rn(__fmul2_rn(x, make_float2(-L, -L)), x, r);
    return __fmul2_rn(t, make_float2(ex2_approx(ex.x), ex2_approx(ex.y)));
}

// Per-vertex part of (p, q): s = 1 / (sigma sqrt 2), or s = 0 marks var == 0.
struct VertexG {
    float mu, s;
};
__device__ __forceinline__ VertexG vertex_g(float mu, float var) {
    VertexG g;
    g.mu = mu;
    g.s = var == 0.0f ? 0.0f : rsqrtf(2.0f * var);  // NaN var stays NaN
    return g;
}

// t = (mu - c) / (sigma sqrt 2); p = erfc(t)/2, q = erfc(-t)/2 = 1 - p.  Only
// erfc(|t|) <= 1 is evaluated: the small one of (p, q) is that tail value
// itself (full relative accuracy) and the large one is 1 minus it, which has
// no cancellation because it lies in [1/2, 1].  var == 0 gives the indicator
// [mu < c]; a NaN mean or variance gives NaN for both.
__device__ __forceinline__ void below_above(const VertexG& g, float c, float& p, float& q) {
    if (g.s == 0.0f) {
        p = (g.mu < c) ? 1.0f : 0.0f;
        q = 1.0f - p;
        return;
    }
    const float t = (g.mu - c) * g.s;
    const float e = half_erfc_nonneg(fabsf(t));
    if (t >= 0.0f) {
        p = e;
        q = 1.0f - e;
    } else {
        q = e;
        p = 1.0f - e;
    }
}

__device__ __forceinline__ void below_above(float mu, float var, float c, float& p, float& q) {
    below_above(vertex_g(mu, var), c, p, q);
}

// (P(D < c), P(D >= c)) of a vertex (mu, s = 1/(sigma sqrt 2)); below = mu < c.
// Zero variance takes the argument +-1e4, whose erfc underflows to 0, giving the
// indicator [mu < c] (also when mu == c) without a separate branch.
__device__ __forceinline__ float2 vertex_pq(float mu, float s, bool zero, float c, bool below) {
    float t = (mu - c) * s;
    if (zero) t = below ? -1.0e4f : 1.0e4f;
    const float e = half_erfc_nonneg(fabsf(t));
    const bool pos = t >= 0.0f;  // NaN: false, and both results stay NaN
    return make_float2(pos ? e : 1.0f - e, pos ? 1.0f - e : e);
}

// vertex_pq for two isovalues (c.x, c.y) of one vertex, paired erfc.
__device__ __forceinline__ void vertex_pq2(float mu, float s, bool zero, float2 c, bool below0, bool below1,
                                           float2& pq0, float2& pq1) {
    float2 t = __fmul2_rn(__fadd2_rn(make_float2(mu, mu), make_float2(-c.x, -c.y)), make_float2(s, s));
    if (zero) {
        t.x = below0 ? -1.0e4f : 1.0e4f;
        t.y = below1 ? -1.0e4f : 1.0e4f;
    }
    const float2 e = half_erfc_nonneg2(make_float2(fabsf(t.x), fabsf(t.y)));
    const bool pos0 = t.x >= 0.0f, pos1 = t.y >= 0.0f;
    pq0 = make_float2(pos0 ? e.x : 1.0f - e.x, pos0 ? 1.0f - e.x : e.x);
    pq1 = make_float2(pos1 ? e.y : 1.0f - e.y, pos1 ? 1.0f - e.y : e.y);
}

// The same pair from d = mu - c given directly (t = d s): for a mean carried as
// hi + lo, d = (hi - c) + lo keeps the digits that hi alone cannot hold.
__device__ __forceinline__ float2 vertex_pq_d(float d, float s, bool zero, bool below) {
    float t = d * s;
    if (zero) t = below ? -1.0e4f : 1.0e4f;
    const float e = half_erfc_nonneg(fabsf(t));
    const bool pos = t >= 0.0f;
    return make_float2(pos ? e : 1.0f - e, pos ? 1.0f - e : e);
}
__device__ __forceinline__ void vertex_pq2_d(float2 d, float s, bool zero, bool below0, bool below1, float2& pq0,
                                             float2& pq1) {
    float2 t = __fmul2_rn(d, make_float2(s, s));
    if (zero) {
        t.x = below0 ? -1.0e4f : 1.0e4f;
        t.y = below1 ? -1.0e4f : 1.0e4f;
    }
    const float2 e = half_erfc_nonneg2(make_float2(fabsf(t.x), fabsf(t.y)));
    const bool pos0 = t.x >= 0.0f, pos1 = t.y >= 0.0f;
    pq0 = make_float2(pos0 ? e.x : 1.0f - e.x, pos0 ? 1.0f - e.x : e.x);
    pq1 = make_float2(pos1 ? e.y : 1.0f - e.y, pos1 ? 1.0f - e.y : e.y);
}

// Clamp to [0, 1] with NaN propagated (max.NaN / min.NaN).
__device__ __forceinline__ float clamp01_nan(float x) {
    float r;
    asm("max.NaN.f32 %0, %1, 0f00000000;" : "=f"(r) : "f"(x));
    asm("min.NaN.f32 %0, %0, 0f3F800000;" : "+f"(r));
    return r;
}

// Clamp to [0, 1] without turning NaN into a number.
__device__ __forceinline__ float clamp01(float x) {
    if (x < 0.0f) x = 0.0f;
    if (x > 1.0f) x = 1.0f;
    return x;
}

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint2 k) {
    constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;  // round multipliers
    constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;  // Weyl key increments
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kM0, x.x), lo0 = kM0 * x.x;
        const uint32_t hi1 = __umulhi(kM1, x.z), lo1 = kM1 * x.z;
        x = make_uint4(hi1 ^ x.y ^ k.x, lo1, hi0 ^ x.w ^ k.y, lo0);
        k.x += kW0;
        k.y += kW1;
    }
    return x;
}

// Uniform in (0, 1): midpoint of the 2^-24 sub-interval indexed by the top 24 bits.
__device__ __forceinline__ float uniform01(uint32_t w) {
    return (__uint2float_rn(w >> 8) + 0.5f) * 5.9604644775390625e-8f;
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
    const float r = sqrtf(-2.0f * logf(uniform01(a)));
    float s, c;
    sincospif(2.0f * uniform01(b), &s, &c);
    z0 = r * c;
    z1 = r * s;
}

}  // namespace lcp

namespace lcp {

// Stencil scale factors 1/(2 dx), 1/dx (first/last column) and their squares,
// rounded once from double.
struct Spacing {
    float sx2, sx1, sy2, sy1;      // 1/(2dx), 1/dx, 1/(2dy), 1/dy
    float sx2q, sx1q, sy2q, sy1q;  // squares
};
inline Spacing make_spacing(double dx, double dy) {
    Spacing s;
    s.sx2 = (float)(0.5 / dx); s.sx1 = (float)(1.0 / dx);
    s.sy2 = (float)(0.5 / dy); s.sy1 = (float)(1.0 / dy);
    s.sx2q = (float)(0.25 / (dx * dx)); s.sx1q = (float)(1.0 / (dx * dx));
    s.sy2q = (float)(0.25 / (dy * dy)); s.sy1q = (float)(1.0 / (dy * dy));
    return s;
}

}  // namespace lcp
