// Speed-gradient preprocessing (Sec. 4.2, Red Sea): per member the velocity
// magnitude s = sqrt(u^2 + v^2) and its gradient (ds/dx, ds/dy) with the
// stencil of Eq. 1 (central inside, first-order one-sided at the ends); the
// gradient vectors are the ensemble whose divergence LCP is mapped.
//
// lcp_speed_gradient_ws fuses the preprocessing into the statistics pass:
// grad_stats_kernel reads every member value once, forms the speeds of a warp
// tile (30 vertex columns + one halo column each side, 8 vertex rows + one
// halo row each side) in registers, takes the x differences by warp shuffle and
// the y differences down the thread's own rows, and accumulates the shifted
// sums of both gradient components over the members.  It writes the same
// 16-byte records as the statistics stream of lcp_fused_ws into the same
// L2-resident band workspace, whose LCP kernels then run unchanged.  No
// gradient member ever reaches HBM.
//
// lcp_speed_gradient writes the gradient members themselves (fp32), for any
// other entry point (Monte Carlo, the exact empirical judge) or for checking.
#include <algorithm>
#include <cmath>

#include "lcp_common.cuh"

namespace lcp {
namespace {

constexpr int kGW = 8;          // warps per block
constexpr int kGR = 8;          // vertex rows per warp tile
constexpr int kGC = 30;         // vertex columns per warp tile (lanes 1..30; lanes 0 and 31 load the halo)
constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ float ldm(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldm(const __nv_bfloat16* p) {
    return __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p)) << 16);
}

// Speed |(a, b)| with the hardware square root (relative error ~2^-22; the
// speed-gradient path states FP32 accuracy, not correct rounding).  Every kernel
// of this file uses it, so the fused and two-step paths agree bit for bit.
__device__ __forceinline__ float speed_of(float a, float b) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(fmaf(a, a, b * b)));
    return r;
}
__device__ __forceinline__ float2 speed_of2(float2 a, float2 b) {
    const float2 q = __ffma2_rn(a, a, __fmul2_rn(b, b));
    float2 r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r.x) : "f"(q.x));
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r.y) : "f"(q.y));
    return r;
}

// Paired subtraction a - b (sub.rn.f32x2): each half one IEEE operation.
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
    float2 r;
    asm("{.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

__device__ __forceinline__ void st_evict_last_f4(float4* p, float4 v) {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w), "l"(pol)
                 : "memory");
}

struct GradParams {
    const void* u;
    const void* v;
    int64_t stride;  // elements between members
    int M, H, W, ddof;
    int s0, s1;      // statistics rows [s0, s1] of this band
    int row0;        // grid row of workspace row 0
    float4* st;      // record planes: gx at st, gy at st + ps
    int64_t ps;
    float sx1, sx2, sy1, sy2;  // 1/dx, 1/(2dx), 1/dy, 1/(2dy)
};

template <typename T>
__global__ void __launch_bounds__(kGW * 32, 2) grad_stats_kernel(const __grid_constant__ GradParams p) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = (blockIdx.x * kGW + warp) * kGC;  // first vertex column of the warp tile
    const int r0 = p.s0 + blockIdx.y * kGR;          // first vertex row of the warp tile
    if (c0 >= p.W || r0 > p.s1) return;              // uniform per warp; no block barriers below
    const int H = p.H, W = p.W;
    const int col = c0 - 1 + lane;                   // this lane's column (may lie outside the grid)
    const int cl = min(max(col, 0), W - 1);
    const bool out_lane = lane >= 1 && lane <= kGC && col < W;
    const bool xlo = col <= 0, xhi = col >= W - 1;   // one-sided x difference at the ends
    const int nr = min(kGR, p.s1 - r0 + 1);
    int off[kGR + 2];                                 // rows r0-1 .. r0+kGR, clamped (H*W < 2^31)
#pragma unroll
    for (int q = 0; q < kGR + 2; ++q) off[q] = min(max(r0 - 1 + q, 0), H - 1) * W + cl;
    const T* u = reinterpret_cast<const T*>(p.u);
    const T* v = reinterpret_cast<const T*>(p.v);
    float x0x[kGR], x0y[kGR], s1x[kGR], s2x[kGR], s1y[kGR], s2y[kGR];
#pragma unroll
    for (int q = 0; q < kGR; ++q) x0x[q] = x0y[q] = s1x[q] = s2x[q] = s1y[q] = s2y[q] = 0.f;
    for (int m = 0; m < p.M; ++m) {
        const T* um = u + (int64_t)m * p.stride;
        const T* vm = v + (int64_t)m * p.stride;
        float a[kGR + 2], b[kGR + 2];
#pragma unroll
        for (int q = 0; q < kGR + 2; ++q) {
            a[q] = ldm(um + off[q]);
            b[q] = ldm(vm + off[q]);
        }
        float s[kGR + 2];
#pragma unroll
        for (int q = 0; q < kGR + 2; ++q) s[q] = speed_of(a[q], b[q]);
#pragma unroll
        for (int q = 0; q < kGR; ++q) {
            const float sc = s[q + 1];
            const float sl = __shfl_up_sync(kFull, sc, 1), sr = __shfl_down_sync(kFull, sc, 1);
            const float gx = xlo ? (sr - sc) * p.sx1 : (xhi ? (sc - sl) * p.sx1 : (sr - sl) * p.sx2);
            const int r = r0 + q;
            const float gy = r == 0 ? (s[q + 2] - sc) * p.sy1
                                    : (r >= H - 1 ? (sc - s[q]) * p.sy1 : (s[q + 2] - s[q]) * p.sy2);
            if (m == 0) {
                x0x[q] = gx;
                x0y[q] = gy;
            } else {
                const float dx_ = gx - x0x[q], dy_ = gy - x0y[q];
                s1x[q] += dx_;
                s2x[q] = fmaf(dx_, dx_, s2x[q]);
                s1y[q] += dy_;
                s2y[q] = fmaf(dy_, dy_, s2y[q]);
            }
        }
    }
    if (!out_lane) return;
    const float fm = (float)p.M, fdof = (float)(p.M - p.ddof);
#pragma unroll
    for (int q = 0; q < kGR; ++q) {
        if (q < nr) {
            const int64_t n = (int64_t)(r0 + q - p.row0) * W + col;
            float dl = s1x[q] / fm, vv = (s2x[q] - s1x[q] * dl) / fdof;
            st_evict_last_f4(p.st + n, make_float4(x0x[q], dl, vv < 0.f ? 0.f : vv, 0.f));
            dl = s1y[q] / fm;
            vv = (s2y[q] - s1y[q] * dl) / fdof;
            st_evict_last_f4(p.st + p.ps + n, make_float4(x0y[q], dl, vv < 0.f ? 0.f : vv, 0.f));
        }
    }
}

// ---- paired variant: two columns per lane ------------------------------------
// Lane l of a warp tile holds columns c0 - 2 + 2l and c0 - 1 + 2l (loaded as one
// bf16x2 / float2), of vertex rows r0 - 1 .. r0 + 4; lanes 1..30 own the 60
// vertex columns c0 .. c0 + 59.  Loads are clamped to the grid, which turns the
// one-sided differences at the ends into the same subtraction with the scale
// 1/dx (1/dy) instead of 1/(2dx): no selects per member.  Speeds, differences
// and shifted sums run on float2 pairs (FFMA2 / FADD2 / FMUL2), and the next
// member's loads are issued before the current member is processed.
constexpr int kPR = 4;   // vertex rows per warp tile
constexpr int kPC = 60;  // vertex columns per warp tile

template <typename T>
struct PairLd;
template <>
struct PairLd<float> {
    using raw = float2;
    static __device__ __forceinline__ raw ld(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
    static __device__ __forceinline__ raw ld2(const float* p0, const float* p1) { return make_float2(__ldg(p0), __ldg(p1)); }
    static __device__ __forceinline__ float2 cvt(raw r) { return r; }
};
template <>
struct PairLd<__nv_bfloat16> {
    using raw = uint32_t;
    static __device__ __forceinline__ raw ld(const __nv_bfloat16* p) { return __ldg(reinterpret_cast<const unsigned*>(p)); }
    static __device__ __forceinline__ raw ld2(const __nv_bfloat16* p0, const __nv_bfloat16* p1) {
        return (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p0)) |
               ((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p1)) << 16);
    }
    static __device__ __forceinline__ float2 cvt(raw r) {
        return make_float2(__uint_as_float(r << 16), __uint_as_float(r & 0xFFFF0000u));
    }
};

template <typename T>
__global__ void __launch_bounds__(kGW * 32, 2) grad_stats_pair_kernel(const __grid_constant__ GradParams p) {
    using L = PairLd<T>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = (blockIdx.x * kGW + warp) * kPC;  // even
    const int r0 = p.s0 + blockIdx.y * kPR;
    if (c0 >= p.W || r0 > p.s1) return;              // uniform per warp; no block barriers below
    const int H = p.H, W = p.W;
    const int ca = c0 - 2 + 2 * lane;                // this lane's first column (even; W is even)
    const bool inside = ca >= 0 && ca + 1 < W;       // both columns in the grid: one paired load
    const int cal = min(max(ca, 0), W - 1), cbl = min(max(ca + 1, 0), W - 1);
    const bool own = lane >= 1 && lane <= 30 && ca < W;
    // x scales: the ends take the one-sided step (the clamped neighbour is the vertex itself)
    const float2 kx = make_float2(ca == 0 ? p.sx1 : p.sx2, ca + 1 == W - 1 ? p.sx1 : p.sx2);
    const int nr = min(kPR, p.s1 - r0 + 1);
    int off[kPR + 2];  // rows r0-1 .. r0+kPR, clamped (H*W < 2^31)
#pragma unroll
    for (int q = 0; q < kPR + 2; ++q) off[q] = min(max(r0 - 1 + q, 0), H - 1) * W;
    float ky[kPR];
#pragma unroll
    for (int q = 0; q < kPR; ++q) ky[q] = (r0 + q == 0 || r0 + q >= H - 1) ? p.sy1 : p.sy2;
    const T* u = reinterpret_cast<const T*>(p.u);
    const T* v = reinterpret_cast<const T*>(p.v);
    auto load = [&](int m, typename L::raw (&ru)[kPR + 2], typename L::raw (&rv)[kPR + 2]) {
        const T* um = u + (int64_t)m * p.stride;
        const T* vm = v + (int64_t)m * p.stride;
        if (inside) {
#pragma unroll
            for (int q = 0; q < kPR + 2; ++q) {
                ru[q] = L::ld(um + off[q] + ca);
                rv[q] = L::ld(vm + off[q] + ca);
            }
        } else {
#pragma unroll
            for (int q = 0; q < kPR + 2; ++q) {
                ru[q] = L::ld2(um + off[q] + cal, um + off[q] + cbl);
                rv[q] = L::ld2(vm + off[q] + cal, vm + off[q] + cbl);
            }
        }
    };
    float2 x0x[kPR], x0y[kPR], s1x[kPR], s2x[kPR], s1y[kPR], s2y[kPR];
    using raw_t = typename L::raw;
    auto grads = [&](const raw_t (&ru)[kPR + 2], const raw_t (&rv)[kPR + 2], float2 (&gx)[kPR], float2 (&gy)[kPR]) {
        float2 sp[kPR + 2];
#pragma unroll
        for (int q = 0; q < kPR + 2; ++q) sp[q] = speed_of2(L::cvt(ru[q]), L::cvt(rv[q]));
#pragma unroll
        for (int q = 0; q < kPR; ++q) {
            const float2 sc = sp[q + 1];
            const float sl = __shfl_up_sync(kFull, sc.y, 1);    // speed one column left of ca
            const float sr = __shfl_down_sync(kFull, sc.x, 1);  // speed one column right of ca + 1
            gx[q] = __fmul2_rn(fsub2(make_float2(sc.y, sr), make_float2(sl, sc.x)), kx);
            gy[q] = __fmul2_rn(fsub2(sp[q + 2], sp[q]), make_float2(ky[q], ky[q]));
        }
    };
    auto accumulate = [&](const raw_t (&ru)[kPR + 2], const raw_t (&rv)[kPR + 2]) {
        float2 gx[kPR], gy[kPR];
        grads(ru, rv, gx, gy);
#pragma unroll
        for (int q = 0; q < kPR; ++q) {
            const float2 dxv = fsub2(gx[q], x0x[q]), dyv = fsub2(gy[q], x0y[q]);
            s1x[q] = __fadd2_rn(s1x[q], dxv);
            s2x[q] = __ffma2_rn(dxv, dxv, s2x[q]);
            s1y[q] = __fadd2_rn(s1y[q], dyv);
            s2y[q] = __ffma2_rn(dyv, dyv, s2y[q]);
        }
    };
    // two load buffers in ping-pong: the next member's loads are in flight
    // while the current one is processed, without register copies
    raw_t au[kPR + 2], av[kPR + 2], bu[kPR + 2], bv[kPR + 2];
    load(0, au, av);
    if (p.M > 1) load(1, bu, bv);
    {
        float2 gx[kPR], gy[kPR];
        grads(au, av, gx, gy);
#pragma unroll
        for (int q = 0; q < kPR; ++q) {
            x0x[q] = gx[q];
            x0y[q] = gy[q];
            s1x[q] = s2x[q] = s1y[q] = s2y[q] = make_float2(0.f, 0.f);
        }
    }
    int m = 1;
    for (; m + 1 < p.M; m += 2) {  // b holds member m
        load(m + 1, au, av);
        accumulate(bu, bv);
        if (m + 2 < p.M) load(m + 2, bu, bv);
        accumulate(au, av);
    }
    if (m < p.M) accumulate(bu, bv);
    if (!own) return;
    const float fm = (float)p.M, fdof = (float)(p.M - p.ddof);
    auto rec = [&](float x0, float a1, float a2) {
        const float dl = a1 / fm;
        const float vv = (a2 - a1 * dl) / fdof;
        return make_float4(x0, dl, vv < 0.f ? 0.f : vv, 0.f);
    };
#pragma unroll
    for (int q = 0; q < kPR; ++q) {
        if (q < nr) {
            const int64_t n = (int64_t)(r0 + q - p.row0) * W + ca;
            st_evict_last_f4(p.st + n, rec(x0x[q].x, s1x[q].x, s2x[q].x));
            st_evict_last_f4(p.st + p.ps + n, rec(x0y[q].x, s1y[q].x, s2y[q].x));
            if (ca + 1 < W) {
                st_evict_last_f4(p.st + n + 1, rec(x0x[q].y, s1x[q].y, s2x[q].y));
                st_evict_last_f4(p.st + p.ps + n + 1, rec(x0y[q].y, s1y[q].y, s2y[q].y));
            }
        }
    }
}

// gradient members: one thread per (member, vertex)
template <typename T>
__global__ void __launch_bounds__(256) grad_members_kernel(const T* __restrict__ u, const T* __restrict__ v,
                                                           int64_t stride, int M, int H, int W, float sx1, float sx2,
                                                           float sy1, float sy2, float* __restrict__ gx,
                                                           float* __restrict__ gy) {
    const int64_t plane = (int64_t)H * W, n = plane * M;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = q / plane, r = q - m * plane;
        const int j = (int)(r / W), i = (int)(r - (int64_t)j * W);
        const T* um = u + m * stride;
        const T* vm = v + m * stride;
        auto speed = [&](int jj, int ii) {
            const int64_t o = (int64_t)jj * W + ii;
            return speed_of(ldm(um + o), ldm(vm + o));
        };
        const int il = max(i - 1, 0), ih = min(i + 1, W - 1), jl = max(j - 1, 0), jh = min(j + 1, H - 1);
        gx[q] = (speed(j, ih) - speed(j, il)) * (ih - il == 2 ? sx2 : sx1);
        gy[q] = (speed(jh, i) - speed(jl, i)) * (jh - jl == 2 ? sy2 : sy1);
    }
}

template <typename T>
lcp_status run_grad(const void* u, const void* v, int M, int H, int W, int64_t stride, int ddof, double dx, double dy,
                    const float* iso, int K, void* out, lcp_dtype out_dtype, uint32_t* mask, void* ws,
                    size_t ws_bytes, cudaStream_t st) {
    // paired loads need every row and member to start on an even column
    const bool paired = W % 2 == 0 && stride % 2 == 0 && ((uintptr_t)u % (2 * sizeof(T))) == 0 &&
                        ((uintptr_t)v % (2 * sizeof(T))) == 0;
    const WsGeometry G = ws_geometry(H, W, ws_bytes);
    float4* rec = reinterpret_cast<float4*>(reinterpret_cast<char*>(ws) + G.ctr_bytes);
    const int64_t ps = (int64_t)(G.plane_bytes / sizeof(float4));
    const int Hc = H - 1;
    for (int r0 = 0; r0 < Hc; r0 += G.band_rows) {
        const int r1 = std::min(r0 + G.band_rows, Hc);
        const int s0 = std::max(r0 - 1, 0), s1 = std::min(r1 + 1, H - 1);
        GradParams gp;
        gp.u = u;
        gp.v = v;
        gp.stride = stride;
        gp.M = M;
        gp.H = H;
        gp.W = W;
        gp.ddof = ddof;
        gp.s0 = s0;
        gp.s1 = s1;
        gp.row0 = s0;
        gp.st = rec;
        gp.ps = ps;
        gp.sx1 = (float)(1.0 / dx);
        gp.sx2 = (float)(0.5 / dx);
        gp.sy1 = (float)(1.0 / dy);
        gp.sy2 = (float)(0.5 / dy);
        if (paired) {
            const dim3 grid((W + kGW * kPC - 1) / (kGW * kPC), (s1 - s0 + 1 + kPR - 1) / kPR);
            grad_stats_pair_kernel<T><<<grid, kGW * 32, 0, st>>>(gp);
        } else {
            const dim3 grid((W + kGW * kGC - 1) / (kGW * kGC), (s1 - s0 + 1 + kGR - 1) / kGR);
            grad_stats_kernel<T><<<grid, kGW * 32, 0, st>>>(gp);
        }
        lcp_status s = check_launch("lcp_speed_gradient_ws (statistics)");
        if (s != LCP_OK) return s;
        s = ws_lcp_rows(rec, ps, s0, H, W, r0, r1, dx, dy, iso, K, out, out_dtype, mask, st);
        if (s != LCP_OK) return s;
    }
    return LCP_OK;
}

}  // namespace
}  // namespace lcp

using namespace lcp;

extern "C" lcp_status lcp_speed_gradient(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                                         int64_t member_stride, double dx, double dy, float* gx, float* gy,
                                         lcp_stream_t stream) {
    static const char* fn = "lcp_speed_gradient";
    lcp_status s = check_members(fn, u, v, in_dtype, M, H, W, member_stride, 0);
    if (s != LCP_OK) return s;
    if ((s = check_spacing(fn, dx, dy)) != LCP_OK) return s;
    if (!gx || !gy) return fail(LCP_ERR_ARG, "%s: NULL gx or gy", fn);
    const int64_t stride = M > 1 ? member_stride : (int64_t)H * W;
    const int64_t n = (int64_t)M * H * W;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16);
    cudaStream_t st = (cudaStream_t)stream;
    const float sx1 = (float)(1.0 / dx), sx2 = (float)(0.5 / dx), sy1 = (float)(1.0 / dy), sy2 = (float)(0.5 / dy);
    if (in_dtype == LCP_F32)
        grad_members_kernel<float><<<grid, 256, 0, st>>>((const float*)u, (const float*)v, stride, M, H, W, sx1, sx2,
                                                          sy1, sy2, gx, gy);
    else
        grad_members_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>((const __nv_bfloat16*)u, (const __nv_bfloat16*)v,
                                                                  stride, M, H, W, sx1, sx2, sy1, sy2, gx, gy);
    return check_launch(fn);
}

extern "C" lcp_status lcp_speed_gradient_ws(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                                            int64_t member_stride, int ddof, double dx, double dy, const float* iso,
                                            int K, void* lcp_out, lcp_dtype out_dtype, uint32_t* mask,
                                            void* workspace, size_t workspace_bytes, lcp_stream_t stream) {
    static const char* fn = "lcp_speed_gradient_ws";
    lcp_status s = check_members(fn, u, v, in_dtype, M, H, W, member_stride, ddof);
    if (s != LCP_OK) return s;
    if ((s = check_iso(fn, iso, K)) != LCP_OK) return s;
    if ((s = check_spacing(fn, dx, dy)) != LCP_OK) return s;
    if (!lcp_out) return fail(LCP_ERR_ARG, "%s: NULL output", fn);
    if (out_dtype != LCP_F32 && out_dtype != LCP_F16) return fail(LCP_ERR_ARG, "%s: out dtype must be F32 or F16", fn);
    if ((uintptr_t)mask & 3) return fail(LCP_ERR_ARG, "%s: mask must be 4-byte aligned", fn);
    if (!workspace || ((uintptr_t)workspace & 255)) return fail(LCP_ERR_ARG, "%s: need a 256-byte aligned workspace", fn);
    if ((int64_t)H * W >= (1ll << 31)) return fail(LCP_ERR_UNSUPPORTED, "%s: H * W must be below 2^31", fn);
    const WsGeometry G = ws_geometry(H, W, workspace_bytes);
    if (workspace_bytes < G.total)
        return fail(LCP_ERR_ARG, "%s: workspace too small (%zu < %zu bytes for the smallest band)", fn, workspace_bytes,
                    G.total);
    if ((H + 2 + kPR - 1) / kPR > 65535) return fail(LCP_ERR_UNSUPPORTED, "%s: H too large", fn);
    const int64_t stride = M > 1 ? member_stride : (int64_t)H * W;
    cudaStream_t st = (cudaStream_t)stream;
    if (in_dtype == LCP_F32)
        return run_grad<float>(u, v, M, H, W, stride, ddof, dx, dy, iso, K, lcp_out, out_dtype, mask, workspace,
                               workspace_bytes, st);
    return run_grad<__nv_bfloat16>(u, v, M, H, W, stride, ddof, dx, dy, iso, K, lcp_out, out_dtype, mask, workspace,
                                   workspace_bytes, st);
}
