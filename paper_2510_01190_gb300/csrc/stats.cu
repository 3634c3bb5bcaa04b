// lcp_stats: per-vertex mean and variance of u and v over the ensemble
// (Sec. 3.1, closing paragraph).  A flat, fully coalesced stream over the
// member planes: each thread owns VEC consecutive vertices and walks the
// members with UNROLL independent loads per component in flight (fp32: 16-byte
// loads of 4 vertices, 8 members a batch; bf16: stats_bf16x4_kernel below,
// 8-byte loads of 4 vertices, 10 members a batch).
//
// Numerics: shifted sums about member 0 (Chan, Golub, LeVeque 1983):
//   d_m = x_m - x_0,  S1 = sum d_m,  S2 = sum d_m^2,
//   mean = x_0 + S1 / M,  var = (S2 - S1 * (S1 / M)) / (M - ddof).
// Because x_0 is a member, |mean - x_0| is a few sigma at most, so the
// subtraction in var loses at most log2(M) bits whatever |mean| / sigma is.
#include "lcp_common.cuh"

namespace lcp {
namespace {

template <typename T>
__device__ __forceinline__ void stats_point(const T* __restrict__ x, int M, int64_t stride, int64_t n, int ddof,
                                            float& mean, float& var) {
    using L = Loader<T, 1>;
    float x0, a;
    L::cvt(L::load(x + n), &x0);
    float s1 = 0.f, s2 = 0.f;
    for (int m = 1; m < M; ++m) {
        L::cvt(L::load(x + (int64_t)m * stride + n), &a);
        const float d = a - x0;
        s1 += d;
        s2 = fmaf(d, d, s2);
    }
    const float delta = s1 / (float)M;
    var = (s2 - s1 * delta) / (float)(M - ddof);
    if (var < 0.f) var = 0.f;
    mean = x0 + delta;
}

template <typename T, int VEC, int UNROLL>
__global__ void __launch_bounds__(256) stats_kernel(const T* __restrict__ u, const T* __restrict__ v, int M,
                                                    int64_t nv, int64_t stride, int ddof, bool vec_out,
                                                    float* __restrict__ mu_u, float* __restrict__ var_u,
                                                    float* __restrict__ mu_v, float* __restrict__ var_v) {
    const int64_t n0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VEC;
    if (n0 >= nv) return;
    if (VEC > 1 && n0 + VEC > nv) {  // ragged tail of the plane
        for (int64_t n = n0; n < nv; ++n) {
            stats_point(u, M, stride, n, ddof, mu_u[n], var_u[n]);
            stats_point(v, M, stride, n, ddof, mu_v[n], var_v[n]);
        }
        return;
    }
    using L = Loader<T, VEC>;
    float x0u[VEC], x0v[VEC], s1u[VEC], s2u[VEC], s1v[VEC], s2v[VEC];
    L::cvt(L::load(u + n0), x0u);
    L::cvt(L::load(v + n0), x0v);
#pragma unroll
    for (int e = 0; e < VEC; ++e) s1u[e] = s2u[e] = s1v[e] = s2v[e] = 0.f;

    auto acc = [&](const typename L::raw_t& ru, const typename L::raw_t& rv) {
        float a[VEC], b[VEC];
        L::cvt(ru, a);
        L::cvt(rv, b);
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const float du = a[e] - x0u[e], dv = b[e] - x0v[e];
            s1u[e] += du;
            s2u[e] = fmaf(du, du, s2u[e]);
            s1v[e] += dv;
            s2v[e] = fmaf(dv, dv, s2v[e]);
        }
    };
    int m = 1;
    for (; m + UNROLL <= M; m += UNROLL) {
        typename L::raw_t ru[UNROLL], rv[UNROLL];
#pragma unroll
        for (int q = 0; q < UNROLL; ++q) {
            ru[q] = L::load(u + (int64_t)(m + q) * stride + n0);
            rv[q] = L::load(v + (int64_t)(m + q) * stride + n0);
        }
#pragma unroll
        for (int q = 0; q < UNROLL; ++q) acc(ru[q], rv[q]);
    }
    for (; m < M; ++m) acc(L::load(u + (int64_t)m * stride + n0), L::load(v + (int64_t)m * stride + n0));

    float mu_o[2][VEC], var_o[2][VEC];
    const float fm = (float)M, fdof = (float)(M - ddof);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
        float du = s1u[e] / fm, dv = s1v[e] / fm;
        float vu = (s2u[e] - s1u[e] * du) / fdof, vv = (s2v[e] - s1v[e] * dv) / fdof;
        if (vu < 0.f) vu = 0.f;
        if (vv < 0.f) vv = 0.f;
        mu_o[0][e] = x0u[e] + du;
        var_o[0][e] = vu;
        mu_o[1][e] = x0v[e] + dv;
        var_o[1][e] = vv;
    }
    if (VEC % 4 == 0 && vec_out) {
#pragma unroll
        for (int e = 0; e < VEC; e += 4) {
            *reinterpret_cast<float4*>(mu_u + n0 + e) = make_float4(mu_o[0][e], mu_o[0][e + 1], mu_o[0][e + 2], mu_o[0][e + 3]);
            *reinterpret_cast<float4*>(var_u + n0 + e) = make_float4(var_o[0][e], var_o[0][e + 1], var_o[0][e + 2], var_o[0][e + 3]);
            *reinterpret_cast<float4*>(mu_v + n0 + e) = make_float4(mu_o[1][e], mu_o[1][e + 1], mu_o[1][e + 2], mu_o[1][e + 3]);
            *reinterpret_cast<float4*>(var_v + n0 + e) = make_float4(var_o[1][e], var_o[1][e + 1], var_o[1][e + 2], var_o[1][e + 3]);
        }
    } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            mu_u[n0 + e] = mu_o[0][e];
            var_u[n0 + e] = var_o[0][e];
            mu_v[n0 + e] = mu_o[1][e];
            var_v[n0 + e] = var_o[1][e];
        }
    }
}

// bf16 members with 8-byte loads (4 vertices per thread) in batches of kB8 members,
// member 0 (the shift) in the first: a 20-member ensemble streams in two round trips
// per thread instead of eight, at up to 80 registers (3 blocks per SM).  The members
// are summed in the same order as stats_kernel, so the results are identical.
constexpr int kB8 = 10;
inline bool aligned8(const void* p) { return ((uintptr_t)p & 7) == 0; }

__device__ __forceinline__ uint2 ld_bf16x4(const __nv_bfloat16* p) {
    uint2 r;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ void cvt_bf16x4(uint2 r, float* x) {
    x[0] = __uint_as_float(r.x << 16);
    x[1] = __uint_as_float(r.x & 0xFFFF0000u);
    x[2] = __uint_as_float(r.y << 16);
    x[3] = __uint_as_float(r.y & 0xFFFF0000u);
}

__global__ void __launch_bounds__(256, 3) stats_bf16x4_kernel(const __nv_bfloat16* __restrict__ u,
                                                            const __nv_bfloat16* __restrict__ v, int M, int64_t nv,
                                                            int64_t stride, int ddof, bool vec_out,
                                                            float* __restrict__ mu_u, float* __restrict__ var_u,
                                                            float* __restrict__ mu_v, float* __restrict__ var_v) {
    const int64_t n0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (n0 >= nv) return;
    if (n0 + 4 > nv) {  // ragged tail of the plane
        for (int64_t n = n0; n < nv; ++n) {
            stats_point(u, M, stride, n, ddof, mu_u[n], var_u[n]);
            stats_point(v, M, stride, n, ddof, mu_v[n], var_v[n]);
        }
        return;
    }
    float x0u[4], x0v[4], s1u[4], s2u[4], s1v[4], s2v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) s1u[e] = s2u[e] = s1v[e] = s2v[e] = 0.f;
    auto acc = [&](uint2 ru, uint2 rv) {
        float a[4], b[4];
        cvt_bf16x4(ru, a);
        cvt_bf16x4(rv, b);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float du = a[e] - x0u[e], dv = b[e] - x0v[e];
            s1u[e] += du;
            s2u[e] = fmaf(du, du, s2u[e]);
            s1v[e] += dv;
            s2v[e] = fmaf(dv, dv, s2v[e]);
        }
    };
    int m = 0;
    // full batches (the first one holds member 0), then the rest as one predicated batch
    for (; m + kB8 <= M; m += kB8) {
        uint2 ru[kB8], rv[kB8];
#pragma unroll
        for (int q = 0; q < kB8; ++q) {
            ru[q] = ld_bf16x4(u + (int64_t)(m + q) * stride + n0);
            rv[q] = ld_bf16x4(v + (int64_t)(m + q) * stride + n0);
        }
        if (m == 0) {
            cvt_bf16x4(ru[0], x0u);
            cvt_bf16x4(rv[0], x0v);
        }
#pragma unroll
        for (int q = 0; q < kB8; ++q)
            if (m + q > 0) acc(ru[q], rv[q]);
    }
    if (m < M) {
        uint2 ru[kB8], rv[kB8];
#pragma unroll
        for (int q = 0; q < kB8; ++q)
            if (m + q < M) {
                ru[q] = ld_bf16x4(u + (int64_t)(m + q) * stride + n0);
                rv[q] = ld_bf16x4(v + (int64_t)(m + q) * stride + n0);
            }
        if (m == 0) {
            cvt_bf16x4(ru[0], x0u);
            cvt_bf16x4(rv[0], x0v);
        }
#pragma unroll
        for (int q = 0; q < kB8; ++q)
            if (m + q < M && m + q > 0) acc(ru[q], rv[q]);
    }
    const float fm = (float)M, fdof = (float)(M - ddof);
    float mo[4][4];  // mu_u, var_u, mu_v, var_v of the 4 vertices
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float du = s1u[e] / fm, dv = s1v[e] / fm;
        float vu = (s2u[e] - s1u[e] * du) / fdof, vv = (s2v[e] - s1v[e] * dv) / fdof;
        if (vu < 0.f) vu = 0.f;
        if (vv < 0.f) vv = 0.f;
        mo[0][e] = x0u[e] + du;
        mo[1][e] = vu;
        mo[2][e] = x0v[e] + dv;
        mo[3][e] = vv;
    }
    float* const outs[4] = {mu_u, var_u, mu_v, var_v};
    if (vec_out) {
#pragma unroll
        for (int o = 0; o < 4; ++o)
            *reinterpret_cast<float4*>(outs[o] + n0) = make_float4(mo[o][0], mo[o][1], mo[o][2], mo[o][3]);
    } else {
#pragma unroll
        for (int o = 0; o < 4; ++o)
#pragma unroll
            for (int e = 0; e < 4; ++e) outs[o][n0 + e] = mo[o][e];
    }
}

template <typename T, int VEC, int UNROLL>
void launch_stats(const void* u, const void* v, int M, int64_t nv, int64_t stride, int ddof, bool vec_out, float* a,
                  float* b, float* c, float* d, cudaStream_t st) {
    const int64_t groups = (nv + VEC - 1) / VEC;
    const unsigned blocks = (unsigned)((groups + 255) / 256);
    stats_kernel<T, VEC, UNROLL><<<blocks, 256, 0, st>>>((const T*)u, (const T*)v, M, nv, stride, ddof, vec_out, a,
                                                          b, c, d);
}

}  // namespace
}  // namespace lcp

using namespace lcp;

extern "C" lcp_status lcp_stats(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                                int64_t member_stride, int ddof, float* mu_u, float* var_u, float* mu_v,
                                float* var_v, lcp_stream_t stream) {
    lcp_status s = check_members("lcp_stats", u, v, in_dtype, M, H, W, member_stride, ddof);
    if (s != LCP_OK) return s;
    if (!mu_u || !var_u || !mu_v || !var_v) return fail(LCP_ERR_ARG, "lcp_stats: NULL output");
    if (((uintptr_t)mu_u | (uintptr_t)var_u | (uintptr_t)mu_v | (uintptr_t)var_v) & 3)
        return fail(LCP_ERR_ARG, "lcp_stats: outputs must be 4-byte aligned");
    const int64_t nv = (int64_t)H * W;
    const int64_t stride = M > 1 ? member_stride : nv;
    const bool vec_out = aligned16(mu_u) && aligned16(var_u) && aligned16(mu_v) && aligned16(var_v);
    const bool in16 = aligned16(u) && aligned16(v);
    cudaStream_t st = (cudaStream_t)stream;
    if (in_dtype == LCP_F32) {
        if (in16 && stride % 4 == 0)
            launch_stats<float, 4, 8>(u, v, M, nv, stride, ddof, vec_out, mu_u, var_u, mu_v, var_v, st);
        else
            launch_stats<float, 1, 8>(u, v, M, nv, stride, ddof, false, mu_u, var_u, mu_v, var_v, st);
    } else {
        if (aligned8(u) && aligned8(v) && stride % 4 == 0) {
            const unsigned blocks = (unsigned)(((nv + 3) / 4 + 255) / 256);
            stats_bf16x4_kernel<<<blocks, 256, 0, st>>>((const __nv_bfloat16*)u, (const __nv_bfloat16*)v, M, nv,
                                                        stride, ddof, vec_out, mu_u, var_u, mu_v, var_v);
        } else
            launch_stats<__nv_bfloat16, 1, 8>(u, v, M, nv, stride, ddof, false, mu_u, var_u, mu_v, var_v, st);
    }
    return check_launch("lcp_stats");
}
