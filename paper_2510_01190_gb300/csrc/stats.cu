// lcp_stats: per-vertex mean and variance of u and v over the ensemble
// (Sec. 3.1, closing paragraph).  A flat, fully coalesced stream over the
// member planes: each thread owns VEC consecutive vertices and walks the
// members with UNROLL independent 16-byte loads per component in flight.
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
        if (in16 && stride % 8 == 0)
            launch_stats<__nv_bfloat16, 8, 4>(u, v, M, nv, stride, ddof, vec_out, mu_u, var_u, mu_v, var_v, st);
        else
            launch_stats<__nv_bfloat16, 1, 8>(u, v, M, nv, stride, ddof, false, mu_u, var_u, mu_v, var_v, st);
    }
    return check_launch("lcp_stats");
}
