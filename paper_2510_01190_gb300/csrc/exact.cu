// Exact LCP under the empirical model (every vertex component an independent
// uniform draw from its own members): the limit Monte Carlo approaches as the
// sample count grows, computed by counting instead of sampling.
//
// At an interior vertex D = X + Y with X = (U_{i+1} - U_{i-1}) / (2 dx) and
// Y = (V_{j+1} - V_{j-1}) / (2 dy); X takes M^2 equally likely values, Y too, and
// they are independent, so P(D < c) = #{(x, y) : y < c - x} / M^4.  One warp
// per vertex: the M^2 values of X and of Y go to shared memory (padded with
// +inf to a power of two), a bitonic network sorts each, and per isovalue the
// lanes count with two pointers over contiguous chunks of X (each chunk's
// starting pointer by binary search).  Interior vertex stencils share no member
// values, so the four vertex divergences of a cell with four interior vertices
// are independent and LCP = 1 - prod p - prod q holds exactly there.
#include <cmath>
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "lcp_common.cuh"

namespace lcp {
namespace {

constexpr int kEW = 2;  // warps (vertices in flight) per CTA: 2 x 32 KB of sort buffers at M = 50

__device__ __forceinline__ float ld_member(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld_member(const __nv_bfloat16* p) {
    return __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p)) << 16);
}

// One compare-exchange of the bitonic network: pair (i, l = i + j), where i is t
// with a zero inserted at bit log2(j) (j a power of two); ascending where bit k
// of i is clear.
__device__ __forceinline__ void bitonic_ce(float* a, int t, int j, int k) {
    const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1)), l = i + j;
    const bool up = (i & k) == 0;
    const float x = a[i], y = a[l];
    if ((x > y) == up) {
        a[i] = y;
        a[l] = x;
    }
}

// Ascending bitonic sort of n (a power of two) floats in shared memory by one
// warp.  From n = 512 on every lane has a multiple of 8 exchanges per stage,
// done 8 at a time so that their shared-memory loads overlap.
__device__ void warp_bitonic_sort(float* a, int n, int lane) {
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (n >= 512) {
                for (int t0 = 0; t0 < (n >> 1); t0 += 256) {
#pragma unroll
                    for (int r = 0; r < 8; ++r) bitonic_ce(a, t0 + 32 * r + lane, j, k);
                }
            } else {
                for (int t = lane; t < (n >> 1); t += 32) bitonic_ce(a, t, j, k);
            }
            __syncwarp();
        }
    }
}

// Number of elements of the ascending array a[0..n) that are < v.
__device__ __forceinline__ int lower_count(const float* a, int n, float v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <typename T>
__global__ void __launch_bounds__(kEW * 32) exact_below_kernel(const T* __restrict__ u, const T* __restrict__ v, int M,
                                                              int64_t stride, int H, int W, float sx, float sy,
                                                              const __grid_constant__ IsoParams iso, int n2,
                                                              float* __restrict__ below) {
    extern __shared__ __align__(16) float ex_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* X = ex_smem + (size_t)warp * 2 * n2;
    float* Y = X + n2;
    const int nin = (H - 2) * (W - 2);  // interior vertices
    const int m2 = M * M;
    const double m4 = (double)m2 * (double)m2;
    for (int vid = blockIdx.x * kEW + warp; vid < nin; vid += gridDim.x * kEW) {
        const int j = 1 + vid / (W - 2), i = 1 + vid % (W - 2);
        const int64_t o = (int64_t)j * W + i;
        for (int q = lane; q < n2; q += 32) {  // X[a M + b] = (U_a(i+1) - U_b(i-1)) sx, Y likewise along j
            float x = INFINITY, y = INFINITY;
            if (q < m2) {
                const int aa = q / M, bb = q - aa * M;
                x = (ld_member(u + (int64_t)aa * stride + o + 1) - ld_member(u + (int64_t)bb * stride + o - 1)) * sx;
                y = (ld_member(v + (int64_t)aa * stride + o + W) - ld_member(v + (int64_t)bb * stride + o - W)) * sy;
            }
            X[q] = x;
            Y[q] = y;
        }
        __syncwarp();
        warp_bitonic_sort(X, n2, lane);
        warp_bitonic_sort(Y, n2, lane);
        // count pairs with x + y < c: lane takes X[s0 .. s1), Y pointer by binary search then descending
        const int chunk = (m2 + 31) / 32, s0 = min(lane * chunk, m2), s1 = min(s0 + chunk, m2);
        for (int k = 0; k < iso.K; ++k) {
            const float c = iso.c[k];
            uint32_t cnt = 0;
            if (s0 < s1) {
                int p = lower_count(Y, m2, c - X[s0]);
                for (int s = s0; s < s1; ++s) {
                    const float t = c - X[s];  // non-increasing in s
                    while (p > 0 && !(Y[p - 1] < t)) --p;
                    cnt += (uint32_t)p;
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, off);
            if (lane == 0) below[(int64_t)k * H * W + o] = (float)((double)cnt / m4);
        }
        __syncwarp();
    }
}

// Cells whose four vertices are interior: LCP = 1 - prod p - prod (1 - p); the others NaN.
__global__ void exact_cells_kernel(const float* __restrict__ below, int H, int W, int K, float* __restrict__ out) {
    const int Hc = H - 1, Wc = W - 1;
    const int64_t plane = (int64_t)Hc * Wc, n = plane * K;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(q / plane);
        const int64_t r = q - (int64_t)k * plane;
        const int j = (int)(r / Wc), i = (int)(r - (int64_t)j * Wc);
        float l = NAN;
        if (i >= 1 && i <= W - 3 && j >= 1 && j <= H - 3) {
            const float* b = below + (int64_t)k * H * W + (int64_t)j * W + i;
            const float p0 = b[0], p1 = b[1], p2 = b[W], p3 = b[W + 1];
            l = 1.0f - (p0 * p1) * (p2 * p3) - ((1.0f - p0) * (1.0f - p1)) * ((1.0f - p2) * (1.0f - p3));
        }
        out[q] = l;
    }
}

}  // namespace
}  // namespace lcp

using namespace lcp;

extern "C" lcp_status lcp_exact_empirical(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                                          int64_t member_stride, double dx, double dy, const float* iso, int K,
                                          float* below, float* lcp_out, lcp_stream_t stream) {
    static const char* fn = "lcp_exact_empirical";
    lcp_status s = check_members(fn, u, v, in_dtype, M, H, W, member_stride, 0);
    if (s != LCP_OK) return s;
    if (M > 64) return fail(LCP_ERR_UNSUPPORTED, "%s: M <= 64 members (M^4 counts exact in fp32)", fn);
    if (H < 4 || W < 4) return fail(LCP_ERR_ARG, "%s: need H, W >= 4 (a cell with four interior vertices)", fn);
    if ((s = check_spacing(fn, dx, dy)) != LCP_OK) return s;
    if (!iso || K < 1 || K > kMaxIsoPerLaunch) return fail(LCP_ERR_ARG, "%s: need a host iso array, 1 <= K <= %d", fn, kMaxIsoPerLaunch);
    if (!below || !lcp_out) return fail(LCP_ERR_ARG, "%s: NULL below or lcp_out", fn);
    IsoParams ip;
    ip.K = K;
    for (int k = 0; k < K; ++k) ip.c[k] = iso[k];
    int n2 = 1;
    while (n2 < M * M) n2 <<= 1;
    const size_t smem = (size_t)kEW * 2 * n2 * sizeof(float);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t stride = M > 1 ? member_stride : (int64_t)H * W;
    const float sx = (float)(0.5 / dx), sy = (float)(0.5 / dy);
    const int nin = (H - 2) * (W - 2);
    const int grid = (int)std::min<int64_t>((nin + kEW - 1) / kEW, (int64_t)num_sms() * 8);
    {
        static std::mutex mu;
        std::lock_guard<std::mutex> lk(mu);
        const cudaError_t e = in_dtype == LCP_F32
                                  ? cudaFuncSetAttribute(exact_below_kernel<float>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                                  : cudaFuncSetAttribute(exact_below_kernel<__nv_bfloat16>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LCP_ERR_CUDA, "%s: %zu bytes of shared memory not available", fn, smem);
        }
    }
    if (in_dtype == LCP_F32)
        exact_below_kernel<float><<<grid, kEW * 32, smem, st>>>((const float*)u, (const float*)v, M, stride, H, W, sx,
                                                                 sy, ip, n2, below);
    else
        exact_below_kernel<__nv_bfloat16><<<grid, kEW * 32, smem, st>>>(
            (const __nv_bfloat16*)u, (const __nv_bfloat16*)v, M, stride, H, W, sx, sy, ip, n2, below);
    if ((s = check_launch(fn)) != LCP_OK) return s;
    const int64_t cells = (int64_t)K * (H - 1) * (W - 1);
    exact_cells_kernel<<<(int)std::min<int64_t>((cells + 255) / 256, (int64_t)num_sms() * 16), 256, 0, st>>>(
        below, H, W, K, lcp_out);
    return check_launch(fn);
}
