// lcp_map: level-crossing probability of every cell and isovalue from the
// divergence Gaussians (Sec. 3.1, last paragraph, after Poethkow et al.):
//   LCP = 1 - prod_k P(D_k < c) - prod_k P(D_k >= c) over the 4 cell vertices,
// plus the optional mean-field crossing bits ([mu_d < c] not constant on the cell).
// Each thread owns 4 consecutive cells of one row, so a warp covers 128 cells
// starting on a multiple of 128: mask words are assembled with shuffles and
// written whole (no atomics, no pre-clearing).
#include "lcp_common.cuh"

namespace lcp {
namespace {

constexpr int kCellsPerThread = 4;
constexpr int kThreads = 128;

template <typename OutT>
__global__ void __launch_bounds__(kThreads) map_kernel(const float* __restrict__ mu_d, const float* __restrict__ var_d,
                                                       int H, int W, const __grid_constant__ IsoParams iso, int kbase,
                                                       OutT* __restrict__ out, uint32_t* __restrict__ mask,
                                                       int n_words) {
    const int j = blockIdx.y;  // cell row: vertex rows j and j + 1
    const int Hc = H - 1, Wc = W - 1;
    const int lane = threadIdx.x & 31;
    const int i0 = (blockIdx.x * kThreads + threadIdx.x) * kCellsPerThread;
    float m0[kCellsPerThread + 1], v0[kCellsPerThread + 1], m1[kCellsPerThread + 1], v1[kCellsPerThread + 1];
#pragma unroll
    for (int e = 0; e <= kCellsPerThread; ++e) {
        const int i = min(i0 + e, W - 1);
        m0[e] = mu_d[(int64_t)j * W + i];
        v0[e] = var_d[(int64_t)j * W + i];
        m1[e] = mu_d[(int64_t)(j + 1) * W + i];
        v1[e] = var_d[(int64_t)(j + 1) * W + i];
    }
    for (int k = 0; k < iso.K; ++k) {
        const float c = iso.c[k];
        float p0[kCellsPerThread + 1], q0[kCellsPerThread + 1], p1[kCellsPerThread + 1], q1[kCellsPerThread + 1];
        uint32_t b0 = 0, b1 = 0;
#pragma unroll
        for (int e = 0; e <= kCellsPerThread; ++e) {
            below_above(m0[e], v0[e], c, p0[e], q0[e]);
            below_above(m1[e], v1[e], c, p1[e], q1[e]);
            b0 |= (uint32_t)(m0[e] < c) << e;
            b1 |= (uint32_t)(m1[e] < c) << e;
        }
        const int64_t obase = ((int64_t)(kbase + k) * Hc + j) * Wc;
        uint32_t nib = 0;
#pragma unroll
        for (int e = 0; e < kCellsPerThread; ++e) {
            const int col = i0 + e;
            if (col < Wc) {
                const float lcp = 1.0f - (p0[e] * p0[e + 1]) * (p1[e] * p1[e + 1]) - (q0[e] * q0[e + 1]) * (q1[e] * q1[e + 1]);
                out[obase + col] = to_out<OutT>(clamp01(lcp));
                const uint32_t four = ((b0 >> e) & 3u) | (((b1 >> e) & 3u) << 2);
                nib |= (uint32_t)(four != 0u && four != 15u) << e;
            }
        }
        if (mask) {
            uint32_t val = nib << ((lane & 7) * kCellsPerThread);
            val |= __shfl_xor_sync(0xFFFFFFFFu, val, 1);
            val |= __shfl_xor_sync(0xFFFFFFFFu, val, 2);
            val |= __shfl_xor_sync(0xFFFFFFFFu, val, 4);
            const int word = i0 >> 5;
            if ((lane & 7) == 0 && word < n_words) mask[((int64_t)(kbase + k) * Hc + j) * n_words + word] = val;
        }
    }
}

}  // namespace
}  // namespace lcp

using namespace lcp;

extern "C" lcp_status lcp_map(const float* mu_d, const float* var_d, int H, int W, const float* iso, int K,
                              void* lcp_out, lcp_dtype out_dtype, uint32_t* mask, lcp_stream_t stream) {
    if (!mu_d || !var_d || !lcp_out) return fail(LCP_ERR_ARG, "lcp_map: NULL pointer");
    if (H < 2 || W < 2) return fail(LCP_ERR_ARG, "lcp_map: need H >= 2 and W >= 2");
    lcp_status s = check_iso("lcp_map", iso, K);
    if (s != LCP_OK) return s;
    if (out_dtype != LCP_F32 && out_dtype != LCP_F16) return fail(LCP_ERR_ARG, "lcp_map: out dtype must be F32 or F16");
    if ((uintptr_t)mask & 3) return fail(LCP_ERR_ARG, "lcp_map: mask must be 4-byte aligned");
    if (H - 1 > 65535) return fail(LCP_ERR_UNSUPPORTED, "lcp_map: H - 1 > 65535");
    const int Wc = W - 1, n_words = (Wc + 31) / 32;
    dim3 grid((Wc + kThreads * kCellsPerThread - 1) / (kThreads * kCellsPerThread), H - 1);
    cudaStream_t st = (cudaStream_t)stream;
    for (int kb = 0; kb < K; kb += kMaxIsoPerLaunch) {
        IsoParams p;
        p.K = K - kb < kMaxIsoPerLaunch ? K - kb : kMaxIsoPerLaunch;
        for (int k = 0; k < p.K; ++k) p.c[k] = iso[kb + k];
        if (out_dtype == LCP_F32)
            map_kernel<float><<<grid, kThreads, 0, st>>>(mu_d, var_d, H, W, p, kb, (float*)lcp_out, mask, n_words);
        else
            map_kernel<__half><<<grid, kThreads, 0, st>>>(mu_d, var_d, H, W, p, kb, (__half*)lcp_out, mask, n_words);
        s = check_launch("lcp_map");
        if (s != LCP_OK) return s;
    }
    return LCP_OK;
}
