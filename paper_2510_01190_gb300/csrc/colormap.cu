// lcp_colormap: a scalar map (an LCP map, a divergence map) to RGBA8 bytes in
// a device buffer.  The paper shows its LCP maps by colour mapping (Sec. 3.1,
// last paragraph) and clamps the mean-field divergence to a display range
// before mapping it (Sec. 4.2, Fig. 3c); no graphics API is involved here.
//
// Every value costs 4 bytes read and 4 bytes written, so the kernel is a
// plain stream: each thread maps 4 consecutive values (one 16-byte load and
// one 16-byte store when the buffers allow it).  The colour stops are staged
// in shared memory, so lanes that fall in different stop segments index them
// without serialising on the constant cache.  Each channel is computed by a
// fixed sequence of IEEE fp32 operations rounded to nearest (no contraction
// into fused multiply-adds), which the header states, so the bytes do not
// depend on the compiler.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "lcp_common.cuh"

namespace lcp {
namespace {

constexpr int kCT = 256;  // threads per block

struct ColorParams {
    const float* x;
    const uint32_t* mask;
    uint32_t* rgba;
    int64_t n;        // values
    int cols, rows;   // mask geometry: values are [planes][rows][cols]
    int n_words;      // mask words per row
    float vmin, vmax;
    uint32_t nan_rgba, mask_rgba;
    int n_stops;
    float stops[LCP_MAX_COLOR_STOPS * 5];
};

__device__ __forceinline__ uint32_t quantise(float ch) {
    float b = floorf(__fadd_rn(__fmul_rn(ch, 255.0f), 0.5f));
    b = fminf(fmaxf(b, 0.0f), 255.0f);
    return (uint32_t)b;
}

__device__ __forceinline__ uint32_t map_one(const ColorParams& p, const float* st, float x) {
    if (x != x) return p.nan_rgba;
    float t = __fdiv_rn(__fsub_rn(x, p.vmin), __fsub_rn(p.vmax, p.vmin));
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    int s = 0;
    for (int q = 1; q < p.n_stops - 1; ++q) s = t >= st[5 * q] ? q : s;
    const float* a = st + 5 * s;
    const float* b = a + 5;
    const float f = __fdiv_rn(__fsub_rn(t, a[0]), __fsub_rn(b[0], a[0]));
    uint32_t out = 0;
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        const float c = __fadd_rn(a[1 + ch], __fmul_rn(f, __fsub_rn(b[1 + ch], a[1 + ch])));
        out |= quantise(c) << (8 * ch);
    }
    return out;
}

template <bool MASK, typename Idx>
__global__ void __launch_bounds__(kCT) colormap_kernel(const __grid_constant__ ColorParams p) {
    __shared__ float st[LCP_MAX_COLOR_STOPS * 5];
    for (int q = threadIdx.x; q < p.n_stops * 5; q += kCT) st[q] = p.stops[q];
    __syncthreads();
    const bool vec = ((reinterpret_cast<uintptr_t>(p.x) | reinterpret_cast<uintptr_t>(p.rgba)) & 15) == 0;
    const Idx n = (Idx)p.n;
    for (Idx g = ((Idx)blockIdx.x * kCT + threadIdx.x) * 4; g < n; g += (Idx)gridDim.x * kCT * 4) {
        float x[4];
        const int cnt = n - g >= 4 ? 4 : (int)(n - g);
        if (vec && cnt == 4) {
            const float4 r = __ldcs(reinterpret_cast<const float4*>(p.x + g));
            x[0] = r.x;
            x[1] = r.y;
            x[2] = r.z;
            x[3] = r.w;
        } else {
            for (int e = 0; e < 4; ++e) x[e] = e < cnt ? p.x[g + e] : 0.0f;
        }
        uint32_t c[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) c[e] = map_one(p, st, x[e]);
        if (MASK) {  // row and column of the first value; the next three follow along the row
            const Idx rowg = g / (Idx)p.cols;
            int col = (int)(g - rowg * (Idx)p.cols);
            Idx row = rowg;
            for (int e = 0; e < cnt; ++e) {
                const uint32_t w = p.mask[(int64_t)row * p.n_words + (col >> 5)];
                if (((w >> (col & 31)) & 1u) && x[e] == x[e]) c[e] = p.mask_rgba;  // NaN keeps its colour
                if (++col == p.cols) {
                    col = 0;
                    ++row;
                }
            }
        }
        if (vec && cnt == 4) {
            __stcs(reinterpret_cast<uint4*>(p.rgba + g), make_uint4(c[0], c[1], c[2], c[3]));
        } else {
            for (int e = 0; e < cnt; ++e) p.rgba[g + e] = c[e];
        }
    }
}

}  // namespace
}  // namespace lcp

using namespace lcp;

extern "C" lcp_status lcp_colormap(const float* values, int planes, int rows, int cols, float vmin, float vmax,
                                   const float* stops, int n_stops, uint32_t nan_rgba, const uint32_t* mask,
                                   uint32_t mask_rgba, uint8_t* rgba, lcp_stream_t stream) {
    static const char* fn = "lcp_colormap";
    if (planes < 0 || rows < 0 || cols < 0) return fail(LCP_ERR_ARG, "%s: negative size", fn);
    const int64_t n = (int64_t)planes * rows * cols;
    if (!(std::isfinite(vmin) && std::isfinite(vmax) && vmin < vmax))
        return fail(LCP_ERR_ARG, "%s: need finite vmin < vmax", fn);
    if (!stops || n_stops < 2 || n_stops > LCP_MAX_COLOR_STOPS)
        return fail(LCP_ERR_ARG, "%s: need a host array of 2..%d stops", fn, LCP_MAX_COLOR_STOPS);
    for (int q = 0; q < n_stops; ++q) {
        const float* s = stops + 5 * q;
        for (int c = 0; c < 5; ++c)
            if (!(s[c] >= 0.0f && s[c] <= 1.0f)) return fail(LCP_ERR_ARG, "%s: stop %d has a value outside [0, 1]", fn, q);
        if (q > 0 && !(s[0] > s[-5])) return fail(LCP_ERR_ARG, "%s: stop positions must increase", fn);
    }
    if (stops[0] != 0.0f || stops[5 * (n_stops - 1)] != 1.0f)
        return fail(LCP_ERR_ARG, "%s: the first stop must sit at 0 and the last at 1", fn);
    if (n == 0) return LCP_OK;
    if (!values || !rgba) return fail(LCP_ERR_ARG, "%s: NULL values or rgba", fn);
    if (((uintptr_t)values & 3) || ((uintptr_t)rgba & 3) || ((uintptr_t)mask & 3))
        return fail(LCP_ERR_ARG, "%s: values, mask and rgba must be 4-byte aligned", fn);
    ColorParams p;
    p.x = values;
    p.mask = mask;
    p.rgba = reinterpret_cast<uint32_t*>(rgba);
    p.n = n;
    p.cols = cols;
    p.rows = rows;
    p.n_words = (cols + 31) / 32;
    p.vmin = vmin;
    p.vmax = vmax;
    p.nan_rgba = nan_rgba;
    p.mask_rgba = mask_rgba;
    p.n_stops = n_stops;
    for (int q = 0; q < 5 * n_stops; ++q) p.stops[q] = stops[q];
    const int64_t groups = (n + 3) / 4;
    const int grid = (int)std::min<int64_t>((groups + kCT - 1) / kCT, (int64_t)num_sms() * 8);
    cudaStream_t st = (cudaStream_t)stream;
    const bool small = n < (1ll << 31) - 4 * (int64_t)kCT * grid;
    if (mask) {
        if (small) colormap_kernel<true, uint32_t><<<grid, kCT, 0, st>>>(p);
        else colormap_kernel<true, int64_t><<<grid, kCT, 0, st>>>(p);
    } else {
        if (small) colormap_kernel<false, uint32_t><<<grid, kCT, 0, st>>>(p);
        else colormap_kernel<false, int64_t><<<grid, kCT, 0, st>>>(p);
    }
    return check_launch(fn);
}
