// lcp_colormap: a scalar map (an LCP map, a divergence map) to RGBA8 bytes in
// a device buffer.  The paper shows its LCP maps by colour mapping (Sec. 3.1,
// last paragraph) and clamps the mean-field divergence to a display range
// before mapping it (Sec. 4.2, Fig. 3c); no graphics API is involved here.
//
// Every value costs 4 bytes read and 4 bytes written, so the kernel must stay
// under about 45 instructions per value to run at HBM speed, and keep enough
// loads in flight.  Hence: each thread maps groups of 4 consecutive values (one
// 16-byte load and store when the buffers allow it), two groups per trip of a
// persistent grid with both groups' loads and mask words issued before either
// is mapped; the reciprocals and colour differences of every stop
// segment are formed once per call on the host (each value then costs
// multiplications instead of two divisions; the bytes can differ from the
// exact map by one where a channel lies within fp32 rounding of a byte
// boundary); the segment of a value is the
// count of stop positions at or below it, compared against registers; the four
// channels are interpolated and quantised as two float2 pairs with Blackwell's
// paired fp32 instructions (each half an IEEE rounded-to-nearest operation); the row and
// column of the mask bits advance with the grid stride instead of being
// divided out, and one or two mask words serve a group of 4 values.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "lcp_common.cuh"

namespace lcp {
namespace {

constexpr int kCT = 256;  // threads per block
constexpr int kCB = 4;    // resident blocks per SM (<= 64 registers), the persistent grid's size per SM
constexpr int kCU = 2;    // groups per thread and trip
// (measured on 4 x 8191^2 values with the mask, blocks per SM x groups per trip: 4 x 2 0.461 ms,
// 5 x 2 0.488, 3 x 3 0.489, 3 x 2 0.494, 6 x 1 0.503, 2 x 4 0.578)

struct Seg {  // one stop segment s: position, 1 / width, colour c_s, difference d_s
    float t, r, pad0, pad1;
    float4 c, d;
};

struct ColorParams {
    const float* x;
    const uint32_t* mask;
    uint32_t* rgba;
    int64_t n;        // values
    int cols;         // values per mask row ([planes][rows][cols])
    int n_words;      // mask words per row
    float vmin, big_r;
    uint32_t nan_rgba, mask_rgba;
    int n_seg;        // n_stops - 1
    Seg seg[LCP_MAX_COLOR_STOPS - 1];
};

// Paired add rounded toward minus infinity (add.rm.f32x2).
__device__ __forceinline__ float2 fadd2_rm(float2 a, float2 b) {
    float2 r;
    asm("{.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "add.rm.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

template <int NT, int NA>  // NT >= n_stops - 2 interior stop positions, held in registers
__device__ __forceinline__ uint32_t map_one(const ColorParams& p, const Seg* seg, const float (&thr)[NA], float x) {
    float t = __fmul_rn(__fsub_rn(x, p.vmin), p.big_r);
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    int s = 0;
#pragma unroll
    for (int q = 0; q < NT; ++q) s += t >= thr[q] ? 1 : 0;  // unused entries hold 2 > t
    const Seg& g = seg[s];
    const float f = __fmul_rn(__fsub_rn(t, g.t), g.r);
    const float2 ff = make_float2(f, f);
    const float2 h = make_float2(255.0f, 255.0f), half = make_float2(0.5f, 0.5f);
    const float2 rg = __fadd2_rn(__fmul2_rn(__fadd2_rn(make_float2(g.c.x, g.c.y), __fmul2_rn(ff, make_float2(g.d.x, g.d.y))), h), half);
    const float2 ba = __fadd2_rn(__fmul2_rn(__fadd2_rn(make_float2(g.c.z, g.c.w), __fmul2_rn(ff, make_float2(g.d.z, g.d.w))), h), half);
    // floor of y in [0.4999, 255.5001] (the clamp of the header never binds: f <= 1 + 2^-23 and the
    // colours lie in [0, 1]): y + 2^23 rounded down is 2^23 + floor(y) exactly, so the low byte of its
    // bit pattern is the channel byte; three byte permutes pack r, g, b, a
    const float2 kb = fadd2_rm(rg, make_float2(8388608.0f, 8388608.0f));
    const float2 kc = fadd2_rm(ba, make_float2(8388608.0f, 8388608.0f));
    const uint32_t lo = __byte_perm(__float_as_uint(kb.x), __float_as_uint(kb.y), 0x0040);
    const uint32_t hi = __byte_perm(__float_as_uint(kc.x), __float_as_uint(kc.y), 0x0040);
    const uint32_t c = __byte_perm(lo, hi, 0x5410);
    return x != x ? p.nan_rgba : c;
}

// Mask bits of the cnt values from flat position (row, col) on: one or two
// words when the group lies in one mask row (loaded by the caller: w0, w1),
// element by element when it wraps into the next row.
template <typename Idx>
__device__ __forceinline__ uint32_t group_bits(const ColorParams& p, Idx row, int col, int cnt, uint32_t w0,
                                               uint32_t w1) {
    if (col + cnt <= p.cols) {
        const int sh = col & 31;
        const uint64_t w2 = (uint64_t)w0 | ((uint64_t)w1 << 32);
        return (uint32_t)(w2 >> sh);
    }
    uint32_t bits = 0;
    int cc = col;
    Idx rr = row;
    for (int e = 0; e < cnt; ++e) {
        bits |= ((p.mask[(int64_t)rr * p.n_words + (cc >> 5)] >> (cc & 31)) & 1u) << e;
        if (++cc == p.cols) {
            cc = 0;
            ++rr;
        }
    }
    return bits;
}

// U groups of 4 values per thread and trip: every group's value load (and its
// mask words) is issued before any group is mapped, so U loads per thread are
// in flight instead of one, and the mask read is no second round trip.
template <bool MASK, typename Idx, int NT, int U>
__global__ void __launch_bounds__(kCT, kCB) colormap_kernel(const __grid_constant__ ColorParams p) {
    __shared__ Seg seg[LCP_MAX_COLOR_STOPS - 1];
    for (int q = threadIdx.x; q < p.n_seg; q += kCT) seg[q] = p.seg[q];
    float thr[NT > 0 ? NT : 1];
#pragma unroll
    for (int q = 0; q < NT; ++q) thr[q] = q + 1 < p.n_seg ? p.seg[q + 1].t : 2.0f;
    __syncthreads();
    const bool vec = ((reinterpret_cast<uintptr_t>(p.x) | reinterpret_cast<uintptr_t>(p.rgba)) & 15) == 0;
    const Idx n = (Idx)p.n;
    const Idx g0 = ((Idx)blockIdx.x * kCT + threadIdx.x) * 4, step = (Idx)gridDim.x * kCT * 4;
    // mask position of the trip's first group, advanced by the stride without division
    int col = 0, dcol = 0;
    Idx row = 0, drow = 0;
    if (MASK) {
        row = g0 / (Idx)p.cols;
        col = (int)(g0 - row * (Idx)p.cols);
        drow = step / (Idx)p.cols;
        dcol = (int)(step - drow * (Idx)p.cols);
    }
    for (Idx g = g0; g < n; g += (Idx)U * step) {
        float x[U][4];
        int cnt[U];
        uint32_t mw0[U], mw1[U];
        Idx mrow[U];
        int mcol[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {  // issue every load of the trip
            const Idx gk = g + (Idx)k * step;
            cnt[k] = gk >= n ? 0 : (n - gk >= 4 ? 4 : (int)(n - gk));
            if (vec && cnt[k] == 4) {
                const float4 r = __ldcs(reinterpret_cast<const float4*>(p.x + gk));
                x[k][0] = r.x;
                x[k][1] = r.y;
                x[k][2] = r.z;
                x[k][3] = r.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) x[k][e] = e < cnt[k] ? p.x[gk + e] : 0.0f;
            }
            if (MASK) {
                mrow[k] = row;
                mcol[k] = col;
                mw0[k] = mw1[k] = 0u;
                if (cnt[k] > 0 && col + cnt[k] <= p.cols) {
                    const uint32_t* wp = p.mask + (int64_t)row * p.n_words + (col >> 5);
                    mw0[k] = wp[0];
                    if ((col & 31) + cnt[k] > 32) mw1[k] = wp[1];
                }
                col += dcol;
                row += drow;
                if (col >= p.cols) {
                    col -= p.cols;
                    ++row;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            if (cnt[k] == 0) break;
            const Idx gk = g + (Idx)k * step;
            uint32_t c[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) c[e] = map_one<NT>(p, seg, thr, x[k][e]);
            if (MASK) {
                const uint32_t bits = group_bits<Idx>(p, mrow[k], mcol[k], cnt[k], mw0[k], mw1[k]);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (((bits >> e) & 1u) && x[k][e] == x[k][e]) c[e] = p.mask_rgba;  // NaN keeps its colour
            }
            if (vec && cnt[k] == 4) {
                __stcs(reinterpret_cast<uint4*>(p.rgba + gk), make_uint4(c[0], c[1], c[2], c[3]));
            } else {
                for (int e = 0; e < cnt[k]; ++e) p.rgba[gk + e] = c[e];
            }
        }
    }
}

template <bool MASK, typename Idx>
void launch_nt(const ColorParams& p, int grid, cudaStream_t st) {
    const int interior = p.n_seg - 1;  // stop positions strictly inside (0, 1)
    if (interior == 0) colormap_kernel<MASK, Idx, 0, kCU><<<grid, kCT, 0, st>>>(p);
    else if (interior <= 2) colormap_kernel<MASK, Idx, 2, kCU><<<grid, kCT, 0, st>>>(p);
    else if (interior <= 4) colormap_kernel<MASK, Idx, 4, kCU><<<grid, kCT, 0, st>>>(p);
    else if (interior <= 6) colormap_kernel<MASK, Idx, 6, kCU><<<grid, kCT, 0, st>>>(p);
    else colormap_kernel<MASK, Idx, LCP_MAX_COLOR_STOPS - 2, kCU><<<grid, kCT, 0, st>>>(p);
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
    {
        volatile float lo = vmin, hi = vmax;
        volatile float range = hi - lo;
        if (!std::isfinite((float)range))
            return fail(LCP_ERR_ARG, "%s: vmax - vmin overflows fp32", fn);
    }
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
    p.n_words = (cols + 31) / 32;
    // the once-per-call terms, each one fp32 operation (volatile keeps the host
    // compiler from contracting or widening them)
    volatile float lo = vmin, hi = vmax;
    volatile float range = hi - lo;
    volatile float big_r = 1.0f / range;
    p.vmin = vmin;
    p.big_r = big_r;
    p.nan_rgba = nan_rgba;
    p.mask_rgba = mask_rgba;
    p.n_seg = n_stops - 1;
    for (int q = 0; q + 1 < n_stops; ++q) {
        const float* a = stops + 5 * q;
        const float* b = a + 5;
        volatile float w = b[0] - a[0];
        volatile float r = 1.0f / w;
        Seg& sg = p.seg[q];
        sg.t = a[0];
        sg.r = r;
        sg.pad0 = sg.pad1 = 0.0f;
        float d[4];
        for (int c = 0; c < 4; ++c) {
            volatile float dc = b[1 + c] - a[1 + c];
            d[c] = dc;
        }
        sg.c = make_float4(a[1], a[2], a[3], a[4]);
        sg.d = make_float4(d[0], d[1], d[2], d[3]);
    }
    const int64_t groups = (n + 3) / 4;
    const int grid = (int)std::min<int64_t>((groups + kCT - 1) / kCT, (int64_t)num_sms() * kCB);
    cudaStream_t st = (cudaStream_t)stream;
    const bool small = n < (1ll << 31) - 4 * (int64_t)kCT * grid;
    if (mask) {
        if (small) launch_nt<true, uint32_t>(p, grid, st);
        else launch_nt<true, int64_t>(p, grid, st);
    } else {
        if (small) launch_nt<false, uint32_t>(p, grid, st);
        else launch_nt<false, int64_t>(p, grid, st);
    }
    return check_launch(fn);
}
