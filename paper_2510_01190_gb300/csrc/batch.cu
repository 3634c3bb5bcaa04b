// Batched closed form: many fields of uneven size in one persistent launch.
//
// Work list: every field is cut into tiles of R cell rows x TW cell columns;
// the tiles of all fields form one list (fields ordered by cost, a prefix sum
// of tile counts per field and tile shape in the workspace).  Each CTA of a
// persistent grid takes the next tile from an atomic counter and evaluates it
// completely on its own:
//   1. the ensemble statistics (shifted FP32 sums) of the tile's vertices and
//      their one-vertex halo -- rows a-1 .. e+1, columns c0-1 .. ce+1 -- into
//      shared memory;
//   2. the divergence Gaussian of Eqs. 2/3 (one-sided at the field's edges) of
//      each tile vertex, into registers;
//   3. per pair of isovalues, (P(D < c), P(D >= c)) of every tile vertex into
//      shared memory, then the LCP of Sec. 3.2 and the mean-field bit of every
//      cell, straight to the field's outputs.
// No CTA waits on another; the halo re-read is (R+3)(TW+3) / (R TW) - 1 of the
// tile's member bytes (about 10 % for 64 x 64 tiles, partly served by L2).
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "lcp_common.cuh"

namespace lcp {
namespace {

constexpr int kBT = 256;    // threads per CTA
constexpr int kShapes = 4;  // tile shapes of lcp_tune, in its documented order
constexpr int kShapeR[kShapes] = {64, 32, 32, 16};
constexpr int kShapeC[kShapes] = {64, 128, 64, 128};

struct FieldRec {
    const void* u;
    const void* v;
    void* out;
    uint32_t* mask;
    int64_t stride;
    int M, H, W, ddof;
    int K, iso_begin, n_words, pad;
    Spacing sp;
};

// Workspace: [256-byte header: tile counter] [FieldRec x n] [int32 prefix
// (n+1) per tile shape] [isovalues]
struct WsLayout {
    size_t rec, pre, iso, total;
};
inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }
WsLayout ws_layout(int n_fields, int n_iso) {
    WsLayout L;
    L.rec = 256;
    L.pre = L.rec + up256((size_t)n_fields * sizeof(FieldRec));
    L.iso = L.pre + up256((size_t)kShapes * (n_fields + 1) * sizeof(int));
    L.total = L.iso + up256((size_t)n_iso * sizeof(float));
    return L;
}

template <typename T>
__device__ __forceinline__ float ldm(const T* p);
template <>
__device__ __forceinline__ float ldm<float>(const float* p) {
    return __ldg(p);
}
template <>
__device__ __forceinline__ float ldm<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short*>(p))));
}

// Shifted sums of u and v over the members of two vertices at once (offsets o0,
// o1 in a member plane), 8 members per step: 32 loads in flight per thread.
template <typename T>
__device__ __forceinline__ void member_sums2(const T* __restrict__ u, const T* __restrict__ v, int64_t stride, int M,
                                             int64_t o0, int64_t o1, float (&x0)[4], float (&s1)[4],
                                             float (&s2)[4]) {
    const T* b[4] = {u + o0, v + o0, u + o1, v + o1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        s1[q] = 0.f;
        s2[q] = 0.f;
    }
    int m = 1;
    if (M >= 8) {  // member 0 (the shift) travels with members 1 .. 7: one round trip fewer
        float x[8][4];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) x[r][q] = ldm(b[q] + (int64_t)r * stride);
#pragma unroll
        for (int q = 0; q < 4; ++q) x0[q] = x[0][q];
#pragma unroll
        for (int r = 1; r < 8; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float d = x[r][q] - x0[q];
                s1[q] += d;
                s2[q] = fmaf(d, d, s2[q]);
            }
        m = 8;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) x0[q] = ldm(b[q]);
    }
    for (; m + 8 <= M; m += 8) {
        float x[8][4];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) x[r][q] = ldm(b[q] + (int64_t)(m + r) * stride);
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float d = x[r][q] - x0[q];
                s1[q] += d;
                s2[q] = fmaf(d, d, s2[q]);
            }
    }
    for (; m < M; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float d = ldm(b[q] + (int64_t)m * stride) - x0[q];
            s1[q] += d;
            s2[q] = fmaf(d, d, s2[q]);
        }
}

// (mean - ref, variance) from the shifted sums; the mean keeps the member-0
// shift apart from the small shifted mean until the reference is removed.
__device__ __forceinline__ float2 mean_var(float x0, float s1, float s2, float ref, float fm, float fdof) {
    const float dl = s1 / fm;
    float vv = (s2 - s1 * dl) / fdof;
    vv = vv < 0.f ? 0.f : vv;  // NaN stays NaN
    return make_float2((x0 - ref) + dl, vv);
}

template <typename T, typename OutT, int R, int TW>
// At most 64 registers (a few bytes of spill): 4 resident CTAs per SM instead of 3, so
// that more CTAs are in their member stream while others run the barrier-separated LCP
// phases (measured, 64 fields, 32 x 64 tiles: 3.556 -> 3.297 ms, identical maps).
__global__ void __launch_bounds__(kBT, 4) batch_kernel(const FieldRec* __restrict__ fr, const int* __restrict__ prefix,
                                                   int n_fields, const float* __restrict__ isos, uint32_t* ctr) {
    static_assert(TW % 32 == 0 && kBT % TW == 0, "a warp covers 32 cells of one row");
    constexpr int NR = R + 3, NC = TW + 3;  // statistics region (stride NC)
    constexpr int NVMAX = (R + 1) * (TW + 1);
    constexpr int PER = (NVMAX + kBT - 1) / kBT;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* su = reinterpret_cast<float2*>(smem);  // [NR][NC] (mean - ref, var) of u
    float2* sv = su + NR * NC;                     // [NR][NC] of v
    float2* pq0 = su;                              // [NVMAX] after the divergence (aliases su, sv)
    float2* pq1 = su + NVMAX;
    uint8_t* cls = reinterpret_cast<uint8_t*>(sv + NR * NC);  // [NVMAX] class bits of the pair
    __shared__ int s_tile;

    const int t = threadIdx.x, lane = t & 31;
    const int n_tiles = __ldg(prefix + n_fields);
    for (;;) {
        if (t == 0) s_tile = (int)atomicAdd(ctr, 1u);
        __syncthreads();
        const int g = s_tile;
        if (g >= n_tiles) break;
        int lo = 0, hi = n_fields - 1;  // the field of tile g: last f with prefix[f] <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(prefix + mid) <= g) lo = mid;
            else hi = mid - 1;
        }
        const FieldRec& F = fr[lo];
        const T* __restrict__ u = reinterpret_cast<const T*>(F.u);
        const T* __restrict__ v = reinterpret_cast<const T*>(F.v);
        const int H = F.H, W = F.W, Hc = H - 1, Wc = W - 1, M = F.M;
        const int64_t stride = F.stride;
        const int nbc = (Wc + TW - 1) / TW;
        const int local = g - __ldg(prefix + lo);
        const int a = (local / nbc) * R, c0 = (local % nbc) * TW;
        const int e = min(a + R, Hc), ce = min(c0 + TW, Wc);  // cells [a, e) x [c0, ce); vertices a..e, c0..ce
        const int rb = max(a - 1, 0), cb = max(c0 - 1, 0);
        const int nr = min(e + 1, H - 1) - rb + 1, nc = min(ce + 1, W - 1) - cb + 1;

        // 1. statistics of the region, two vertices per thread and step
        float refu = ldm(u + (int64_t)a * W + c0), refv = ldm(v + (int64_t)a * W + c0);
        if (!isfinite(refu)) refu = 0.f;
        if (!isfinite(refv)) refv = 0.f;
        const float fm = (float)M, fdof = (float)(M - F.ddof);
        const int nreg = nr * nc;
        for (int q = t; q < nreg; q += 2 * kBT) {
            const int qb = min(q + kBT, nreg - 1);
            const int r0 = q / nc, r1 = qb / nc;
            const int x0c = q - r0 * nc, x1c = qb - r1 * nc;
            float x0[4], s1[4], s2[4];
            member_sums2<T>(u, v, stride, M, (int64_t)(rb + r0) * W + cb + x0c, (int64_t)(rb + r1) * W + cb + x1c,
                            x0, s1, s2);
            su[r0 * NC + x0c] = mean_var(x0[0], s1[0], s2[0], refu, fm, fdof);
            sv[r0 * NC + x0c] = mean_var(x0[1], s1[1], s2[1], refv, fm, fdof);
            if (q + kBT < nreg) {
                su[r1 * NC + x1c] = mean_var(x0[2], s1[2], s2[2], refu, fm, fdof);
                sv[r1 * NC + x1c] = mean_var(x0[3], s1[3], s2[3], refv, fm, fdof);
            }
        }
        __syncthreads();

        // 2. divergence Gaussian of the tile's vertices (Eqs. 2/3), one-sided at the edges
        const int nvc = ce - c0 + 1, nv = (e - a + 1) * nvc;
        const Spacing sp = F.sp;
        float dmu[PER], ds[PER];
#pragma unroll
        for (int s = 0; s < PER; ++s) {
            const int p = t + s * kBT;
            dmu[s] = 0.f;
            ds[s] = 0.f;
            if (p < nv) {
                const int jj = p / nvc, ii = p - jj * nvc;
                const int j = a + jj, i = c0 + ii;
                const int ry = j - rb, rx = i - cb;
                const float2 L = su[ry * NC + (i > 0 ? rx - 1 : rx)];
                const float2 Rr = su[ry * NC + (i < W - 1 ? rx + 1 : rx)];
                const float2 Vl = sv[(j > 0 ? ry - 1 : ry) * NC + rx];
                const float2 Vh = sv[(j < H - 1 ? ry + 1 : ry) * NC + rx];
                const bool osx = i == 0 || i == W - 1, osy = j == 0 || j == H - 1;
                const float sx = osx ? sp.sx1 : sp.sx2, sxq = osx ? sp.sx1q : sp.sx2q;
                const float sy = osy ? sp.sy1 : sp.sy2, syq = osy ? sp.sy1q : sp.sy2q;
                dmu[s] = fmaf(Rr.x - L.x, sx, (Vh.x - Vl.x) * sy);
                const float var = fmaf(Rr.y + L.y, sxq, (Vh.y + Vl.y) * syq);
                ds[s] = var == 0.0f ? -1.0f : rsqrtf(2.0f * var);  // -1 marks zero variance; NaN stays NaN
            }
        }
        __syncthreads();  // the statistics are dead; their space holds (p, q) from here on

        // 3. isovalues in pairs: vertex (p, q) and class bits, then the cells
        const int K = F.K, ib = F.iso_begin;
        const int64_t plane = (int64_t)Hc * Wc, mplane = (int64_t)Hc * F.n_words;
        OutT* out = reinterpret_cast<OutT*>(F.out);
        uint32_t* mask = F.mask;
        for (int kk = 0; kk < K; kk += 2) {
            const bool two = kk + 1 < K;
            const float2 c = make_float2(__ldg(isos + ib + kk), __ldg(isos + ib + (two ? kk + 1 : kk)));
#pragma unroll
            for (int s = 0; s < PER; ++s) {
                const int p = t + s * kBT;
                if (p < nv) {
                    const bool b0 = dmu[s] < c.x, b1 = dmu[s] < c.y;
                    float2 a0, a1;
                    vertex_pq2(dmu[s], ds[s], ds[s] < 0.0f, c, b0, b1, a0, a1);
                    pq0[p] = a0;
                    pq1[p] = a1;
                    cls[p] = (uint8_t)(b0 | (b1 << 1));
                }
            }
            __syncthreads();
            const int cc = t % TW;
#pragma unroll 4
            for (int rr = t / TW; rr < R; rr += kBT / TW) {
                const bool ok = a + rr < e && c0 + cc < ce;
                uint32_t cross = 0;
                const int64_t o = (int64_t)(a + rr) * Wc + c0 + cc;
                if (ok) {
                    const int p = rr * nvc + cc;
                    const uint32_t k00 = cls[p], k01 = cls[p + 1], k10 = cls[p + nvc], k11 = cls[p + nvc + 1];
                    cross = (k00 | k01 | k10 | k11) & ~(k00 & k01 & k10 & k11);
                    {
                        const float2 top = __fmul2_rn(pq0[p], pq0[p + 1]);
                        const float2 bot = __fmul2_rn(pq0[p + nvc], pq0[p + nvc + 1]);
                        const float l = fmaf(-top.y, bot.y, fmaf(-top.x, bot.x, 1.0f));
                        out[(int64_t)kk * plane + o] = to_out<OutT>(clamp01_nan(l));
                    }
                    if (two) {
                        const float2 top = __fmul2_rn(pq1[p], pq1[p + 1]);
                        const float2 bot = __fmul2_rn(pq1[p + nvc], pq1[p + nvc + 1]);
                        const float l = fmaf(-top.y, bot.y, fmaf(-top.x, bot.x, 1.0f));
                        out[(int64_t)(kk + 1) * plane + o] = to_out<OutT>(clamp01_nan(l));
                    }
                }
                if (mask) {  // uniform per warp: its 32 cells share one row and one mask word
                    const uint32_t w0 = __ballot_sync(0xFFFFFFFFu, cross & 1u);
                    const uint32_t w1 = __ballot_sync(0xFFFFFFFFu, (cross >> 1) & 1u);
                    const int word = (c0 + (cc & ~31)) >> 5;
                    if (lane == 0 && a + rr < e && word < F.n_words) {
                        uint32_t* mw = mask + ((int64_t)kk * Hc + a + rr) * F.n_words + word;
                        *mw = w0;
                        if (two) mw[mplane] = w1;
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <int R, int TW>
constexpr size_t smem_bytes() {
    return (size_t)2 * (R + 3) * (TW + 3) * sizeof(float2) + (size_t)(R + 1) * (TW + 1);
}

using KernelFn = void (*)(const FieldRec*, const int*, int, const float*, uint32_t*);

template <typename T, typename OutT>
KernelFn pick_kernel(int shape, size_t* smem) {
    switch (shape) {
        case 0: *smem = smem_bytes<64, 64>(); return batch_kernel<T, OutT, 64, 64>;
        case 1: *smem = smem_bytes<32, 128>(); return batch_kernel<T, OutT, 32, 128>;
        case 2: *smem = smem_bytes<32, 64>(); return batch_kernel<T, OutT, 32, 64>;
        case 3: *smem = smem_bytes<16, 128>(); return batch_kernel<T, OutT, 16, 128>;
    }
    return nullptr;
}

KernelFn pick(lcp_dtype in, lcp_dtype out, int shape, size_t* smem) {
    if (in == LCP_F32) return out == LCP_F16 ? pick_kernel<float, __half>(shape, smem) : pick_kernel<float, float>(shape, smem);
    return out == LCP_F16 ? pick_kernel<__nv_bfloat16, __half>(shape, smem)
                          : pick_kernel<__nv_bfloat16, float>(shape, smem);
}

int shape_index(const lcp_tune* tune) {
    if (!tune) return 0;
    for (int s = 0; s < kShapes; ++s)
        if (tune->tile_rows == kShapeR[s] && tune->tile_cols == kShapeC[s]) return s;
    return -1;
}

// Shared-memory limit of every kernel variant, once per device.
lcp_status set_smem_limits(lcp_dtype in, lcp_dtype out) {
    static std::mutex mu;
    static bool done[64][4] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return fail(LCP_ERR_CUDA, "lcp_batch: no usable current device");
    }
    const int combo = (in == LCP_BF16 ? 2 : 0) + (out == LCP_F16 ? 1 : 0);
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev][combo]) return LCP_OK;
    for (int s = 0; s < kShapes; ++s) {
        size_t smem = 0;
        KernelFn k = pick(in, out, s, &smem);
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            cudaGetLastError();
            return fail(LCP_ERR_CUDA, "lcp_batch: %zu bytes of shared memory not available", smem);
        }
    }
    done[dev][combo] = true;
    return LCP_OK;
}

lcp_status check_plan(const char* fn, const lcp_batch_plan* plan) {
    if (!plan || !plan->workspace || plan->n_fields < 1 || plan->n_iso < 1)
        return fail(LCP_ERR_ARG, "%s: plan is NULL or not prepared", fn);
    if ((plan->in_dtype != LCP_F32 && plan->in_dtype != LCP_BF16) ||
        (plan->out_dtype != LCP_F32 && plan->out_dtype != LCP_F16))
        return fail(LCP_ERR_ARG, "%s: plan has unsupported dtypes", fn);
    if (plan->workspace_bytes < ws_layout(plan->n_fields, plan->n_iso).total)
        return fail(LCP_ERR_ARG, "%s: plan workspace too small", fn);
    return LCP_OK;
}

lcp_status launch(const lcp_batch_plan* plan, int shape, int ctas_per_sm, cudaStream_t st) {
    size_t smem = 0;
    KernelFn k = pick(plan->in_dtype, plan->out_dtype, shape, &smem);
    lcp_status s = set_smem_limits(plan->in_dtype, plan->out_dtype);
    if (s != LCP_OK) return s;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kBT, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return fail(LCP_ERR_CUDA, "lcp_batch: kernel does not fit on an SM");
    }
    if (ctas_per_sm > 0) occ = std::min(occ, ctas_per_sm);
    const WsLayout L = ws_layout(plan->n_fields, plan->n_iso);
    char* ws = reinterpret_cast<char*>(plan->workspace);
    uint32_t* ctr = reinterpret_cast<uint32_t*>(ws);
    if (cudaMemsetAsync(ctr, 0, sizeof(uint32_t), st) != cudaSuccess) {
        cudaGetLastError();
        return fail(LCP_ERR_CUDA, "lcp_batch: counter reset failed");
    }
    const int* prefix = reinterpret_cast<const int*>(ws + L.pre) + (size_t)shape * (plan->n_fields + 1);
    k<<<num_sms() * occ, kBT, smem, st>>>(reinterpret_cast<const FieldRec*>(ws + L.rec), prefix, plan->n_fields,
                                         reinterpret_cast<const float*>(ws + L.iso), ctr);
    return check_launch("lcp_batch");
}

}  // namespace
}  // namespace lcp

using namespace lcp;

extern "C" size_t lcp_batch_workspace_bytes(int n_fields, int n_iso) {
    if (n_fields < 1 || n_iso < 1) return 0;
    return ws_layout(n_fields, n_iso).total;
}

extern "C" lcp_status lcp_batch_prepare(const lcp_field_desc* fields, int n_fields, const float* iso, int n_iso,
                                        lcp_dtype in_dtype, lcp_dtype out_dtype, void* workspace,
                                        size_t workspace_bytes, lcp_stream_t stream, lcp_batch_plan* plan) {
    static const char* fn = "lcp_batch_prepare";
    if (!fields || n_fields < 1) return fail(LCP_ERR_ARG, "%s: need at least one field", fn);
    if (!plan) return fail(LCP_ERR_ARG, "%s: NULL plan", fn);
    if (in_dtype != LCP_F32 && in_dtype != LCP_BF16) return fail(LCP_ERR_ARG, "%s: in dtype must be F32 or BF16", fn);
    if (out_dtype != LCP_F32 && out_dtype != LCP_F16) return fail(LCP_ERR_ARG, "%s: out dtype must be F32 or F16", fn);
    if (!iso || n_iso < 1) return fail(LCP_ERR_ARG, "%s: iso must be a non-NULL host table of n_iso >= 1 values", fn);
    lcp_status s = LCP_OK;
    const WsLayout L = ws_layout(n_fields, n_iso);
    if (!workspace || ((uintptr_t)workspace & 255)) return fail(LCP_ERR_ARG, "%s: workspace must be 256-byte aligned", fn);
    if (workspace_bytes < L.total)
        return fail(LCP_ERR_ARG, "%s: workspace too small (%zu < %zu bytes)", fn, workspace_bytes, L.total);
    const size_t in_el = in_dtype == LCP_F32 ? 4 : 2, out_el = out_dtype == LCP_F32 ? 4 : 2;
    std::vector<FieldRec> rec(n_fields);
    lcp_batch_plan P = {};
    for (int f = 0; f < n_fields; ++f) {
        const lcp_field_desc& d = fields[f];
        if ((s = check_members(fn, d.u, d.v, in_dtype, d.M, d.H, d.W, d.member_stride, d.ddof)) != LCP_OK ||
            (s = check_spacing(fn, d.dx, d.dy)) != LCP_OK) {
            char msg[512];
            snprintf(msg, sizeof(msg), "%s", lcp_last_error());
            return fail(s, "field %d: %s", f, msg);
        }
        if (d.K < 1 || d.K > LCP_MAX_ISOVALUES || d.iso_begin < 0 || (int64_t)d.iso_begin + d.K > n_iso)
            return fail(LCP_ERR_ARG, "%s: field %d: isovalues [%d, %d+%d) outside the table of %d", fn, f, d.iso_begin,
                        d.iso_begin, d.K, n_iso);
        if (!d.lcp_out || ((uintptr_t)d.lcp_out & (out_el - 1)))
            return fail(LCP_ERR_ARG, "%s: field %d: NULL or misaligned output", fn, f);
        if ((uintptr_t)d.mask & 3) return fail(LCP_ERR_ARG, "%s: field %d: mask must be 4-byte aligned", fn, f);
        FieldRec& r = rec[f];
        r.u = d.u;
        r.v = d.v;
        r.out = d.lcp_out;
        r.mask = d.mask;
        r.stride = d.M > 1 ? d.member_stride : (int64_t)d.H * d.W;
        r.M = d.M;
        r.H = d.H;
        r.W = d.W;
        r.ddof = d.ddof;
        r.K = d.K;
        r.iso_begin = d.iso_begin;
        r.n_words = (d.W - 1 + 31) / 32;
        r.pad = 0;
        r.sp = make_spacing(d.dx, d.dy);
        const int64_t cells = (int64_t)(d.H - 1) * (d.W - 1);
        P.cells += cells;
        P.cell_isovalues += cells * d.K;
        P.member_bytes += (int64_t)2 * d.M * d.H * d.W * (int64_t)in_el;
        P.out_bytes += cells * d.K * (int64_t)out_el + (d.mask ? (int64_t)d.K * (d.H - 1) * r.n_words * 4 : 0);
    }
    // costliest fields first (member bytes per cell), so that the last tiles are cheap ones
    std::stable_sort(rec.begin(), rec.end(), [](const FieldRec& x, const FieldRec& y) { return x.M > y.M; });
    std::vector<unsigned char> host(L.total, 0);
    memcpy(host.data() + L.rec, rec.data(), rec.size() * sizeof(FieldRec));
    int* pre = reinterpret_cast<int*>(host.data() + L.pre);
    for (int sh = 0; sh < kShapes; ++sh) {
        int64_t acc = 0;
        int* p = pre + (size_t)sh * (n_fields + 1);
        for (int f = 0; f < n_fields; ++f) {
            p[f] = (int)acc;
            const int64_t tiles = (int64_t)((rec[f].H - 1 + kShapeR[sh] - 1) / kShapeR[sh]) *
                                  ((rec[f].W - 1 + kShapeC[sh] - 1) / kShapeC[sh]);
            acc += tiles;
            if (acc > INT_MAX - 1) return fail(LCP_ERR_ARG, "%s: more than 2^31 tiles", fn);
        }
        p[n_fields] = (int)acc;
    }
    memcpy(host.data() + L.iso, iso, (size_t)n_iso * sizeof(float));
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(workspace, host.data(), L.total, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        return fail(LCP_ERR_CUDA, "%s: work table copy failed: %s", fn, cudaGetErrorString(e));
    }
    if ((s = set_smem_limits(in_dtype, out_dtype)) != LCP_OK) return s;
    P.workspace = workspace;
    P.workspace_bytes = workspace_bytes;
    P.n_fields = n_fields;
    P.n_iso = n_iso;
    P.in_dtype = in_dtype;
    P.out_dtype = out_dtype;
    *plan = P;
    return LCP_OK;
}

extern "C" lcp_status lcp_batch(const lcp_batch_plan* plan, const lcp_tune* tune, lcp_stream_t stream) {
    lcp_status s = check_plan("lcp_batch", plan);
    if (s != LCP_OK) return s;
    const int shape = shape_index(tune);
    if (shape < 0)
        return fail(LCP_ERR_ARG, "lcp_batch: tile %d x %d is not one of 64x64, 32x128, 32x64, 16x128", tune->tile_rows,
                    tune->tile_cols);
    if (tune && tune->ctas_per_sm < 0) return fail(LCP_ERR_ARG, "lcp_batch: ctas_per_sm < 0");
    return launch(plan, shape, tune ? tune->ctas_per_sm : 0, (cudaStream_t)stream);
}

extern "C" lcp_status lcp_batch_autotune(const lcp_batch_plan* plan, int reps, lcp_tune* best, float* ms,
                                         lcp_stream_t stream) {
    lcp_status s = check_plan("lcp_batch_autotune", plan);
    if (s != LCP_OK) return s;
    if (!best || reps < 1) return fail(LCP_ERR_ARG, "lcp_batch_autotune: NULL best or reps < 1");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return fail(LCP_ERR_CUDA, "lcp_batch_autotune: event creation failed");
    }
    float best_ms = 0.f;
    int best_shape = -1;
    for (int sh = 0; sh < kShapes && s == LCP_OK; ++sh) {
        if ((s = launch(plan, sh, 0, st)) != LCP_OK) break;  // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && s == LCP_OK; ++r) s = launch(plan, sh, 0, st);
        cudaEventRecord(e1, st);
        if (s != LCP_OK) break;
        float t = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            cudaGetLastError();
            s = fail(LCP_ERR_CUDA, "lcp_batch_autotune: timing failed");
            break;
        }
        t /= reps;
        if (ms) ms[sh] = t;
        if (best_shape < 0 || t < best_ms) {
            best_ms = t;
            best_shape = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != LCP_OK) return s;
    best->tile_rows = kShapeR[best_shape];
    best->tile_cols = kShapeC[best_shape];
    best->ctas_per_sm = 0;
    return LCP_OK;
}
