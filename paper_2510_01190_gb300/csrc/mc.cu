// lcp_mc: the classical Monte Carlo LCP estimator the paper compares against
// (Sec. 3.2 and Sec. 4): each sample is one realisation of the whole uncertain
// field; its divergence (Eq. 1, one-sided at the boundary) is tested per cell,
// a cell crossing isovalue c when min < c <= max over its 4 vertices.
//
// One CTA owns a 32 x 8 tile of cells.  Per sample pair it draws the field on
// the tile's vertices plus a one-vertex halo into shared memory (Philox is
// keyed by the global vertex index, so halo draws equal the neighbour tile's),
// forms the divergence of both samples, and updates per-cell counters held in
// registers.  The work is ALU-bound (Philox rounds, log, sqrt, sincos).
#include "lcp_common.cuh"

namespace lcp {
namespace {

constexpr int kTX = 32, kTY = 8;               // cells per tile
constexpr int kThreads = kTX * kTY;            // one cell per thread
constexpr int kVX = kTX + 3, kVY = kTY + 3;    // draw region: columns -1..kTX+1, rows -1..kTY+1
constexpr int kNV = kVX * kVY;                 // 385 draw vertices
constexpr int kDX = kTX + 1, kDY = kTY + 1;    // divergence vertices of the tile
constexpr int kND = kDX * kDY;                 // 297
constexpr int kVPT = (kNV + kThreads - 1) / kThreads;  // draw vertices per thread (2)
constexpr int kKReg = 16;                      // isovalues per launch (counters live in registers)

struct McParams {
    const float *mu_u, *var_u, *mu_v, *var_v;  // GAUSS
    const void *u, *v;                          // EMPIRICAL
    int M;
    int64_t stride;
    int H, W;
    Spacing sp;
    uint2 key, off;
    uint64_t n_samples;
    uint32_t* counts;
    float* est;
};

template <typename T>
__device__ __forceinline__ float member_at(const void* base, int64_t idx) {
    float x;
    Loader<T, 1>::cvt(Loader<T, 1>::load(reinterpret_cast<const T*>(base) + idx), &x);
    return x;
}

template <int MODE, typename T>
__global__ void __launch_bounds__(kThreads) mc_kernel(const __grid_constant__ McParams p,
                                                      const __grid_constant__ IsoParams iso, int kbase) {
    __shared__ float su[2][kNV], sv[2][kNV];
    __shared__ float sd[2][kND];
    const int tid = threadIdx.x;
    const int cx0 = blockIdx.x * kTX, cy0 = blockIdx.y * kTY;
    const int H = p.H, W = p.W, Hc = H - 1, Wc = W - 1;

    // draw vertices owned by this thread: global index and Gaussian parameters
    uint32_t vn[kVPT];
    bool vok[kVPT];
    float mu_u[kVPT], sd_u[kVPT], mu_v[kVPT], sd_v[kVPT];
#pragma unroll
    for (int r = 0; r < kVPT; ++r) {
        const int lv = tid + r * kThreads;
        const int gi = cx0 - 1 + lv % kVX, gj = cy0 - 1 + lv / kVX;
        vok[r] = lv < kNV && gi >= 0 && gi < W && gj >= 0 && gj < H;
        vn[r] = vok[r] ? (uint32_t)gj * (uint32_t)W + (uint32_t)gi : 0u;
        mu_u[r] = sd_u[r] = mu_v[r] = sd_v[r] = 0.f;
        if (MODE == LCP_MC_GAUSS && vok[r]) {
            mu_u[r] = p.mu_u[vn[r]];
            sd_u[r] = sqrtf(p.var_u[vn[r]]);
            mu_v[r] = p.mu_v[vn[r]];
            sd_v[r] = sqrtf(p.var_v[vn[r]]);
        }
    }
    // this thread's cell
    const int ci = cx0 + tid % kTX, cj = cy0 + tid / kTX;
    const bool cok = ci < Wc && cj < Hc;
    const int lci = tid % kTX, lcj = tid / kTX;  // its corner (i, j) in the divergence region

    uint32_t cnt[kKReg];
#pragma unroll
    for (int k = 0; k < kKReg; ++k) cnt[k] = 0;

    const uint64_t n_pairs = (p.n_samples + 1) / 2;
    for (uint64_t t = 0; t < n_pairs; ++t) {
        // 1) draw both samples of the pair on the tile + halo
#pragma unroll
        for (int r = 0; r < kVPT; ++r) {
            const int lv = tid + r * kThreads;
            if (!vok[r]) continue;
            const uint4 w = philox4x32_10(make_uint4(vn[r], (uint32_t)t, p.off.x, p.off.y), p.key);
            if (MODE == LCP_MC_GAUSS) {
                float zu0, zv0, zu1, zv1;
                box_muller(w.x, w.y, zu0, zv0);
                box_muller(w.z, w.w, zu1, zv1);
                su[0][lv] = fmaf(sd_u[r], zu0, mu_u[r]);
                sv[0][lv] = fmaf(sd_v[r], zv0, mu_v[r]);
                su[1][lv] = fmaf(sd_u[r], zu1, mu_u[r]);
                sv[1][lv] = fmaf(sd_v[r], zv1, mu_v[r]);
            } else {
                const uint32_t m = (uint32_t)p.M;
                su[0][lv] = member_at<T>(p.u, (int64_t)__umulhi(w.x, m) * p.stride + vn[r]);
                sv[0][lv] = member_at<T>(p.v, (int64_t)__umulhi(w.y, m) * p.stride + vn[r]);
                su[1][lv] = member_at<T>(p.u, (int64_t)__umulhi(w.z, m) * p.stride + vn[r]);
                sv[1][lv] = member_at<T>(p.v, (int64_t)__umulhi(w.w, m) * p.stride + vn[r]);
            }
        }
        __syncthreads();
        // 2) divergence (Eq. 1) of both samples at the tile's vertices
        for (int d = tid; d < kND; d += kThreads) {
            const int li = d % kDX, lj = d / kDX;
            const int gi = cx0 + li, gj = cy0 + lj;
            if (gi >= W || gj >= H) continue;
            const int ilo = gi > 0 ? gi - 1 : 0, ihi = gi < W - 1 ? gi + 1 : W - 1;
            const int jlo = gj > 0 ? gj - 1 : 0, jhi = gj < H - 1 ? gj + 1 : H - 1;
            const float sx = (ihi - ilo == 2) ? p.sp.sx2 : p.sp.sx1;
            const float sy = (jhi - jlo == 2) ? p.sp.sy2 : p.sp.sy1;
            // draw-region coordinates are offset by the halo of 1
            const int r = (gj - cy0 + 1) * kVX;
            const int a = r + (ihi - cx0 + 1), b = r + (ilo - cx0 + 1);
            const int cc = gi - cx0 + 1;
            const int hi = (jhi - cy0 + 1) * kVX + cc, lo = (jlo - cy0 + 1) * kVX + cc;
#pragma unroll
            for (int s = 0; s < 2; ++s) sd[s][d] = fmaf(su[s][a] - su[s][b], sx, (sv[s][hi] - sv[s][lo]) * sy);
        }
        __syncthreads();
        // 3) crossing test of this thread's cell for both samples
        if (cok) {
            const bool has2 = 2 * t + 1 < p.n_samples;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (s == 1 && !has2) break;
                const float d00 = sd[s][lcj * kDX + lci], d10 = sd[s][lcj * kDX + lci + 1];
                const float d01 = sd[s][(lcj + 1) * kDX + lci], d11 = sd[s][(lcj + 1) * kDX + lci + 1];
                const float mn = fminf(fminf(d00, d10), fminf(d01, d11));
                const float mx = fmaxf(fmaxf(d00, d10), fmaxf(d01, d11));
#pragma unroll
                for (int k = 0; k < kKReg; ++k)
                    if (k < iso.K) cnt[k] += (mn < iso.c[k] && mx >= iso.c[k]) ? 1u : 0u;
            }
        }
        // the next pair's draws write su/sv only; sd is rewritten after its barrier
    }
    if (!cok) return;
    const float inv_s = 1.0f / (float)p.n_samples;
#pragma unroll
    for (int k = 0; k < kKReg; ++k) {
        if (k >= iso.K) break;
        const int64_t o = ((int64_t)(kbase + k) * Hc + cj) * Wc + ci;
        p.counts[o] = cnt[k];
        if (p.est) p.est[o] = (p.n_samples < (1ull << 24)) ? (float)cnt[k] / (float)p.n_samples : (float)((double)cnt[k] / (double)p.n_samples);
    }
    (void)inv_s;
}

}  // namespace
}  // namespace lcp

using namespace lcp;

extern "C" lcp_status lcp_mc(lcp_mc_mode mode, const float* mu_u, const float* var_u, const float* mu_v,
                             const float* var_v, const void* u, const void* v, lcp_dtype in_dtype, int M,
                             int64_t member_stride, int H, int W, double dx, double dy, const float* iso, int K,
                             int64_t n_samples, uint64_t seed, uint64_t offset, uint32_t* counts, float* lcp_out,
                             lcp_stream_t stream) {
    lcp_status s;
    if (mode == LCP_MC_GAUSS) {
        if (!mu_u || !var_u || !mu_v || !var_v) return fail(LCP_ERR_ARG, "lcp_mc: GAUSS mode needs the 4 statistics");
        if (H < 2 || W < 2) return fail(LCP_ERR_ARG, "lcp_mc: need H >= 2 and W >= 2");
    } else if (mode == LCP_MC_EMPIRICAL) {
        s = check_members("lcp_mc", u, v, in_dtype, M, H, W, member_stride, 0);
        if (s != LCP_OK) return s;
    } else {
        return fail(LCP_ERR_ARG, "lcp_mc: unknown mode %d", (int)mode);
    }
    if ((s = check_iso("lcp_mc", iso, K)) != LCP_OK) return s;
    if ((s = check_spacing("lcp_mc", dx, dy)) != LCP_OK) return s;
    if (!counts) return fail(LCP_ERR_ARG, "lcp_mc: counts is required");
    if (n_samples < 1 || n_samples > 0xFFFFFFFFll) return fail(LCP_ERR_ARG, "lcp_mc: need 1 <= n_samples < 2^32");
    if ((int64_t)H * W > (int64_t(1) << 32)) return fail(LCP_ERR_ARG, "lcp_mc: H*W must be <= 2^32");
    McParams p;
    p.mu_u = mu_u; p.var_u = var_u; p.mu_v = mu_v; p.var_v = var_v;
    p.u = u; p.v = v; p.M = M; p.stride = M > 1 ? member_stride : (int64_t)H * W;
    p.H = H; p.W = W; p.sp = make_spacing(dx, dy);
    p.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    p.off = make_uint2((uint32_t)offset, (uint32_t)(offset >> 32));
    p.n_samples = (uint64_t)n_samples;
    p.counts = counts;
    p.est = lcp_out;
    dim3 grid((W - 1 + kTX - 1) / kTX, (H - 1 + kTY - 1) / kTY);
    if (grid.y > 65535) return fail(LCP_ERR_UNSUPPORTED, "lcp_mc: grid too tall");
    cudaStream_t st = (cudaStream_t)stream;
    for (int kb = 0; kb < K; kb += kKReg) {
        IsoParams ip;
        ip.K = K - kb < kKReg ? K - kb : kKReg;
        for (int k = 0; k < ip.K; ++k) ip.c[k] = iso[kb + k];
        if (mode == LCP_MC_GAUSS)
            mc_kernel<LCP_MC_GAUSS, float><<<grid, kThreads, 0, st>>>(p, ip, kb);
        else if (in_dtype == LCP_F32)
            mc_kernel<LCP_MC_EMPIRICAL, float><<<grid, kThreads, 0, st>>>(p, ip, kb);
        else
            mc_kernel<LCP_MC_EMPIRICAL, __nv_bfloat16><<<grid, kThreads, 0, st>>>(p, ip, kb);
        if ((s = check_launch("lcp_mc")) != LCP_OK) return s;
    }
    return LCP_OK;
}
