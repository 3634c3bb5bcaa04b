// lcp_fused: ensemble statistics (Sec. 3.1), the divergence Gaussian (Eqs. 2,
// 3, one-sided at the boundary) and the level-crossing probability (Sec. 3.1,
// last paragraph) in one kernel that reads every member byte from HBM once.
//
// Decomposition.  A CTA owns a tile of cells: TW = 128 * VEC consecutive cell
// columns of a band of cell rows.  It marches the band row by row, keeping a
// rolling window of per-vertex statistics in shared memory (2 rows of u, 3 rows
// of v), so the vertical stencil never re-reads members inside the band.  The
// horizontal stencil needs u one column beyond each side: one extra column
// group per side, loaded by a small halo warp (those bytes are also read, at
// the same time, by the neighbouring tile, so L2 serves one of the two).
// Bands alternate marching direction (down / up), so the rows a band boundary
// shares are read by both neighbours at the same moment (start or end of the
// march) and the second read hits L2.  The grid is sized to one wave.
//
// Member reduction.  Each member row is reduced by `ms` thread groups
// ("member splits"), each summing a contiguous slice of members into shifted
// sums about member 0 (see stats.cu); the splits are combined in shared
// memory.  Splitting keeps many independent 16-byte loads in flight per SM
// without holding them all in one thread's registers.
//
// Cells.  After a vertex row's statistics are complete, every own thread forms
// the divergence Gaussian of its VEC + 1 vertices (its VEC columns plus the
// next one), then for each of its isovalues p = P(D < c), q = P(D >= c) and the
// horizontal products p_i p_{i+1}, q_i q_{i+1}; the previous vertex row's
// products (kept per thread in shared memory) close the cell:
//   LCP = 1 - (p00 p10)(p01 p11) - (q00 q10)(q01 q11).
// Isovalues are dealt round-robin to the member splits.
//
// Mean precision.  A vertex mean is kept as (x0, delta): member 0 plus the FP32
// mean of the shifted values.  Stencil differences take (x0_hi - x0_lo) +
// (delta_hi - delta_lo); the first term is exact whenever the two members are
// within a factor of 2 (Sterbenz), so large offsets (|mean| / sigma >> 1e3)
// cancel exactly instead of being rounded into the divergence.
#include <mutex>

#include "lcp_common.cuh"

namespace lcp {
namespace {

constexpr int kOwn = 128;      // own column groups = threads per member split
constexpr int kMaxKPass = 32;  // isovalues per launch (larger K runs in passes)

template <int VEC>
struct Geom {
    static constexpr int NR = VEC >= 2 ? 1 : 2;  // right halo groups (u at TW and TW + 1)
    static constexpr int NGRP = kOwn + 1 + NR;   // column groups held: left halo, own, right halo
    static constexpr int NCOL = NGRP * VEC;
    static constexpr int TW = kOwn * VEC;        // cell columns per tile
};

struct FusedParams {
    const void* u;
    const void* v;
    int64_t stride;
    int M, H, W, ddof;
    Spacing sp;
    void* out;
    uint32_t* mask;
    int n_words;
    int n_ty;   // bands
    int ms;     // member splits
    int kbase;  // index of this pass's first isovalue in the output
};

// shared-memory carve-up (all offsets in 4-byte words)
template <int VEC>
struct Smem {
    float* part;   // [ms][NGRP][4][VEC]  s1u s2u s1v s2v
    float* x0;     // [NGRP][2][VEC]      member-0 values of u, v
    float* ru;     // [3 planes][2 slots][NCOL]  x0, delta, var of u
    float* rv;     // [3 planes][3 slots][NCOL]  x0, delta, var of v
    float* pp;     // [kslots][ms][kOwn][VEC]    previous row p_i p_{i+1}
    float* pq;     // [kslots][ms][kOwn][VEC]    previous row q_i q_{i+1}
    uint32_t* pb;  // [kslots][ms][kOwn]         previous row mean-field bits
    static __host__ __device__ size_t words(int ms, int kslots) {
        using G = Geom<VEC>;
        return (size_t)4 * ms * G::NGRP * VEC + 2 * G::NGRP * VEC + 6 * G::NCOL + 9 * G::NCOL +
               (size_t)2 * kslots * ms * kOwn * VEC + (size_t)kslots * ms * kOwn;
    }
    __device__ Smem(float* base, int ms, int kslots) {
        using G = Geom<VEC>;
        part = base;
        x0 = part + 4 * ms * G::NGRP * VEC;
        ru = x0 + 2 * G::NGRP * VEC;
        rv = ru + 6 * G::NCOL;
        pp = rv + 9 * G::NCOL;
        pq = pp + (size_t)kslots * ms * kOwn * VEC;
        pb = reinterpret_cast<uint32_t*>(pq + (size_t)kslots * ms * kOwn * VEC);
    }
};

// Shifted sums of one column group over members [m_lo, m_hi) of one row.
template <typename T, int VEC, bool DO_U, bool DO_V>
__device__ __forceinline__ void reduce_members(const T* __restrict__ u, const T* __restrict__ v, int64_t stride,
                                               int64_t off, int m_lo, int m_hi, const float* x0u, const float* x0v,
                                               float* s1u, float* s2u, float* s1v, float* s2v) {
    using L = Loader<T, VEC>;
    constexpr int UNROLL = VEC >= 8 ? ((DO_U && DO_V) ? 2 : 4) : ((DO_U && DO_V) ? 4 : 8);
    auto acc = [&](const typename L::raw_t& r, const float* x0, float* s1, float* s2) {
        float a[VEC];
        L::cvt(r, a);
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const float d = a[e] - x0[e];
            s1[e] += d;
            s2[e] = fmaf(d, d, s2[e]);
        }
    };
    int m = m_lo;
    for (; m + UNROLL <= m_hi; m += UNROLL) {
        typename L::raw_t ru[UNROLL], rv[UNROLL];
#pragma unroll
        for (int q = 0; q < UNROLL; ++q) {
            if (DO_U) ru[q] = L::load(u + (int64_t)(m + q) * stride + off);
            if (DO_V) rv[q] = L::load(v + (int64_t)(m + q) * stride + off);
        }
#pragma unroll
        for (int q = 0; q < UNROLL; ++q) {
            if (DO_U) acc(ru[q], x0u, s1u, s2u);
            if (DO_V) acc(rv[q], x0v, s1v, s2v);
        }
    }
    for (; m < m_hi; ++m) {
        if (DO_U) acc(L::load(u + (int64_t)m * stride + off), x0u, s1u, s2u);
        if (DO_V) acc(L::load(v + (int64_t)m * stride + off), x0v, s1v, s2v);
    }
}

template <typename T, int VEC, typename OutT, int MS>
__global__ void __launch_bounds__(kOwn * MS + 32, MS >= 4 ? 1 : 2)
    fused_kernel(const __grid_constant__ FusedParams p, const __grid_constant__ IsoParams iso) {
    using G = Geom<VEC>;
    using L = Loader<T, VEC>;
    extern __shared__ __align__(16) float smem_raw[];
    constexpr int ms = MS;
    const int K = iso.K;
    const int kslots = (K + ms - 1) / ms;
    Smem<VEC> sm(smem_raw, ms, kslots);

    const int H = p.H, W = p.W, M = p.M, Hc = H - 1, Wc = W - 1;
    const T* __restrict__ u = reinterpret_cast<const T*>(p.u);
    const T* __restrict__ v = reinterpret_cast<const T*>(p.v);
    const int tid = threadIdx.x, lane = tid & 31;
    const int n_own_threads = kOwn * ms;

    // tile
    const int c0 = blockIdx.x * G::TW;
    const int ty = blockIdx.y;
    const int r0 = (int)(((int64_t)ty * Hc) / p.n_ty);
    const int r1 = (int)(((int64_t)(ty + 1) * Hc) / p.n_ty);  // cells [r0, r1), vertex rows [r0, r1]
    const bool down = (ty & 1) == 0;
    const int jfirst = down ? max(r0 - 1, 0) : min(r1 + 1, H - 1);
    const int jlast = down ? min(r1 + 1, H - 1) : max(r0 - 1, 0);
    const int nsteps = (down ? jlast - jfirst : jfirst - jlast) + 1;

    // this thread's load assignment: member split s, column group lg (local index)
    int s = -1, lg = -1;
    if (tid < n_own_threads) {
        s = tid / kOwn;
        lg = tid % kOwn + 1;
    } else {
        const int hl = tid - n_own_threads;
        if (hl < ms * (1 + G::NR)) {
            s = hl / (1 + G::NR);
            const int h = hl % (1 + G::NR);
            lg = h == 0 ? 0 : kOwn + h;
        }
    }
    const int gcol = c0 - VEC + lg * VEC;
    const bool colok = lg >= 0 && gcol >= 0 && gcol < W;
    const int m_lo = s <= 0 ? 1 : (int)((int64_t)s * M / ms);
    const int m_hi = s < 0 ? 0 : (int)((int64_t)(s + 1) * M / ms);
    const float fm = (float)M, fdof = (float)(M - p.ddof);

    bool have_prev = false;
    for (int step = 0; step < nsteps; ++step) {
        const int j = down ? jfirst + step : jfirst - step;
        const bool needU = j >= r0 && j <= r1;
        // ---- 1) member reduction of row j --------------------------------
        if (lg >= 0) {
            float x0u[VEC], x0v[VEC], s1u[VEC], s2u[VEC], s1v[VEC], s2v[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) x0u[e] = x0v[e] = s1u[e] = s2u[e] = s1v[e] = s2v[e] = 0.f;
            const bool needV = lg != 0;  // the left halo column group only feeds u
            if (colok) {
                const int64_t off = (int64_t)j * W + gcol;
                if (needU) L::cvt(L::load(u + off), x0u);
                if (needV) L::cvt(L::load(v + off), x0v);
                if (needU && needV)
                    reduce_members<T, VEC, true, true>(u, v, p.stride, off, m_lo, m_hi, x0u, x0v, s1u, s2u, s1v, s2v);
                else if (needU)
                    reduce_members<T, VEC, true, false>(u, v, p.stride, off, m_lo, m_hi, x0u, x0v, s1u, s2u, s1v, s2v);
                else if (needV)
                    reduce_members<T, VEC, false, true>(u, v, p.stride, off, m_lo, m_hi, x0u, x0v, s1u, s2u, s1v, s2v);
            }
            float* pt = sm.part + ((size_t)s * G::NGRP + lg) * 4 * VEC;
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                pt[e] = s1u[e];
                pt[VEC + e] = s2u[e];
                pt[2 * VEC + e] = s1v[e];
                pt[3 * VEC + e] = s2v[e];
            }
            if (s == 0) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    sm.x0[lg * 2 * VEC + e] = x0u[e];
                    sm.x0[lg * 2 * VEC + VEC + e] = x0v[e];
                }
            }
        }
        __syncthreads();
        // ---- 2) combine the member splits into (x0, delta, var) rings -------
        if (s == 0) {
            const int su = j & 1, sv = j % 3;
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                float a1 = 0.f, a2 = 0.f, b1 = 0.f, b2 = 0.f;
                for (int q = 0; q < ms; ++q) {
                    const float* pt = sm.part + ((size_t)q * G::NGRP + lg) * 4 * VEC;
                    a1 += pt[e];
                    a2 += pt[VEC + e];
                    b1 += pt[2 * VEC + e];
                    b2 += pt[3 * VEC + e];
                }
                const int col = lg * VEC + e;
                const float du = a1 / fm, dv = b1 / fm;
                float vu = (a2 - a1 * du) / fdof, vv = (b2 - b1 * dv) / fdof;
                if (vu < 0.f) vu = 0.f;
                if (vv < 0.f) vv = 0.f;
                if (needU) {
                    sm.ru[(0 * 2 + su) * G::NCOL + col] = sm.x0[lg * 2 * VEC + e];
                    sm.ru[(1 * 2 + su) * G::NCOL + col] = du;
                    sm.ru[(2 * 2 + su) * G::NCOL + col] = vu;
                }
                sm.rv[(0 * 3 + sv) * G::NCOL + col] = sm.x0[lg * 2 * VEC + VEC + e];
                sm.rv[(1 * 3 + sv) * G::NCOL + col] = dv;
                sm.rv[(2 * 3 + sv) * G::NCOL + col] = vv;
            }
        }
        __syncthreads();
        // ---- 3) divergence rows completed by row j, then their cells --------
        for (int pass = 0; pass < 2; ++pass) {
            int d;
            if (down) {
                d = pass == 0 ? j - 1 : j;
                if (pass == 1 && j != H - 1) continue;
            } else {
                d = pass == 0 ? j + 1 : j;
                if (pass == 1 && j != 0) continue;
            }
            if (d < r0 || d > r1) continue;
            if (tid < n_own_threads) {
                const int g = tid % kOwn;
                const int su = d & 1;
                const int jlo = d > 0 ? d - 1 : 0, jhi = d < H - 1 ? d + 1 : H - 1;
                const float sy = (jhi - jlo == 2) ? p.sp.sy2 : p.sp.sy1;
                const float syq = (jhi - jlo == 2) ? p.sp.sy2q : p.sp.sy1q;
                const int vlo = jlo % 3, vhi = jhi % 3;
                float mu[VEC + 1], var[VEC + 1];
#pragma unroll
                for (int e = 0; e <= VEC; ++e) {
                    const int ic = min(c0 + g * VEC + e, W - 1);
                    const int ilo = ic > 0 ? ic - 1 : 0, ihi = ic < W - 1 ? ic + 1 : W - 1;
                    const float sx = (ihi - ilo == 2) ? p.sp.sx2 : p.sp.sx1;
                    const float sxq = (ihi - ilo == 2) ? p.sp.sx2q : p.sp.sx1q;
                    const int lcl = ilo - c0 + VEC, lch = ihi - c0 + VEC, lc = ic - c0 + VEC;
                    const float* rx0 = sm.ru + (0 * 2 + su) * G::NCOL;
                    const float* rdl = sm.ru + (1 * 2 + su) * G::NCOL;
                    const float* rvr = sm.ru + (2 * 2 + su) * G::NCOL;
                    const float du = (rx0[lch] - rx0[lcl]) + (rdl[lch] - rdl[lcl]);
                    const float dv = (sm.rv[(0 * 3 + vhi) * G::NCOL + lc] - sm.rv[(0 * 3 + vlo) * G::NCOL + lc]) +
                                     (sm.rv[(1 * 3 + vhi) * G::NCOL + lc] - sm.rv[(1 * 3 + vlo) * G::NCOL + lc]);
                    const float vu = rvr[lch] + rvr[lcl];
                    const float vv = sm.rv[(2 * 3 + vhi) * G::NCOL + lc] + sm.rv[(2 * 3 + vlo) * G::NCOL + lc];
                    mu[e] = fmaf(du, sx, dv * sy);
                    var[e] = fmaf(vu, sxq, vv * syq);
                }
                const int cr = down ? d - 1 : d;  // cell row closed by this divergence row
                const int cbase = c0 + g * VEC;
                for (int t = 0, k = s; k < K; ++t, k += ms) {
                    const float c = iso.c[k];
                    float pr[VEC + 1], qr[VEC + 1];
                    uint32_t bits = 0;
#pragma unroll
                    for (int e = 0; e <= VEC; ++e) {
                        below_above(mu[e], var[e], c, pr[e], qr[e]);
                        bits |= (uint32_t)(mu[e] < c) << e;
                    }
                    float ph[VEC], qh[VEC];
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        ph[e] = pr[e] * pr[e + 1];
                        qh[e] = qr[e] * qr[e + 1];
                    }
                    const size_t slot = ((size_t)t * ms + s) * kOwn + g;
                    float* PP = sm.pp + slot * VEC;
                    float* PQ = sm.pq + slot * VEC;
                    if (have_prev) {
                        const uint32_t bp = sm.pb[slot];
                        const int64_t obase = ((int64_t)(p.kbase + k) * Hc + cr) * Wc;
                        OutT* out = reinterpret_cast<OutT*>(p.out);
                        uint32_t nib = 0;
#pragma unroll
                        for (int e = 0; e < VEC; ++e) {
                            const int col = cbase + e;
                            if (col < Wc) {
                                const float lcp = 1.0f - PP[e] * ph[e] - PQ[e] * qh[e];
                                out[obase + col] = to_out<OutT>(clamp01(lcp));
                                const uint32_t four = ((bp >> e) & 3u) | (((bits >> e) & 3u) << 2);
                                nib |= (uint32_t)(four != 0u && four != 15u) << e;
                            }
                        }
                        if (p.mask) {
                            constexpr int LPW = 32 / VEC;  // lanes per mask word
                            uint32_t val = nib << (VEC * (lane % LPW));
#pragma unroll
                            for (int o = 1; o < LPW; o <<= 1) val |= __shfl_xor_sync(0xFFFFFFFFu, val, o);
                            const int word = cbase >> 5;
                            if (lane % LPW == 0 && word < p.n_words)
                                p.mask[((int64_t)(p.kbase + k) * Hc + cr) * p.n_words + word] = val;
                        }
                    }
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        PP[e] = ph[e];
                        PQ[e] = qh[e];
                    }
                    sm.pb[slot] = bits;
                }
            }
            have_prev = true;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T, int VEC, typename OutT, int MS>
lcp_status launch_fused_ms(FusedParams p, const float* iso, int K, cudaStream_t st) {
    using G = Geom<VEC>;
    auto kern = fused_kernel<T, VEC, OutT, MS>;
    p.ms = MS;
    const int Hc = p.H - 1, Wc = p.W - 1;
    const int n_tx = (Wc + G::TW - 1) / G::TW;
    const int threads = kOwn * p.ms + 32;
    const int kmax_pass = K < kMaxKPass ? K : kMaxKPass;
    const int kslots = (kmax_pass + p.ms - 1) / p.ms;
    const size_t smem = Smem<VEC>::words(p.ms, kslots) * 4;
    {
        static std::mutex mu;
        static size_t set_bytes[64] = {0};
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && set_bytes[dev] < smem) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return fail(LCP_ERR_CUDA, "lcp_fused: %zu bytes of shared memory not available", smem);
            set_bytes[dev] = smem;
        }
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
        return fail(LCP_ERR_CUDA, "lcp_fused: kernel does not fit on an SM (smem %zu)", smem);
    const long slots = (long)per_sm * num_sms();
    long n_ty = slots / n_tx;
    if (n_ty < 1) n_ty = 1;
    if (n_ty > Hc) n_ty = Hc;
    if (n_ty > 65535) n_ty = 65535;
    p.n_ty = (int)n_ty;
    dim3 grid(n_tx, (unsigned)n_ty);
    for (int kb = 0; kb < K; kb += kMaxKPass) {
        IsoParams ip;
        ip.K = K - kb < kMaxKPass ? K - kb : kMaxKPass;
        for (int k = 0; k < ip.K; ++k) ip.c[k] = iso[kb + k];
        p.kbase = kb;
        kern<<<grid, threads, smem, st>>>(p, ip);
        lcp_status s = check_launch("lcp_fused");
        if (s != LCP_OK) return s;
    }
    return LCP_OK;
}

// Member splits: 1, 2 or 4 groups of 128 threads reduce disjoint member slices.
// Instantiated: fp32 x4 with 1, 2 or 4 splits; bf16 x8 with 1 split (its
// 8-wide accumulators need the register budget of 2 CTAs of 160 threads);
// the scalar fallbacks with 2 splits.
template <typename T, int VEC, typename OutT>
lcp_status launch_fused(FusedParams p, const float* iso, int K, cudaStream_t st) {
    if constexpr (VEC == 4) {
        if (p.ms >= 4) return launch_fused_ms<T, VEC, OutT, 4>(p, iso, K, st);
        if (p.ms == 2) return launch_fused_ms<T, VEC, OutT, 2>(p, iso, K, st);
        return launch_fused_ms<T, VEC, OutT, 1>(p, iso, K, st);
    } else if constexpr (VEC == 8) {
        return launch_fused_ms<T, VEC, OutT, 1>(p, iso, K, st);
    } else {
        return launch_fused_ms<T, VEC, OutT, 2>(p, iso, K, st);
    }
}

int choose_member_splits(int M) {
    static int env = -1;
    if (env < 0) {
        const char* e = getenv("LCP_FUSED_MS");
        env = e ? atoi(e) : 0;
    }
    if (env == 1 || env == 2 || env == 4) return env;
    if (M >= 16) return 2;
    return 1;
}

}  // namespace
}  // namespace lcp

using namespace lcp;

extern "C" lcp_status lcp_fused(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                                int64_t member_stride, int ddof, double dx, double dy, const float* iso, int K,
                                void* lcp_out, lcp_dtype out_dtype, uint32_t* mask, lcp_stream_t stream) {
    lcp_status s = check_members("lcp_fused", u, v, in_dtype, M, H, W, member_stride, ddof);
    if (s != LCP_OK) return s;
    if ((s = check_iso("lcp_fused", iso, K)) != LCP_OK) return s;
    if ((s = check_spacing("lcp_fused", dx, dy)) != LCP_OK) return s;
    if (!lcp_out) return fail(LCP_ERR_ARG, "lcp_fused: NULL output");
    if (out_dtype != LCP_F32 && out_dtype != LCP_F16) return fail(LCP_ERR_ARG, "lcp_fused: out dtype must be F32 or F16");
    if ((uintptr_t)mask & 3) return fail(LCP_ERR_ARG, "lcp_fused: mask must be 4-byte aligned");
    FusedParams p;
    p.u = u;
    p.v = v;
    p.M = M;
    p.H = H;
    p.W = W;
    p.ddof = ddof;
    p.stride = M > 1 ? member_stride : (int64_t)H * W;
    p.sp = make_spacing(dx, dy);
    p.out = lcp_out;
    p.mask = mask;
    p.n_words = (W - 1 + 31) / 32;
    p.ms = choose_member_splits(M);
    if (p.ms > M) p.ms = 1;
    p.kbase = 0;
    p.n_ty = 1;
    cudaStream_t st = (cudaStream_t)stream;
    // The TMA row-march is opt-in (LCP_FUSED_TMA=1): on GB300 it measures a few
    // percent slower than register streaming at K = 8 and more at K >= 16.
    static const bool tma_enabled = [] {
        const char* e = getenv("LCP_FUSED_TMA");
        return e && e[0] == '1';
    }();
    if (tma_enabled) {
        s = fused_tma(u, v, in_dtype, M, H, W, p.stride, ddof, dx, dy, iso, K, lcp_out, out_dtype, mask, st);
        if (s != LCP_ERR_UNSUPPORTED) return s;
    }
    const bool in16 = aligned16(u) && aligned16(v);
    const bool f16 = out_dtype == LCP_F16;
    if (in_dtype == LCP_F32) {
        const bool vec = in16 && W % 4 == 0 && p.stride % 4 == 0;
        if (vec) return f16 ? launch_fused<float, 4, __half>(p, iso, K, st) : launch_fused<float, 4, float>(p, iso, K, st);
        return f16 ? launch_fused<float, 1, __half>(p, iso, K, st) : launch_fused<float, 1, float>(p, iso, K, st);
    }
    const bool vec = in16 && W % 8 == 0 && p.stride % 8 == 0;
    if (vec)
        return f16 ? launch_fused<__nv_bfloat16, 8, __half>(p, iso, K, st)
                   : launch_fused<__nv_bfloat16, 8, float>(p, iso, K, st);
    return f16 ? launch_fused<__nv_bfloat16, 1, __half>(p, iso, K, st)
               : launch_fused<__nv_bfloat16, 1, float>(p, iso, K, st);
}
