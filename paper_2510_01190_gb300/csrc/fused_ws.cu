// lcp_fused_ws: the closed-form path in two kernels that share an L2-resident
// workspace (statistics, Sec. 3.1; Eqs. 2/3 with the one-sided boundary rule;
// the LCP of every cell, Sec. 3.1 last paragraph).
//
// 1) stats_ws_kernel: a flat, fully coalesced stream over the member planes --
//    each thread owns VEC consecutive vertices of a chunk and keeps 16
//    independent loads in flight, the access pattern that runs near HBM peak.
//    Per vertex and component it stores one 16-byte record (x0, delta, var, 0):
//    member 0, the FP32 mean of the values shifted by member 0, and the
//    variance.  Member loads carry an L2 evict-first policy and the record
//    stores evict-last, so the 32 bytes per vertex stay in the 129 MB L2.  The
//    same pass clears the mean-field mask rows of its chunk.
// 2) LCP from the records.  Up to 8 isovalues: lcp_warp_rows_kernel, where every
//    warp marches down 8 cell rows of a 31-cell strip with a sliding register
//    window (own u record, horizontal neighbours by warp shuffle; v records of
//    rows j-1, j, j+1), the next row always in flight; each lane forms its
//    vertex's divergence Gaussian and its (P(D<c), P(D>=c)) per isovalue, takes
//    its right neighbour's by shuffle, closes its cell with the previous row's
//    products, and the warp ORs the mean-field crossing bits into the mask
//    words.  More isovalues: lcp_rows_kernel, a 256-column tile that shares a
//    row's vertex values through shared memory (passes of up to 32).  Both are
//    compiled for exact isovalue counts, so the isovalue loop has no guards.
//
// Overlap.  The statistics grid triggers its programmatic dependents as each
// block starts and, after storing a chunk, counts it into per-row-band counters
// in the workspace (fence, then atomic add).  The LCP grid, launched as its
// programmatic dependent, therefore starts as soon as every statistics block
// is resident, and each LCP block waits -- bounded, with backoff -- only for
// the statistics rows of its own band.  The wait cannot deadlock: every block
// it waits for is already running.
//
// Grids whose records would not fit comfortably in L2 (a 96 MB budget) are
// processed in bands of rows (records of the band plus one halo row on each
// side, then its cells), so the workspace never spills to HBM; a smaller
// workspace than lcp_fused_workspace_bytes reports gives smaller bands.  With
// several bands the statistics grid is persistent (3 blocks per SM for fp32
// members, 2 for bf16), so that the LCP grid runs beside each band's stream
// rather than after it.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <mutex>
#include <type_traits>

#include "lcp_common.cuh"

namespace lcp {

__device__ unsigned int g_ws_status;  // bit 0: an LCP block's dependency wait gave up

namespace {

constexpr int kST = 256;           // stats kernel threads
constexpr int kRT = 256;           // LCP kernel threads = cell columns per tile
constexpr int kTR = 8;             // cell rows per LCP tile
constexpr int kMaxKPass = 32;      // isovalues per LCP launch
constexpr size_t kL2Budget = 96ull << 20;  // workspace bytes a band may occupy (of the 129 MB L2)

// Statistics blocks [blo, bhi] of the statistics grid that cover the rows LCP
// row band `by` needs (its vertex rows and one halo row each side).  The same
// function decides what a statistics block signals and what an LCP block waits
// for, so the two sides agree by construction.
__device__ __forceinline__ void band_blocks(int64_t n_begin, int sv, int W, int H, int r_begin, int r_end, int by,
                                            int& blo, int& bhi) {
    const int a = r_begin + by * kTR, e = min(a + kTR, r_end);
    const int lo = max(a - 1, 0), hi = min(e + 1, H - 1);
    blo = (int)(((int64_t)lo * W - n_begin) / sv);
    bhi = (int)((((int64_t)hi + 1) * W - 1 - n_begin) / sv);
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ---- cache-policy loads / stores ------------------------------------------
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float4 ld_stream_f4(const float* p, uint64_t pol) {
    float4 r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint4 ld_stream_u4(const void* p, uint64_t pol) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ void st_keep_f4(float* p, float4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w), "l"(pol)
                 : "memory");
}

template <typename T, int VEC>
struct SLoad;
template <>
struct SLoad<float, 4> {
    using raw_t = float4;
    static __device__ __forceinline__ raw_t load(const float* p, uint64_t pol) { return ld_stream_f4(p, pol); }
    static __device__ __forceinline__ void cvt(const raw_t& r, float* x) { x[0] = r.x; x[1] = r.y; x[2] = r.z; x[3] = r.w; }
};
__device__ __forceinline__ uint2 ld_stream_u2(const void* p, uint64_t pol) {
    uint2 r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
                 : "=r"(r.x), "=r"(r.y)
                 : "l"(p), "l"(pol));
    return r;
}
template <>
struct SLoad<__nv_bfloat16, 4> {
    using raw_t = uint2;
    static __device__ __forceinline__ raw_t load(const __nv_bfloat16* p, uint64_t pol) { return ld_stream_u2(p, pol); }
    static __device__ __forceinline__ void cvt(const raw_t& r, float* x) {
        x[0] = __uint_as_float(r.x << 16);
        x[1] = __uint_as_float(r.x & 0xFFFF0000u);
        x[2] = __uint_as_float(r.y << 16);
        x[3] = __uint_as_float(r.y & 0xFFFF0000u);
    }
};
template <typename T>
__device__ __forceinline__ float load1(const T* p) {
    float x;
    Loader<T, 1>::cvt(Loader<T, 1>::load(p), &x);
    return x;
}

// ---- 1) statistics stream ----------------------------------------------------
// Workspace record of one vertex and component: float4 (x0, delta, var, 0) --
// member 0, FP32 mean of the values shifted by member 0, variance -- so that
// the LCP kernel reads a vertex's component with one 16-byte load.  Two
// record planes (u, v) of `ws_rows` rows x W vertices.
struct StatsWsParams {
    const void* u;
    const void* v;
    int64_t stride;
    int M, W, ddof;
    int64_t n_begin, n_end;  // flat vertex range [n_begin, n_end) of this band (member-plane index)
    int row0;                // first row of the band (workspace row 0)
    float4* st;              // record planes: u at st, v at st + ps
    int64_t ps;              // plane stride in records
    int vecload;
    uint32_t* dep;           // per LCP row band: statistics chunks completed
    int H, r_begin, r_end, nby;
    uint32_t* mzero;         // mask whose cell rows [r_begin, r_end) this pass clears (null: none)
    int mK, mwords;          // its planes and words per row
    int64_t mplane;          // words per plane
};

__device__ __forceinline__ void store_stats(const StatsWsParams& p, int64_t n, const float* x0, const float* s1,
                                            const float* s2, int comp, uint64_t keep, int cnt) {
    const float fm = (float)p.M, fdof = (float)(p.M - p.ddof);
    // records are flat-indexed from the band's first row: (j - row0) * W + i = n - row0 * W
    float4* base = p.st + comp * p.ps + (n - (int64_t)p.row0 * p.W);
    for (int e = 0; e < cnt; ++e) {
        const float dl = s1[e] / fm;
        float vv = (s2[e] - s1[e] * dl) / fdof;
        vv = vv < 0.f ? 0.f : vv;  // NaN stays NaN
        st_keep_f4(reinterpret_cast<float*>(base + e), make_float4(x0[e], dl, vv, 0.f), keep);
    }
}

// bf16 members (8-byte loads) take up to 80 registers a thread: 10 members per batch, so
// that a 20-member ensemble streams in two round trips per chunk instead of three.
template <typename T>
struct StatsTune {
    static constexpr int kMinBlocks = sizeof(T) == 2 ? 3 : 4;  // resident blocks per SM the registers allow
    static constexpr int kBatch8 = 10;                          // members per batch of 8-byte loads
    static constexpr int kPersist = sizeof(T) == 2 ? 2 : 3;     // persistent blocks per SM (several bands)
};

template <typename T, int VEC>
__global__ void __launch_bounds__(kST, StatsTune<T>::kMinBlocks) stats_ws_kernel(const __grid_constant__ StatsWsParams p) {
    const T* __restrict__ u = reinterpret_cast<const T*>(p.u);
    const T* __restrict__ v = reinterpret_cast<const T*>(p.v);
    const uint64_t pol = policy_evict_first();
    const uint64_t keep = policy_evict_last();
    // Every block of this grid is resident once all have executed this: the
    // dependent LCP grid may then launch and wait on the per-band counters.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int M = p.M;
    constexpr int sv = kST * VEC;  // vertices per chunk
    const int64_t nchunks = (p.n_end - p.n_begin + sv - 1) / sv;
    for (int64_t blk = blockIdx.x; blk < nchunks; blk += gridDim.x) {  // chunks in vertex order
    const int64_t n0 = p.n_begin + (blk * kST + threadIdx.x) * VEC;
    if (n0 < p.n_end) {
        if (p.vecload && n0 + VEC <= p.n_end) {
            using L = SLoad<T, VEC>;
            float x0u[VEC], x0v[VEC], s1u[VEC], s2u[VEC], s1v[VEC], s2v[VEC];
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
            // 16-byte loads: 8 members (16 loads) per batch; 8-byte loads: StatsTune's batch
            constexpr int UNROLL = sizeof(typename L::raw_t) < 16 ? StatsTune<T>::kBatch8 : 8;
            int m = 1;
            if (sizeof(typename L::raw_t) < 16 && M >= UNROLL) {
                // 8-byte loads: member 0 (the shift) travels with members 1 .. UNROLL-1, one round
                // trip fewer per chunk (measured: 8192^2 bf16 K = 4, 2.545 -> 2.500 ms; with 16-byte
                // loads the extra registers spill and cost more than the round trip)
                typename L::raw_t ru[UNROLL], rv[UNROLL];
#pragma unroll
                for (int q = 0; q < UNROLL; ++q) {
                    ru[q] = L::load(u + (int64_t)q * p.stride + n0, pol);
                    rv[q] = L::load(v + (int64_t)q * p.stride + n0, pol);
                }
                L::cvt(ru[0], x0u);
                L::cvt(rv[0], x0v);
#pragma unroll
                for (int q = 1; q < UNROLL; ++q) acc(ru[q], rv[q]);
                m = UNROLL;
            } else {
                L::cvt(L::load(u + n0, pol), x0u);
                L::cvt(L::load(v + n0, pol), x0v);
            }
            for (; m + UNROLL <= M; m += UNROLL) {
                typename L::raw_t ru[UNROLL], rv[UNROLL];
#pragma unroll
                for (int q = 0; q < UNROLL; ++q) {
                    ru[q] = L::load(u + (int64_t)(m + q) * p.stride + n0, pol);
                    rv[q] = L::load(v + (int64_t)(m + q) * p.stride + n0, pol);
                }
#pragma unroll
                for (int q = 0; q < UNROLL; ++q) acc(ru[q], rv[q]);
            }
            if (sizeof(typename L::raw_t) < 16 && m < M) {  // 8-byte loads: the remaining members as one batch
                typename L::raw_t ru[UNROLL], rv[UNROLL];
#pragma unroll
                for (int q = 0; q < UNROLL; ++q)
                    if (m + q < M) {
                        ru[q] = L::load(u + (int64_t)(m + q) * p.stride + n0, pol);
                        rv[q] = L::load(v + (int64_t)(m + q) * p.stride + n0, pol);
                    }
#pragma unroll
                for (int q = 0; q < UNROLL; ++q)
                    if (m + q < M) acc(ru[q], rv[q]);
                m = M;
            }
            for (; m < M; ++m) acc(L::load(u + (int64_t)m * p.stride + n0, pol), L::load(v + (int64_t)m * p.stride + n0, pol));
            store_stats(p, n0, x0u, s1u, s2u, 0, keep, VEC);
            store_stats(p, n0, x0v, s1v, s2v, 1, keep, VEC);
        } else {
            const int64_t n_end = min(n0 + VEC, p.n_end);
            for (int64_t n = n0; n < n_end; ++n) {
                float x0u = load1(u + n), x0v = load1(v + n);
                float a1 = 0.f, a2 = 0.f, b1 = 0.f, b2 = 0.f;
                for (int m = 1; m < M; ++m) {
                    const float du = load1(u + (int64_t)m * p.stride + n) - x0u;
                    const float dv = load1(v + (int64_t)m * p.stride + n) - x0v;
                    a1 += du;
                    a2 = fmaf(du, du, a2);
                    b1 += dv;
                    b2 = fmaf(dv, dv, b2);
                }
                store_stats(p, n, &x0u, &a1, &a2, 0, keep, 1);
                store_stats(p, n, &x0v, &b1, &b2, 1, keep, 1);
            }
        }
    }
    const int64_t f0 = p.n_begin + blk * sv;  // this chunk's vertices [f0, f1]
    const int64_t f1 = min(f0 + sv, p.n_end) - 1;
    if (p.mzero) {  // clear the mask words of every cell row of this band whose first vertex is in the chunk
        for (int64_t j = (f0 + p.W - 1) / p.W; j * p.W <= f1; ++j) {
            if (j < p.r_begin || j >= p.r_end) continue;
            for (int x = threadIdx.x; x < p.mK * p.mwords; x += kST) {
                const int k = x / p.mwords, w = x - k * p.mwords;
                p.mzero[(int64_t)k * p.mplane + j * p.mwords + w] = 0u;
            }
        }
    }
    // publish: this chunk's statistics (and mask rows) are stored; count it for
    // every LCP row band whose rows it covers
    __syncthreads();
    if (threadIdx.x == 0 && p.dep) {
        __threadfence();
        const int rs0 = (int)(f0 / p.W), rs1 = (int)(f1 / p.W);
        const int lo = max(0, (rs0 - 1 - p.r_begin) / kTR - 1), hi = min(p.nby - 1, (rs1 + 1 - p.r_begin) / kTR + 1);
        for (int by = lo; by <= hi; ++by) {
            int blo, bhi;
            band_blocks(p.n_begin, sv, p.W, p.H, p.r_begin, p.r_end, by, blo, bhi);
            if ((int)blk >= blo && (int)blk <= bhi) atomicAdd(&p.dep[by], 1u);
        }
    }
    }
}

// ---- 2) divergence + LCP from the workspace -----------------------------------
struct RowsParams {
    const float4* st;  // record planes (u at st, v at st + ps); record row 0 = grid row `row0`
    int64_t ps;
    int row0;
    int H, W;            // full grid
    int r_begin, r_end;  // cell rows [r_begin, r_end) of this band (grid coordinates)
    Spacing sp;
    void* out;
    uint32_t* mask;
    int n_words;
    int kbase;            // index of this pass's first isovalue in the output
    const uint32_t* dep;  // per row band: statistics blocks completed
    int64_t n_begin;      // statistics grid geometry, to recompute each band's requirement
    int sv;
    long long budget;     // clock cycles before a dependency wait gives up
    double dsx2, dsx1, dsy2, dsy1;  // the stencil factors in FP64 (flagged vertices, below)
};

inline void set_spacing(RowsParams& rp, double dx, double dy) {
    rp.sp = make_spacing(dx, dy);
    rp.dsx2 = 0.5 / dx;
    rp.dsx1 = 1.0 / dx;
    rp.dsy2 = 0.5 / dy;
    rp.dsy1 = 1.0 / dy;
}

// The divergence mean of a vertex as an unevaluated pair (mu, lo).  The fp32
// stencil rounds the difference of the member-0 values x0 across it with an
// error up to 2^-24 of that difference (exact when the two are within a factor
// of 2), and mu itself keeps 24 bits: both are negligible unless the
// difference is large against sigma, as when a mean of large magnitude
// changes sign across the stencil.  Where A = |dx0_u| sx + |dx0_v| sy exceeds
// 16 sigma (A^2 > 256 var, or any A > 0 at zero variance), the mean is formed
// again in FP64 -- the fp32 x0 and delta differences are exact there -- and
// split into mu + lo; elsewhere lo = 0 and mu is the fp32 value, unchanged.
// With A <= 16 sigma the fp32 stencil moves a z-score by at most ~3 2^-24 16,
// about 3e-6, and the LCP by about 1e-5 in the worst alignment.  Warp-uniform
// (every lane of the warp must call it); the FP64 branch runs only in warps
// with a flagged lane.
// |dx0_u| sx + |dx0_v| sy above kExactZ / (sigma sqrt 2), i.e. above 16 sigma, takes the FP64 stencil.
constexpr float kExactZ = 11.3137085f;  // 16 / sqrt(2)
__device__ __forceinline__ bool mu_needs_fp64(float var, const float4& L, const float4& R, const float4& Vlo,
                                              const float4& Vhi, float sx, float sy) {
    const float A = fmaf(fabsf(R.x - L.x), sx, fabsf(Vhi.x - Vlo.x) * sy);
    return A * A > 256.0f * var;
}
__device__ __forceinline__ float mu_fp64(float& mu, const float4& L, const float4& R, const float4& Vlo,
                                         const float4& Vhi, double dsx, double dsy) {
    const double m = (((double)R.x - (double)L.x) + ((double)R.y - (double)L.y)) * dsx +
                     (((double)Vhi.x - (double)Vlo.x) + ((double)Vhi.y - (double)Vlo.y)) * dsy;
    mu = (float)m;
    return (float)(m - (double)mu);
}
__device__ __forceinline__ float exact_mu(float& mu, float var, const float4& L, const float4& R, const float4& Vlo,
                                          const float4& Vhi, float sx, float sy, double dsx, double dsy) {
    const bool big = mu_needs_fp64(var, L, R, Vlo, Vhi, sx, sy);
    float lo = 0.0f;
    if (__any_sync(0xFFFFFFFFu, big) && big) lo = mu_fp64(mu, L, R, Vlo, Vhi, dsx, dsy);
    return lo;
}

// Bounded wait (thread 0 of the block) until the statistics rows of LCP row
// band `by` are complete; every thread returns whether the wait gave up.
__device__ __forceinline__ bool wait_band(const RowsParams& p, int by) {
    int gave_up = 0;
    if (threadIdx.x == 0) {
        int blo, bhi;
        band_blocks(p.n_begin, p.sv, p.W, p.H, p.r_begin, p.r_end, by, blo, bhi);
        const uint32_t need = (uint32_t)(bhi - blo + 1);
        const long long t0 = clock64();
        while (ld_acquire(&p.dep[by]) < need) {
            if (clock64() - t0 > p.budget) {
                atomicOr(&g_ws_status, 1u);
                gave_up = 1;
                break;
            }
            __nanosleep(200);
        }
    }
    return __syncthreads_or(gave_up) != 0;
}

// After a wait that gave up, the band's records may be incomplete: this
// thread's cell column gets NaN for every cell row [a, e) and isovalue of the
// pass, and the mask word owner clears its words, so that no finite value is
// ever computed from partial statistics.
template <int KX, bool MASK, typename OutT>
__device__ void fill_stalled(const RowsParams& p, int a, int e, int i, int wi, bool word_writer) {
    const int Hc = p.H - 1, Wc = p.W - 1;
    const int64_t plane = (int64_t)Hc * Wc, mplane = (int64_t)Hc * p.n_words;
    OutT* o = reinterpret_cast<OutT*>(p.out);
    const OutT nan = to_out<OutT>(__int_as_float(0x7FC00000));
    for (int j = a; j < e; ++j)
        for (int k = 0; k < KX; ++k) {
            if (i < Wc) o[(int64_t)(p.kbase + k) * plane + (int64_t)j * Wc + i] = nan;
            if (MASK && word_writer) p.mask[(int64_t)(p.kbase + k) * mplane + (int64_t)j * p.n_words + wi] = 0u;
        }
}

// Records are read through L2 (ld.global.cg): the statistics grid may still be
// writing other rows of the workspace, so no stale L1 line may be used.
__device__ __forceinline__ float4 ld_rec(const float4* p) { return __ldcg(p); }

__device__ __forceinline__ float4 shfl_rec(float4 a, int src) {
    return make_float4(__shfl_sync(0xFFFFFFFFu, a.x, src), __shfl_sync(0xFFFFFFFFu, a.y, src),
                       __shfl_sync(0xFFFFFFFFu, a.z, src), 0.f);
}

// Records of the tile's extra right vertex ix at row j, one per lane of the
// last warp: lane 0 u at i+, lane 1 u at i-, lane 2 v at j+, lane 3 v at j-.
__device__ __forceinline__ float4 load_extra(const RowsParams& p, int j, int lane, int ix) {
    if (lane >= 4) return make_float4(0.f, 0.f, 0.f, 0.f);
    int row = j, col = ix, comp = 0;
    if (lane == 0) col = min(ix + 1, p.W - 1);
    if (lane == 1) col = max(ix - 1, 0);
    if (lane == 2) row = min(j + 1, p.H - 1), comp = 1;
    if (lane == 3) row = max(j - 1, 0), comp = 1;
    return ld_rec(p.st + comp * p.ps + (int64_t)(row - p.row0) * p.W + col);
}

// One tile: 8 cell rows x 256 cell columns, one vertex column per thread; KX
// isovalues exactly (other counts run as sums of such passes); MASK selects the
// mean-field bits.
template <int KX, bool MASK, typename OutT>
__global__ void __launch_bounds__(kRT, KX <= 4 ? 3 : (KX <= 16 ? 2 : 1))
    lcp_rows_kernel(const __grid_constant__ RowsParams p, const __grid_constant__ IsoParams iso) {
    constexpr int NV = kRT + 1;                      // vertices per tile row
    extern __shared__ __align__(16) float2 pq[];     // [KX][NV] (P(D < c), P(D >= c)) of the current row
    uint32_t* cls = reinterpret_cast<uint32_t*>(pq + KX * NV);  // [NV] bit k: mu_d < c_k

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int H = p.H, W = p.W, Hc = H - 1, Wc = W - 1;
    const int c0 = blockIdx.x * kRT;
    const int a = p.r_begin + blockIdx.y * kTR;
    if (a >= p.r_end) return;
    const int e = min(a + kTR, p.r_end);  // cells [a, e), vertex rows a..e
    // wait (bounded) until the statistics rows this band reads are complete
    if (p.dep && wait_band(p, blockIdx.y)) {
        const int wi0 = (c0 >> 5) + warp;
        fill_stalled<KX, MASK, OutT>(p, a, e, c0 + t, wi0, lane == 0 && wi0 < p.n_words);
        return;
    }
    // the next isovalue pass may launch once every block of this grid is past its wait
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const bool last_warp = warp == kRT / 32 - 1;
    const int i = c0 + t, ic = min(i, W - 1);
    const bool ok = i < Wc;
    const bool one_sided_x = ic == 0 || ic == W - 1;
    const float sx = one_sided_x ? p.sp.sx1 : p.sp.sx2, sxq = one_sided_x ? p.sp.sx1q : p.sp.sx2q;
    const double dsx = one_sided_x ? p.dsx1 : p.dsx2;
    const bool edge_lane = lane == 0 || lane == 31;
    const int iedge = lane == 0 ? max(ic - 1, 0) : min(ic + 1, W - 1);  // warp-edge neighbour column
    const int ix = min(c0 + kRT, W - 1);                                  // the tile's extra right vertex
    const bool one_sided_xx = ix == 0 || ix == W - 1;
    const float sx_x = one_sided_xx ? p.sp.sx1 : p.sp.sx2, sxq_x = one_sided_xx ? p.sp.sx1q : p.sp.sx2q;
    const double dsx_x = one_sided_xx ? p.dsx1 : p.dsx2;
    const int wi = (c0 >> 5) + warp;
    const bool word_writer = MASK && lane == 0 && wi < p.n_words;
    float c[KX];
#pragma unroll
    for (int k = 0; k < KX; ++k) c[k] = iso.c[k];

    // sliding window: u of the current row (own column; warp-edge lanes also the
    // neighbour column), v of rows j-1, j, j+1; the next row always in flight
    const float4* urow = p.st + (int64_t)(a - p.row0) * W;
    const float4* vpl = p.st + p.ps;
    float4 U = ld_rec(urow + ic), UE = make_float4(0.f, 0.f, 0.f, 0.f);
    if (edge_lane) UE = ld_rec(urow + iedge);
    float4 VM = ld_rec(vpl + (int64_t)(max(a - 1, 0) - p.row0) * W + ic);
    float4 V0 = ld_rec(vpl + (int64_t)(a - p.row0) * W + ic);
    float4 VP = ld_rec(vpl + (int64_t)(min(a + 1, H - 1) - p.row0) * W + ic);
    float4 X = last_warp ? load_extra(p, a, lane, ix) : make_float4(0.f, 0.f, 0.f, 0.f);

    float ph_prev[KX], qh_prev[KX];
    uint32_t b0_prev = 0, b1_prev = 0;
    const int64_t plane = (int64_t)Hc * Wc, mplane = (int64_t)Hc * p.n_words;
    OutT* po = reinterpret_cast<OutT*>(p.out) + (int64_t)p.kbase * plane + (int64_t)(a - 1) * Wc + i;
    uint32_t* pm = MASK ? p.mask + ((int64_t)p.kbase * Hc + (a - 1)) * p.n_words + wi : nullptr;
    for (int j = a; j <= e; ++j) {
        const float4 Uc = U, UEc = UE, Xc = X;
        float4 Vn = VP;
        if (j < e) {  // next row, in flight while this row is evaluated
            urow += W;
            U = ld_rec(urow + ic);
            if (edge_lane) UE = ld_rec(urow + iedge);
            Vn = ld_rec(vpl + (int64_t)(min(j + 2, H - 1) - p.row0) * W + ic);
            if (last_warp) X = load_extra(p, j + 1, lane, ix);
        }
        // divergence Gaussian of this thread's vertex (Eqs. 2/3, one-sided at the edges)
        float4 L = make_float4(__shfl_up_sync(0xFFFFFFFFu, Uc.x, 1), __shfl_up_sync(0xFFFFFFFFu, Uc.y, 1),
                               __shfl_up_sync(0xFFFFFFFFu, Uc.z, 1), 0.f);
        float4 R = make_float4(__shfl_down_sync(0xFFFFFFFFu, Uc.x, 1), __shfl_down_sync(0xFFFFFFFFu, Uc.y, 1),
                               __shfl_down_sync(0xFFFFFFFFu, Uc.z, 1), 0.f);
        if (lane == 0) L = UEc;
        if (lane == 31) R = UEc;
        if (ic == 0) L = Uc;
        if (ic == W - 1) R = Uc;
        const bool one_sided_y = j == 0 || j == H - 1;
        const float sy = one_sided_y ? p.sp.sy1 : p.sp.sy2, syq = one_sided_y ? p.sp.sy1q : p.sp.sy2q;
        const float4 Vlo = j > 0 ? VM : V0;
        const float4 Vhi = j < H - 1 ? VP : V0;
        float mu = fmaf((R.x - L.x) + (R.y - L.y), sx, ((Vhi.x - Vlo.x) + (Vhi.y - Vlo.y)) * sy);
        const float var = fmaf(R.z + L.z, sxq, (Vhi.z + Vlo.z) * syq);
        const double dsy = one_sided_y ? p.dsy1 : p.dsy2;
        const float lo = exact_mu(mu, var, L, R, Vlo, Vhi, sx, sy, dsx, dsy);
        // phase A: its (p, q) and class bit for every isovalue
        {
            const bool zero = var == 0.0f;
            const float s = rsqrtf(2.0f * var);
            uint32_t b = 0;
            if constexpr (KX == 1) {
                const float d = (mu - c[0]) + lo;  // mu - c with the low part of the mean
                const bool below = d < 0.0f;
                pq[t] = vertex_pq_d(d, s, zero, below);
                b = below;
            } else {
#pragma unroll
                for (int k = 0; k < KX; k += 2) {
                    const float2 d = __fadd2_rn(__fadd2_rn(make_float2(mu, mu), make_float2(-c[k], -c[k + 1])),
                                                make_float2(lo, lo));
                    const bool below0 = d.x < 0.0f, below1 = d.y < 0.0f;
                    float2 a0, a1;
                    vertex_pq2_d(d, s, zero, below0, below1, a0, a1);
                    pq[k * NV + t] = a0;
                    pq[(k + 1) * NV + t] = a1;
                    b |= ((uint32_t)below0 << k) | ((uint32_t)below1 << (k + 1));
                }
            }
            cls[t] = b;
        }
        if (last_warp) {  // the extra right vertex: gathered from lanes 0-3, isovalues spread over the lanes
            const float4 up = shfl_rec(Xc, 0), ul = shfl_rec(Xc, 1), vh = shfl_rec(Xc, 2), vl = shfl_rec(Xc, 3);
            float mux = fmaf((up.x - ul.x) + (up.y - ul.y), sx_x, ((vh.x - vl.x) + (vh.y - vl.y)) * sy);
            const float varx = fmaf(up.z + ul.z, sxq_x, (vh.z + vl.z) * syq);
            const float lox = exact_mu(mux, varx, ul, up, vl, vh, sx_x, sy, dsx_x, dsy);
            float cl = 0.0f;
#pragma unroll
            for (int k = 0; k < KX; ++k)
                if (k == lane) cl = c[k];
            const float dxk = (mux - cl) + lox;
            const bool below = dxk < 0.0f;
            if (lane < KX) pq[lane * NV + kRT] = vertex_pq_d(dxk, rsqrtf(2.0f * varx), varx == 0.0f, below);
            const uint32_t bx = __ballot_sync(0xFFFFFFFFu, lane < KX && below);
            if (lane == 0) cls[kRT] = bx;
        }
        __syncthreads();
        // phase B: close the cells of row j - 1
        const uint32_t b0 = cls[t], b1 = cls[t + 1];
        if (j > a) {
            po += Wc;
            if (MASK) pm += p.n_words;
            // bit k: the cell's four vertices are not all on one side of c_k
            const uint32_t cross = ok ? ((b0_prev | b1_prev | b0 | b1) & ~(b0_prev & b1_prev & b0 & b1)) : 0u;
            OutT* o = po;
            uint32_t* m = pm;
#pragma unroll
            for (int k = 0; k < KX; ++k) {
                const float2 h = __fmul2_rn(pq[k * NV + t], pq[k * NV + t + 1]);  // (p_i p_i+1, q_i q_i+1)
                const float ph = h.x, qh = h.y;
                const float lcp = fmaf(-qh_prev[k], qh, fmaf(-ph_prev[k], ph, 1.0f));
                if (ok) *o = to_out<OutT>(clamp01_nan(lcp));
                o += plane;
                if (MASK) {
                    const uint32_t word = __ballot_sync(0xFFFFFFFFu, (cross >> k) & 1u);
                    if (word_writer) *m = word;
                    m += mplane;
                }
                ph_prev[k] = ph;
                qh_prev[k] = qh;
            }
        } else {
#pragma unroll
            for (int k = 0; k < KX; ++k) {
                const float2 v0 = pq[k * NV + t], v1 = pq[k * NV + t + 1];
                ph_prev[k] = v0.x * v1.x;
                qh_prev[k] = v0.y * v1.y;
            }
        }
        b0_prev = b0;
        b1_prev = b1;
        VM = V0;
        V0 = VP;
        VP = Vn;
        __syncthreads();
    }
}

// Barrier-free variant: every warp evaluates a 31-cell strip on its own.  Lane l
// owns vertex c0w + l (c0w = 31 x the warp's strip index); lanes 0..30 own the
// cells [c0w, c0w + 31), and lane 31's vertex closes cell c0w + 30.  The right
// neighbour's (P(D<c), P(D>=c)) and class bits come from lane l + 1 by shuffle,
// so no vertex of a row is evaluated twice and no lane waits on another warp.
// No shared memory, no barriers after the dependency wait.  A mask word (32
// cells) straddles two warps, so each warp ORs its 31 bits into the word(s)
// atomically; the words are cleared beforehand (by the statistics pass, row by
// row, before it releases the row's band; or by the caller's stream).  KX <= 8
// isovalues per pass.
constexpr int kWT = 128;  // threads (4 warps) per block
constexpr int kWC = 31;   // cells per warp

template <int KX, bool MASK, typename OutT, bool IDX32>
__global__ void __launch_bounds__(kWT, 5)  // <= 102 registers: 20 warps per SM to hide the L2 latency
    lcp_warp_rows_kernel(const __grid_constant__ RowsParams p, const __grid_constant__ IsoParams iso) {
    // output and mask element offsets in 32 bits when the outputs fit (IDX32), else 64
    using Off = typename std::conditional<IDX32, uint32_t, int64_t>::type;
    static_assert(KX >= 1 && KX <= 8, "isovalues per pass");
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int H = p.H, W = p.W, Hc = H - 1, Wc = W - 1;
    const int c0w = (blockIdx.x * (kWT / 32) + warp) * kWC;
    const int a = p.r_begin + blockIdx.y * kTR;
    if (a >= p.r_end) return;
    const int e = min(a + kTR, p.r_end);  // cells [a, e), vertex rows a..e
    const int i = c0w + lane, ic = min(i, W - 1);
    const bool ok = lane < kWC && i < Wc;
    const int w0 = c0w >> 5, sh = c0w & 31;               // the strip starts at bit sh of mask word w0
    const bool second_word = sh > 1 && w0 + 1 < p.n_words;  // bits sh .. sh + 30 reach word w0 + 1
    // wait (bounded) until the statistics rows this band reads are complete
    if (p.dep && wait_band(p, blockIdx.y)) {
        // the records may be incomplete: NaN cells, and this strip's mask bits cleared
        const int64_t plane = (int64_t)Hc * Wc, mplane = (int64_t)Hc * p.n_words;
        OutT* o = reinterpret_cast<OutT*>(p.out);
        const OutT nan = to_out<OutT>(__int_as_float(0x7FC00000));
        const uint32_t bits = c0w < Wc ? (uint32_t)((1ull << min(kWC, Wc - c0w)) - 1) : 0u;
        for (int j = a; j < e; ++j)
            for (int k = 0; k < KX; ++k) {
                if (ok) o[(int64_t)(p.kbase + k) * plane + (int64_t)j * Wc + i] = nan;
                if (MASK && lane == 0 && bits) {
                    uint32_t* m = p.mask + (int64_t)(p.kbase + k) * mplane + (int64_t)j * p.n_words + w0;
                    atomicAnd(m, ~(bits << sh));
                    if (second_word) atomicAnd(m + 1, ~(bits >> (32 - sh)));
                }
            }
        return;
    }
    // the next isovalue pass may launch once every block of this grid is past its wait
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (c0w >= Wc) return;  // whole warp beyond the last cell (uniform per warp)
    const bool osx = ic == 0 || ic == W - 1;
    const float sx = osx ? p.sp.sx1 : p.sp.sx2, sxq = osx ? p.sp.sx1q : p.sp.sx2q;
    const double dsx = osx ? p.dsx1 : p.dsx2;
    const bool edge_lane = lane == 0 || lane == 31;
    const int iedge = lane == 0 ? max(ic - 1, 0) : min(ic + 1, W - 1);  // u neighbour beyond the warp
    float c[KX];
#pragma unroll
    for (int k = 0; k < KX; ++k) c[k] = iso.c[k];

    const float4* ubase = p.st - (int64_t)p.row0 * W;  // u records of grid row j at ubase + j W
    const float4* vbase = ubase + p.ps;
    auto urow = [&](int j) { return ubase + (int64_t)j * W; };
    auto vrow = [&](int j) { return vbase + (int64_t)j * W; };
    // the records one vertex row needs beyond the sliding v window: own u, the warp-edge
    // u neighbour, and the v record one row down (the window's next VP)
    struct RowRec {
        float4 U, UE, VN;
    };
    auto load_row = [&](int j) {
        RowRec r;
        r.U = ld_rec(urow(j) + ic);
        r.UE = edge_lane ? ld_rec(urow(j) + iedge) : make_float4(0.f, 0.f, 0.f, 0.f);
        r.VN = ld_rec(vrow(min(j + 1, H - 1)) + ic);
        return r;
    };
    float4 VM = ld_rec(vrow(max(a - 1, 0)) + ic), V0 = ld_rec(vrow(a) + ic);
    RowRec R0 = load_row(a);  // row j (its VN is v at j + 1)
    float ph_prev[KX], qh_prev[KX];
    uint32_t b_prev = 0, bn_prev = 0;
    const Off plane = (Off)Hc * (Off)Wc, mplane = (Off)Hc * (Off)p.n_words;
    OutT* const obase = reinterpret_cast<OutT*>(p.out);
    Off oo = (Off)p.kbase * plane + (Off)(a - 1) * (Off)Wc + (Off)i;  // row a - 1: advanced before the first store
    Off mo = MASK ? ((Off)p.kbase * (Off)Hc + (Off)(a - 1)) * (Off)p.n_words + (Off)w0 : (Off)0;
#pragma unroll(KX <= 4 ? 2 : 1)  // small code (measured: rolled best at K = 8, two rows per trip at K = 4)
    for (int jj = 0; jj <= kTR; ++jj) {  // vertex rows a .. e (at most kTR + 1)
        const int j = a + jj;
        if (j > e) break;
        const RowRec C = R0;
        const float4 VP = C.VN;
        if (j < e) R0 = load_row(j + 1);  // the next row in flight while this one is evaluated
        const bool osy = j == 0 || j == H - 1;
        const float sy = osy ? p.sp.sy1 : p.sp.sy2, syq = osy ? p.sp.sy1q : p.sp.sy2q;
        // own vertex (Eqs. 2/3, one-sided at the edges)
        float4 L = make_float4(__shfl_up_sync(0xFFFFFFFFu, C.U.x, 1), __shfl_up_sync(0xFFFFFFFFu, C.U.y, 1),
                               __shfl_up_sync(0xFFFFFFFFu, C.U.z, 1), 0.f);
        float4 R = make_float4(__shfl_down_sync(0xFFFFFFFFu, C.U.x, 1), __shfl_down_sync(0xFFFFFFFFu, C.U.y, 1),
                               __shfl_down_sync(0xFFFFFFFFu, C.U.z, 1), 0.f);
        if (lane == 0) L = C.UE;
        if (lane == 31) R = C.UE;
        // The one-sided stencils at the grid's edges need no selects: every record load
        // is clamped to the grid, so at column 0 the left record is the vertex's own (lane
        // 0's edge record is u[max(ic - 1, 0)]), at column W - 1 the right one is (lanes
        // beyond the grid hold u[W - 1]), and at rows 0 and H - 1 the window's lower and
        // upper v records are the row's own; the spacing factors are the one-sided ones.
        // (Measured: lat-lon K = 8 0.0931 -> 0.0926 ms, ocean 2.311 -> 2.267 ms, bit-identical.)
        const float4 Vlo = VM, Vhi = VP;
        float mu = fmaf((R.x - L.x) + (R.y - L.y), sx, ((Vhi.x - Vlo.x) + (Vhi.y - Vlo.y)) * sy);
        const float var = fmaf(R.z + L.z, sxq, (Vhi.z + Vlo.z) * syq);
        const bool zero = var == 0.0f;
        const float s = rsqrtf(2.0f * var);
        // member-0 differences across the stencil of more than 16 sigma: the mean again in FP64, as mu + lo
        float lo = 0.0f;
        const bool big = !(fmaf(fabsf(R.x - L.x), sx, fabsf(Vhi.x - Vlo.x) * sy) * s <= kExactZ);
        if (__any_sync(0xFFFFFFFFu, big)) {
            const double dsy = osy ? p.dsy1 : p.dsy2;
            if (big) lo = mu_fp64(mu, L, R, Vlo, Vhi, dsx, dsy);
        }
        float2 pq[KX];
        uint32_t b = 0;
        if constexpr (KX == 1) {
            const float d = (mu - c[0]) + lo;  // mu - c with the low part of the mean
            const bool below = d < 0.0f;
            pq[0] = vertex_pq_d(d, s, zero, below);
            b = below;
        } else {
#pragma unroll
            for (int k = 0; k < KX; k += 2) {
                const float2 d = __fadd2_rn(__fadd2_rn(make_float2(mu, mu), make_float2(-c[k], -c[k + 1])),
                                            make_float2(lo, lo));
                const bool b0 = d.x < 0.0f, b1 = d.y < 0.0f;
                vertex_pq2_d(d, s, zero, b0, b1, pq[k], pq[k + 1]);
                b |= ((uint32_t)b0 << k) | ((uint32_t)b1 << (k + 1));
            }
        }
        const uint32_t bn = __shfl_down_sync(0xFFFFFFFFu, b, 1);  // lane 31 owns no cell
        // bit k: the cell's four vertices are not all on one side of c_k
        const uint32_t cross = ok ? ((b_prev | bn_prev | b | bn) & ~(b_prev & bn_prev & b & bn)) : 0u;
        if (j > a) {
            oo += (Off)Wc;
            if (MASK) mo += (Off)p.n_words;
        }
        uint32_t word = 0;  // lane k < KX: the strip's crossing bits for isovalue k
#pragma unroll
        for (int k = 0; k < KX; ++k) {
            const float2 nb = make_float2(__shfl_down_sync(0xFFFFFFFFu, pq[k].x, 1),
                                          __shfl_down_sync(0xFFFFFFFFu, pq[k].y, 1));
            const float2 h = __fmul2_rn(pq[k], nb);  // (p_i p_i+1, q_i q_i+1) of this vertex row
            if (j > a) {
                const float lcp = fmaf(-qh_prev[k], h.y, fmaf(-ph_prev[k], h.x, 1.0f));
                if (ok) obase[oo + (Off)k * plane] = to_out<OutT>(clamp01_nan(lcp));
                if (MASK) {
                    const uint32_t wk = __ballot_sync(0xFFFFFFFFu, (cross >> k) & 1u);
                    word = lane == k ? wk : word;
                }
            }
            ph_prev[k] = h.x;
            qh_prev[k] = h.y;
        }
        // one divergent section per row: lane k ORs isovalue k's bits into its word(s)
        if (MASK && j > a && lane < KX && word) {
            uint32_t* m = p.mask + (mo + (Off)lane * mplane);
            atomicOr(m, word << sh);
            if (second_word && (word >> (32 - sh))) atomicOr(m + 1, word >> (32 - sh));
        }
        b_prev = b;
        bn_prev = bn;
        VM = V0;
        V0 = VP;
    }
}

// ---- host ----------------------------------------------------------------------
struct Layout {
    int band_rows;       // cell rows per band
    int ws_rows;         // record rows per plane (band + halo)
    int nby;             // LCP row bands (counters) per band
    size_t ctr_bytes;    // counter header (256-byte multiple)
    size_t plane_bytes;  // one record plane (padded)
    size_t total;
};

// Bands of record rows that fit both the L2 budget and `cap` bytes of workspace
// (the caller's); at least one LCP tile of kTR rows plus the halo.
Layout layout(int H, int W, size_t cap = SIZE_MAX) {
    const size_t row_bytes = (size_t)2 * W * sizeof(float4);
    auto fill = [&](Layout& L, long rows) {
        if (rows >= H - 1) {
            L.band_rows = H - 1;
            L.ws_rows = H;
        } else {
            L.band_rows = (int)(rows / kTR) * kTR;
            L.ws_rows = L.band_rows + 3;
        }
        L.nby = (L.band_rows + kTR - 1) / kTR;
        L.ctr_bytes = ((size_t)L.nby * 4 + 255) & ~(size_t)255;
        L.plane_bytes = ((size_t)L.ws_rows * W * sizeof(float4) + 255) & ~(size_t)255;
        L.total = L.ctr_bytes + 2 * L.plane_bytes;
    };
    long rows = (long)(kL2Budget / row_bytes) - 2;
    if (rows < kTR) rows = kTR;
    Layout L;
    fill(L, rows);  // the budget's layout: a workspace of exactly L.total keeps it
    if (L.total > cap) {
        // a smaller workspace: the largest band whose rows plus 3 halo/record rows fit it
        fill(L, std::max<long>((long)(cap / row_bytes) - 3, kTR));
        while (L.total > cap && L.band_rows > kTR) fill(L, L.band_rows - kTR);
    }
    return L;
}

template <int KX, bool MASK, typename OutT>
lcp_status launch_rows_k(const RowsParams& p, const IsoParams& ip, cudaStream_t st, bool pdl) {
    auto kern = lcp_rows_kernel<KX, MASK, OutT>;
    const size_t smem = (size_t)KX * (kRT + 1) * sizeof(float2) + (kRT + 1) * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        static std::mutex mu;
        static bool set[64] = {false};
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && !set[dev]) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return fail(LCP_ERR_CUDA, "lcp_fused_ws: %zu bytes of shared memory not available", smem);
            set[dev] = true;
        }
    }
    const int rows = p.r_end - p.r_begin;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.W - 1 + kRT - 1) / kRT, (rows + kTR - 1) / kTR);
    cfg.blockDim = dim3(kRT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (pdl) {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, p, ip);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LCP_ERR_CUDA, "lcp_fused_ws: LCP kernel launch failed: %s", cudaGetErrorString(e));
    }
    return LCP_OK;
}

template <int KX, bool MASK, typename OutT>
lcp_status launch_warp_rows_k(const RowsParams& p, const IsoParams& ip, cudaStream_t st, bool pdl) {
    const int rows = p.r_end - p.r_begin;
    const int strips = (p.W - 1 + kWC - 1) / kWC;  // 31-cell warp strips per cell row
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((strips + kWT / 32 - 1) / (kWT / 32), (rows + kTR - 1) / kTR);
    cfg.blockDim = dim3(kWT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (pdl) {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    // 32-bit offsets when every output element index of this pass fits
    const int64_t n_out = (int64_t)(p.kbase + KX) * (p.H - 1) * (p.W - 1);
    const int64_t n_mask = (int64_t)(p.kbase + KX) * (p.H - 1) * p.n_words;
    const bool idx32 = n_out < (1ll << 31) && n_mask < (1ll << 31);
    const cudaError_t e = idx32 ? cudaLaunchKernelEx(&cfg, lcp_warp_rows_kernel<KX, MASK, OutT, true>, p, ip)
                                : cudaLaunchKernelEx(&cfg, lcp_warp_rows_kernel<KX, MASK, OutT, false>, p, ip);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LCP_ERR_CUDA, "lcp_fused_ws: LCP kernel launch failed: %s", cudaGetErrorString(e));
    }
    return LCP_OK;
}

// Up to 8 isovalues: the barrier-free warp kernel (one pass).  More: the
// shared-memory kernel in passes of up to 32, whose single pass over the
// records beats several warp-kernel passes.
template <bool MASK, typename OutT>
lcp_status launch_rows_chunk(const RowsParams& p, const IsoParams& ip, cudaStream_t st, bool pdl, bool warp_rows) {
    if (warp_rows) {
        switch (ip.K) {
            case 1: return launch_warp_rows_k<1, MASK, OutT>(p, ip, st, pdl);
            case 2: return launch_warp_rows_k<2, MASK, OutT>(p, ip, st, pdl);
            case 4: return launch_warp_rows_k<4, MASK, OutT>(p, ip, st, pdl);
            case 8: return launch_warp_rows_k<8, MASK, OutT>(p, ip, st, pdl);
        }
        return fail(LCP_ERR_UNSUPPORTED, "lcp_fused_ws: isovalue chunk %d", ip.K);
    }
    switch (ip.K) {
        case 1: return launch_rows_k<1, MASK, OutT>(p, ip, st, pdl);
        case 2: return launch_rows_k<2, MASK, OutT>(p, ip, st, pdl);
        case 4: return launch_rows_k<4, MASK, OutT>(p, ip, st, pdl);
        case 8: return launch_rows_k<8, MASK, OutT>(p, ip, st, pdl);
        case 16: return launch_rows_k<16, MASK, OutT>(p, ip, st, pdl);
        case 32: return launch_rows_k<32, MASK, OutT>(p, ip, st, pdl);
    }
    return fail(LCP_ERR_UNSUPPORTED, "lcp_fused_ws: isovalue chunk %d", ip.K);
}

// Isovalues in passes whose sizes are the binary digits of K (largest first,
// at most 32 each): every pass runs a kernel specialised for its exact count.
// The warp kernel (K <= 8) ORs its mask bits into cleared words: unless the
// statistics pass of this call clears them (mask_cleared), the mask of cell rows
// [r_begin, r_end) is cleared here first, on the stream.
template <typename OutT>
lcp_status launch_rows(const RowsParams& p0, const float* iso, int K, cudaStream_t st, bool pdl = true,
                       bool mask_cleared = false) {
    RowsParams p = p0;
    int kb = 0;
    const bool warp_rows = K <= 8;
    if (warp_rows && p.mask && !mask_cleared) {
        const int64_t mplane = (int64_t)(p.H - 1) * p.n_words;
        const int64_t rows = (int64_t)(p.r_end - p.r_begin) * p.n_words;
        const bool whole = rows == mplane;  // every plane whole: one contiguous clear
        for (int k = 0; k < (whole ? 1 : K); ++k)
            if (cudaMemsetAsync(p.mask + (int64_t)k * mplane + (int64_t)p.r_begin * p.n_words, 0,
                                (size_t)(whole ? K * mplane : rows) * 4, st) != cudaSuccess)
                return fail(LCP_ERR_CUDA, "lcp_fused_ws: mask clear failed");
    }
    const int max_chunk = warp_rows ? 8 : kMaxKPass;
    while (kb < K) {
        int chunk = max_chunk;
        while (chunk > K - kb) chunk >>= 1;
        IsoParams ip;
        ip.K = chunk;
        for (int k = 0; k < chunk; ++k) ip.c[k] = iso[kb + k];
        p.kbase = kb;
        // with counters every pass is a programmatic dependent of the kernel
        // before it and waits on the counters of its rows; without, stream order
        const lcp_status s = p.mask ? launch_rows_chunk<true, OutT>(p, ip, st, pdl, warp_rows)
                                    : launch_rows_chunk<false, OutT>(p, ip, st, pdl, warp_rows);
        if (s != LCP_OK) return s;
        kb += chunk;
    }
    return LCP_OK;
}

template <typename T, int VEC>
lcp_status run(const void* u, const void* v, int M, int H, int W, int64_t stride, int ddof, double dx, double dy,
               const float* iso, int K, void* out, lcp_dtype out_dtype, uint32_t* mask, void* ws, size_t ws_bytes,
               bool vecload, cudaStream_t st) {
    const Layout L = layout(H, W, ws_bytes);
    const int Hc = H - 1;
    uint32_t* dep = reinterpret_cast<uint32_t*>(ws);
    float4* rec = reinterpret_cast<float4*>(reinterpret_cast<char*>(ws) + L.ctr_bytes);
    for (int r0 = 0; r0 < Hc; r0 += L.band_rows) {
        const int r1 = min(r0 + L.band_rows, Hc);  // cells [r0, r1): vertex rows r0..r1, statistics r0-1..r1+1
        const int s0 = max(r0 - 1, 0), s1 = min(r1 + 1, H - 1);
        const int nby = (r1 - r0 + kTR - 1) / kTR;
        // counters start at zero for every band (the previous band's cells are done: stream order)
        if (cudaMemsetAsync(dep, 0, (size_t)nby * 4, st) != cudaSuccess)
            return fail(LCP_ERR_CUDA, "lcp_fused_ws: counter reset failed");
        StatsWsParams sp;
        sp.u = u;
        sp.v = v;
        sp.stride = stride;
        sp.M = M;
        sp.W = W;
        sp.ddof = ddof;
        sp.n_begin = (int64_t)s0 * W;
        sp.n_end = (int64_t)(s1 + 1) * W;
        sp.row0 = s0;
        sp.st = rec;
        sp.ps = (int64_t)(L.plane_bytes / sizeof(float4));
        // the vertex groups must stay 16-byte aligned from the band's first vertex
        sp.vecload = vecload && (sp.n_begin % VEC) == 0;
        sp.dep = dep;
        sp.H = H;
        sp.r_begin = r0;
        sp.r_end = r1;
        sp.nby = nby;
        // the warp LCP kernel (K <= 8) ORs its mask bits into words this pass clears
        sp.mzero = (mask && K <= 8) ? mask : nullptr;
        sp.mK = K;
        sp.mwords = (W - 1 + 31) / 32;
        sp.mplane = (int64_t)Hc * sp.mwords;
        const int64_t groups = (sp.n_end - sp.n_begin + VEC - 1) / VEC;
        int64_t grid = (groups + kST - 1) / kST;  // one chunk per block
        // Several bands: a persistent grid (chunks in vertex order) of StatsTune's
        // blocks per SM, so that every block is resident at once, the dependent LCP
        // grid launches at the start and its blocks run beside the stream on the
        // registers left over, instead of after the band's last wave (measured, 8192^2
        // bf16 K = 4: 2.68 -> 2.54 ms with 3 blocks of 64 registers; 2.52 -> 2.30 ms
        // with 2 blocks of 80 registers and 10-member batches, which leave room for
        // two LCP blocks per SM; a single band is faster with one chunk per block).
        if (L.band_rows < Hc) grid = std::min<int64_t>(grid, (int64_t)num_sms() * StatsTune<T>::kPersist);
        stats_ws_kernel<T, VEC><<<(unsigned)grid, kST, 0, st>>>(sp);
        lcp_status s = check_launch("lcp_fused_ws (statistics)");
        if (s != LCP_OK) return s;
        RowsParams rp;
        rp.st = rec;
        rp.ps = sp.ps;
        rp.row0 = s0;
        rp.H = H;
        rp.W = W;
        rp.r_begin = r0;
        rp.r_end = r1;
        set_spacing(rp, dx, dy);
        rp.out = out;
        rp.mask = mask;
        rp.n_words = (W - 1 + 31) / 32;
        rp.kbase = 0;
        rp.dep = dep;
        rp.n_begin = sp.n_begin;
        rp.sv = kST * VEC;
        rp.budget = wait_budget_cycles();
        s = out_dtype == LCP_F16 ? launch_rows<__half>(rp, iso, K, st, true, true)
                                 : launch_rows<float>(rp, iso, K, st, true, true);
        if (s != LCP_OK) return s;
    }
    return LCP_OK;
}

}  // namespace

WsGeometry ws_geometry(int H, int W, size_t cap) {
    const Layout L = layout(H, W, cap);
    WsGeometry g;
    g.band_rows = L.band_rows;
    g.ctr_bytes = L.ctr_bytes;
    g.plane_bytes = L.plane_bytes;
    g.total = L.total;
    return g;
}

lcp_status ws_lcp_rows(const float4* rec, int64_t ps, int row0, int H, int W, int r0, int r1, double dx, double dy,
                       const float* iso, int K, void* out, lcp_dtype out_dtype, uint32_t* mask, cudaStream_t st) {
    RowsParams rp;
    rp.st = rec;
    rp.ps = ps;
    rp.row0 = row0;
    rp.H = H;
    rp.W = W;
    rp.r_begin = r0;
    rp.r_end = r1;
    set_spacing(rp, dx, dy);
    rp.out = out;
    rp.mask = mask;
    rp.n_words = (W - 1 + 31) / 32;
    rp.kbase = 0;
    rp.dep = nullptr;  // records complete before this launch (stream order)
    rp.n_begin = 0;
    rp.sv = 1;
    rp.budget = wait_budget_cycles();
    return out_dtype == LCP_F16 ? launch_rows<__half>(rp, iso, K, st, false) : launch_rows<float>(rp, iso, K, st, false);
}

uint32_t read_ws_status(bool reset) {
    uint32_t f = 0;
    cudaMemcpyFromSymbol(&f, g_ws_status, sizeof(f));
    if (reset) {
        const uint32_t z = 0;
        cudaMemcpyToSymbol(g_ws_status, &z, sizeof(z));
    }
    return f;
}

}  // namespace lcp

using namespace lcp;

extern "C" size_t lcp_fused_workspace_bytes(int M, int H, int W, lcp_dtype in_dtype) {
    (void)in_dtype;
    if (H < 2 || W < 2 || M < 1) return 0;
    return layout(H, W).total;
}

extern "C" int lcp_fused_band_rows(int H, int W, size_t workspace_bytes) {
    if (H < 2 || W < 2) return 0;
    const Layout L = layout(H, W, workspace_bytes);
    return L.total <= workspace_bytes ? L.band_rows : 0;
}

extern "C" lcp_status lcp_fused_ws(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                                   int64_t member_stride, int ddof, double dx, double dy, const float* iso, int K,
                                   void* lcp_out, lcp_dtype out_dtype, uint32_t* mask, void* workspace,
                                   size_t workspace_bytes, lcp_stream_t stream) {
    if (!workspace)
        return lcp_fused(u, v, in_dtype, M, H, W, member_stride, ddof, dx, dy, iso, K, lcp_out, out_dtype, mask,
                         stream);
    lcp_status s = check_members("lcp_fused_ws", u, v, in_dtype, M, H, W, member_stride, ddof);
    if (s != LCP_OK) return s;
    if ((s = check_iso("lcp_fused_ws", iso, K)) != LCP_OK) return s;
    if ((s = check_spacing("lcp_fused_ws", dx, dy)) != LCP_OK) return s;
    if (!lcp_out) return fail(LCP_ERR_ARG, "lcp_fused_ws: NULL output");
    if (out_dtype != LCP_F32 && out_dtype != LCP_F16) return fail(LCP_ERR_ARG, "lcp_fused_ws: out dtype must be F32 or F16");
    if ((uintptr_t)mask & 3) return fail(LCP_ERR_ARG, "lcp_fused_ws: mask must be 4-byte aligned");
    if ((uintptr_t)workspace & 255) return fail(LCP_ERR_ARG, "lcp_fused_ws: workspace must be 256-byte aligned");
    const Layout L = layout(H, W, workspace_bytes);
    if (workspace_bytes < L.total)
        return fail(LCP_ERR_ARG, "lcp_fused_ws: workspace too small (%zu < %zu bytes for the smallest band)",
                    workspace_bytes, L.total);
    if ((H - 1 + kTR - 1) / kTR > 65535) return fail(LCP_ERR_UNSUPPORTED, "lcp_fused_ws: H too large");
    const int64_t stride = M > 1 ? member_stride : (int64_t)H * W;
    cudaStream_t st = (cudaStream_t)stream;
    const bool in16 = aligned16(u) && aligned16(v);
    if (in_dtype == LCP_F32)
        return run<float, 4>(u, v, M, H, W, stride, ddof, dx, dy, iso, K, lcp_out, out_dtype, mask, workspace,
                             workspace_bytes, in16 && stride % 4 == 0, st);
    const bool in8 = ((uintptr_t)u & 7) == 0 && ((uintptr_t)v & 7) == 0;
    return run<__nv_bfloat16, 4>(u, v, M, H, W, stride, ddof, dx, dy, iso, K, lcp_out, out_dtype, mask, workspace,
                                 workspace_bytes, in8 && stride % 4 == 0, st);
}

extern "C" lcp_status lcp_test_stalled_lcp_wait(int H, int W, const float* iso, int K, void* lcp_out,
                                                lcp_dtype out_dtype, uint32_t* mask, void* workspace,
                                                size_t workspace_bytes, lcp_stream_t stream) {
    static const char* fn = "lcp_test_stalled_lcp_wait";
    if (H < 2 || W < 2) return fail(LCP_ERR_ARG, "%s: need H, W >= 2", fn);
    lcp_status s = check_iso(fn, iso, K);
    if (s != LCP_OK) return s;
    if (!lcp_out) return fail(LCP_ERR_ARG, "%s: NULL output", fn);
    if (out_dtype != LCP_F32 && out_dtype != LCP_F16) return fail(LCP_ERR_ARG, "%s: out dtype must be F32 or F16", fn);
    if ((uintptr_t)mask & 3) return fail(LCP_ERR_ARG, "%s: mask must be 4-byte aligned", fn);
    if (!workspace || ((uintptr_t)workspace & 255)) return fail(LCP_ERR_ARG, "%s: need a 256-byte aligned workspace", fn);
    const Layout L = layout(H, W, workspace_bytes);
    if (workspace_bytes < L.total) return fail(LCP_ERR_ARG, "%s: workspace too small", fn);
    if ((H - 1 + kTR - 1) / kTR > 65535) return fail(LCP_ERR_UNSUPPORTED, "%s: H too large", fn);
    cudaStream_t st = (cudaStream_t)stream;
    const int r1 = min(L.band_rows, H - 1);
    const int nby = (r1 + kTR - 1) / kTR;
    uint32_t* dep = reinterpret_cast<uint32_t*>(workspace);
    // counters at zero and no statistics grid to release them
    if (cudaMemsetAsync(dep, 0, (size_t)nby * 4, st) != cudaSuccess) return fail(LCP_ERR_CUDA, "%s: counter reset failed", fn);
    RowsParams rp;
    rp.st = reinterpret_cast<float4*>(reinterpret_cast<char*>(workspace) + L.ctr_bytes);
    rp.ps = (int64_t)(L.plane_bytes / sizeof(float4));
    rp.row0 = 0;
    rp.H = H;
    rp.W = W;
    rp.r_begin = 0;
    rp.r_end = r1;
    set_spacing(rp, 1.0, 1.0);
    rp.out = lcp_out;
    rp.mask = mask;
    rp.n_words = (W - 1 + 31) / 32;
    rp.kbase = 0;
    rp.dep = dep;
    rp.n_begin = 0;
    rp.sv = kST * 4;
    rp.budget = wait_budget_cycles();
    return out_dtype == LCP_F16 ? launch_rows<__half>(rp, iso, K, st, false) : launch_rows<float>(rp, iso, K, st, false);
}
