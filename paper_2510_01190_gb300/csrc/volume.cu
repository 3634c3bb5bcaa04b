// 3D vector fields (the extension Sec. 5 names as future work): Eq. 1 with the
// z term (w_{k+1} - w_{k-1}) / (2 dz) under the same one-sided boundary rule,
// Eqs. 2/3 with the matching mean and variance terms, and the LCP of
// hexahedral cells, 1 - prod_8 P(D < c) - prod_8 P(D >= c).
//
// lcp3d_fused_ws runs in slabs of z-planes through an L2-resident ring of
// statistics records:
// 1) stats3_kernel: a flat, coalesced stream over the member planes of the
//    slab's new z-planes; per vertex and component one 16-byte record
//    (x0, delta, var, 0) -- member 0, the FP32 mean of the members shifted by
//    member 0, and the variance -- stored with an L2 evict-last policy into
//    ring slot (plane % S).  Planes are computed once: the ring keeps the three
//    older planes the next cells still need, and room for the next slab, whose
//    statistics run on the caller's stream beside this slab's LCP kernel on a
//    second stream (fork and join by events).
// 2) lcp3_kernel: a block owns a tile of 31 x 8 cells (32 x 9 vertices, one
//    thread each) and marches along z over a chunk of cell planes.  Per vertex
//    plane every thread forms its vertex's divergence Gaussian from six
//    records (the x0 and delta differences kept apart, so that equal means
//    cancel exactly) and one erfc per isovalue into shared memory (double
//    buffered, one barrier per plane); then each thread closes its cell from
//    the four vertices of this plane and the four-vertex products of the
//    previous plane, kept in registers.  Every vertex is evaluated ~1.16 times
//    (the tile's halo), not once per cell.  Mean-field crossing bits go out
//    with atomicOr into a mask cleared before the first slab (a tile's 31
//    cells straddle two mask words).
//
// lcp3d_divergence and lcp3d_map are the unfused steps (Eqs. 2/3 from given
// statistics; the LCP map from given divergence Gaussians).
#include <algorithm>
#include <cmath>
#include <mutex>

#include "lcp_common.cuh"

namespace lcp {
namespace {

constexpr int kS3T = 256;           // statistics threads per block
constexpr int kL3C = 31;            // cells per LCP tile along x (32 vertices)
constexpr int kL3R = 8;             // cells per LCP tile along y (9 vertex rows)
constexpr int kL3VY = kL3R + 1;
constexpr int kL3T = 32 * kL3VY;    // LCP threads: one per vertex of the tile
constexpr int kL3Z = 4;             // cell planes per LCP block (z march)
constexpr size_t kL2Budget3 = 96ull << 20;
constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint64_t pol_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t pol_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void st_last(float4* p, float4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w), "l"(pol)
                 : "memory");
}

// ---- member loads: 4 consecutive vertices per thread ------------------------
template <typename T>
struct Ld4;
template <>
struct Ld4<float> {
    using raw = float4;
    static __device__ __forceinline__ raw ld(const float* p, uint64_t pol) {
        float4 r;
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                     : "l"(p), "l"(pol));
        return r;
    }
    static __device__ __forceinline__ void cvt(const raw& r, float* x) {
        x[0] = r.x;
        x[1] = r.y;
        x[2] = r.z;
        x[3] = r.w;
    }
    static __device__ __forceinline__ float one(const float* p) { return __ldg(p); }
};
template <>
struct Ld4<__nv_bfloat16> {
    using raw = uint2;
    static __device__ __forceinline__ raw ld(const __nv_bfloat16* p, uint64_t pol) {
        uint2 r;
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
                     : "=r"(r.x), "=r"(r.y)
                     : "l"(p), "l"(pol));
        return r;
    }
    static __device__ __forceinline__ void cvt(const raw& r, float* x) {
        x[0] = __uint_as_float(r.x << 16);
        x[1] = __uint_as_float(r.x & 0xFFFF0000u);
        x[2] = __uint_as_float(r.y << 16);
        x[3] = __uint_as_float(r.y & 0xFFFF0000u);
    }
    static __device__ __forceinline__ float one(const __nv_bfloat16* p) {
        return __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p)) << 16);
    }
};

struct Stats3Params {
    const void* c[3];   // u, v, w
    int64_t stride;
    int M, ddof;
    int64_t hw;         // vertices per z-plane
    int64_t n_begin, n_end;  // flat vertex range of this slab's new planes
    float4* ring;       // [3][S][hw] records
    int S;
    int vecload;
};

__device__ __forceinline__ float4 make_rec(float x0, float s1, float s2, float fm, float fdof) {
    const float dl = s1 / fm;
    float vv = (s2 - s1 * dl) / fdof;
    vv = vv < 0.f ? 0.f : vv;  // NaN stays NaN
    return make_float4(x0, dl, vv, 0.f);
}

template <typename T>
__global__ void __launch_bounds__(kS3T, 2) stats3_kernel(const __grid_constant__ Stats3Params p) {
    using L = Ld4<T>;
    const uint64_t pf = pol_first(), pl = pol_last();
    const int64_t n0 = p.n_begin + ((int64_t)blockIdx.x * kS3T + threadIdx.x) * 4;
    if (n0 >= p.n_end) return;
    const float fm = (float)p.M, fdof = (float)(p.M - p.ddof);
    const int64_t ring_plane = (int64_t)p.S * p.hw;
    if (p.vecload && n0 + 4 <= p.n_end) {
        float x0[3][4], s1[3][4], s2[3][4];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            L::cvt(L::ld(reinterpret_cast<const T*>(p.c[c]) + n0, pf), x0[c]);
#pragma unroll
            for (int e = 0; e < 4; ++e) s1[c][e] = s2[c][e] = 0.f;
        }
        constexpr int U = 2;  // members per batch: 6 loads in flight per thread (registers left for an LCP block)
        int m = 1;
        auto acc = [&](const typename L::raw (&r)[3]) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float x[4];
                L::cvt(r[c], x);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float d = x[e] - x0[c][e];
                    s1[c][e] += d;
                    s2[c][e] = fmaf(d, d, s2[c][e]);
                }
            }
        };
        for (; m + U <= p.M; m += U) {
            typename L::raw r[U][3];
#pragma unroll
            for (int q = 0; q < U; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    r[q][c] = L::ld(reinterpret_cast<const T*>(p.c[c]) + (int64_t)(m + q) * p.stride + n0, pf);
#pragma unroll
            for (int q = 0; q < U; ++q) acc(r[q]);
        }
        for (; m < p.M; ++m) {
            typename L::raw r[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                r[c] = L::ld(reinterpret_cast<const T*>(p.c[c]) + (int64_t)m * p.stride + n0, pf);
            acc(r);
        }
        const int64_t k = n0 / p.hw, rem = n0 - k * p.hw;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const bool next = rem + e >= p.hw;  // the group may cross into the next plane
            const int64_t kk = next ? k + 1 : k, off = next ? rem + e - p.hw : rem + e;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                st_last(p.ring + c * ring_plane + (kk % p.S) * p.hw + off, make_rec(x0[c][e], s1[c][e], s2[c][e], fm, fdof),
                        pl);
        }
    } else {
        const int64_t n_end = min(n0 + 4, p.n_end);
        for (int64_t n = n0; n < n_end; ++n) {
            const int64_t k = n / p.hw;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T* src = reinterpret_cast<const T*>(p.c[c]);
                const float x0 = L::one(src + n);
                float a1 = 0.f, a2 = 0.f;
                for (int m = 1; m < p.M; ++m) {
                    const float d = L::one(src + (int64_t)m * p.stride + n) - x0;
                    a1 += d;
                    a2 = fmaf(d, d, a2);
                }
                st_last(p.ring + c * ring_plane + (k % p.S) * p.hw + (n - k * p.hw), make_rec(x0, a1, a2, fm, fdof), pl);
            }
        }
    }
}

// ---- LCP from the records -----------------------------------------------------
struct Lcp3Params {
    const float4* ring;  // [3][S][hw]
    int S;
    int D, H, W;
    int k_begin, k_end;  // cell planes of this launch
    float sx1, sx2, sy1, sy2, sz1, sz2;
    float sx1q, sx2q, sy1q, sy2q, sz1q, sz2q;
    void* out;
    uint32_t* mask;
    int n_words;
    int kbase;
};


// one term of Eq. 2 / Eq. 3: the difference of two records and their summed variance
__device__ __forceinline__ void term(const float4& hi, const float4& lo, float s, float sq, float& mu, float& var) {
    mu = fmaf((hi.x - lo.x) + (hi.y - lo.y), s, mu);
    var = fmaf(hi.z + lo.z, sq, var);
}

template <int KX, bool MASK, typename OutT>
__global__ void __launch_bounds__(kL3T, 3) lcp3_kernel(const __grid_constant__ Lcp3Params p,
                                                       const __grid_constant__ IsoParams iso) {
    __shared__ float2 s_pq[2][KX][kL3VY][32];
    __shared__ uint32_t s_bits[2][kL3VY][32];
    const int t = threadIdx.x, lx = t & 31, ly = t >> 5;
    const int D = p.D, H = p.H, W = p.W;
    const int i0 = blockIdx.x * kL3C, j0 = blockIdx.y * kL3R;
    const int ka = p.k_begin + blockIdx.z * kL3Z;
    const int kb = min(ka + kL3Z, p.k_end);  // cell planes [ka, kb): vertex planes ka .. kb
    const int Hc = H - 1, Wc = W - 1, Dc = D - 1;
    // vertex of this thread in the vertex phase (clamped into the grid for loads)
    const int vi = min(i0 + lx, W - 1), vj = min(j0 + ly, H - 1);
    const int il = max(vi - 1, 0), ih = min(vi + 1, W - 1), jl = max(vj - 1, 0), jh = min(vj + 1, H - 1);
    const float sx = ih - il == 2 ? p.sx2 : p.sx1, sxq = ih - il == 2 ? p.sx2q : p.sx1q;
    const float sy = jh - jl == 2 ? p.sy2 : p.sy1, syq = jh - jl == 2 ? p.sy2q : p.sy1q;
    // cell of this thread in the cell phase
    const int ci = i0 + lx, cj = j0 + ly;
    const bool cell_ok = lx < kL3C && ly < kL3R && ci < Wc && cj < Hc;
    const int64_t hw = (int64_t)H * W, ring_plane = (int64_t)p.S * hw;
    const float4* ru = p.ring;
    const float4* rv = p.ring + ring_plane;
    const float4* rw = p.ring + 2 * ring_plane;
    const int64_t ox_l = (int64_t)vj * W + il, ox_h = (int64_t)vj * W + ih;
    const int64_t oy_l = (int64_t)jl * W + vi, oy_h = (int64_t)jh * W + vi, oz = (int64_t)vj * W + vi;
    float c[KX];
#pragma unroll
    for (int k = 0; k < KX; ++k) c[k] = iso.c[k];
    float pp_prev[KX], qq_prev[KX];
    uint32_t or_prev = 0, and_prev = 0;
    OutT* const obase = reinterpret_cast<OutT*>(p.out);
    for (int kv = ka; kv <= kb; ++kv) {
        const int buf = (kv - ka) & 1;
        {  // vertex phase: divergence Gaussian (Eqs. 2/3 with the z term) and (p, q) per isovalue
            const int kl = max(kv - 1, 0), kh = min(kv + 1, D - 1);
            const float sz = kh - kl == 2 ? p.sz2 : p.sz1, szq = kh - kl == 2 ? p.sz2q : p.sz1q;
            const int64_t sv = (int64_t)(kv % p.S) * hw;
            const float4 ul = __ldg(ru + sv + ox_l), uh = __ldg(ru + sv + ox_h);
            const float4 vl = __ldg(rv + sv + oy_l), vh = __ldg(rv + sv + oy_h);
            const float4 wl = __ldg(rw + (int64_t)(kl % p.S) * hw + oz), wh = __ldg(rw + (int64_t)(kh % p.S) * hw + oz);
            float mu = 0.f, var = 0.f;
            term(uh, ul, sx, sxq, mu, var);
            term(vh, vl, sy, syq, mu, var);
            term(wh, wl, sz, szq, mu, var);
            const bool zero = var == 0.f;  // a NaN variance stays NaN
            const float sg = zero ? 0.f : rsqrtf(2.f * var);
            uint32_t bits = 0;
#pragma unroll
            for (int k = 0; k < KX; ++k) {
                const bool below = mu < c[k];
                bits |= below ? (1u << k) : 0u;
                s_pq[buf][k][ly][lx] = vertex_pq(mu, sg, zero, c[k], below);
            }
            s_bits[buf][ly][lx] = bits;
        }
        __syncthreads();
        if (ly < kL3R) {  // cell phase: the 4 vertices of this plane, then the cell with the previous plane
            float pp[KX], qq[KX];
#pragma unroll
            for (int k = 0; k < KX; ++k) {
                const int lx1 = min(lx + 1, 31);
                const float2 a = s_pq[buf][k][ly][lx], b = s_pq[buf][k][ly][lx1];
                const float2 e = s_pq[buf][k][ly + 1][lx], f = s_pq[buf][k][ly + 1][lx1];
                pp[k] = (a.x * b.x) * (e.x * f.x);
                qq[k] = (a.y * b.y) * (e.y * f.y);
            }
            const int lx1 = min(lx + 1, 31);
            const uint32_t b0 = s_bits[buf][ly][lx], b1 = s_bits[buf][ly][lx1];
            const uint32_t b2 = s_bits[buf][ly + 1][lx], b3 = s_bits[buf][ly + 1][lx1];
            const uint32_t o4 = b0 | b1 | b2 | b3, a4 = b0 & b1 & b2 & b3;
            if (kv > ka) {
                const int kc = kv - 1;
#pragma unroll
                for (int k = 0; k < KX; ++k) {
                    if (cell_ok) {
                        const int64_t o = (((int64_t)(p.kbase + k) * Dc + kc) * Hc + cj) * Wc + ci;
                        obase[o] = to_out<OutT>(clamp01_nan(1.f - pp_prev[k] * pp[k] - qq_prev[k] * qq[k]));
                    }
                }
                if (MASK) {
                    const uint32_t cross = (or_prev | o4) & ~(and_prev & a4);
#pragma unroll
                    for (int k = 0; k < KX; ++k) {
                        const uint32_t bal = __ballot_sync(kFull, cell_ok && ((cross >> k) & 1u));
                        if (lx == 0 && bal) {
                            uint32_t* mrow = p.mask + (((int64_t)(p.kbase + k) * Dc + kc) * Hc + cj) * p.n_words;
                            const int w0 = i0 >> 5, sh = i0 & 31;
                            atomicOr(mrow + w0, bal << sh);
                            if (sh && (bal >> (32 - sh))) atomicOr(mrow + w0 + 1, bal >> (32 - sh));
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < KX; ++k) {
                pp_prev[k] = pp[k];
                qq_prev[k] = qq[k];
            }
            or_prev = o4;
            and_prev = a4;
        }
        // the next plane writes the other buffer; the barrier above (next step)
        // keeps it from overwriting this one while cells still read it
    }
}

// ---- unfused steps ----------------------------------------------------------------
__global__ void div3_kernel(const float* __restrict__ mu_u, const float* __restrict__ var_u,
                            const float* __restrict__ mu_v, const float* __restrict__ var_v,
                            const float* __restrict__ mu_w, const float* __restrict__ var_w, int D, int H, int W,
                            float sx1, float sx2, float sy1, float sy2, float sz1, float sz2, float* __restrict__ mu_d,
                            float* __restrict__ var_d) {
    const int64_t hw = (int64_t)H * W, n = hw * D;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(q / hw);
        const int64_t r = q - (int64_t)k * hw;
        const int j = (int)(r / W), i = (int)(r - (int64_t)j * W);
        const int il = max(i - 1, 0), ih = min(i + 1, W - 1), jl = max(j - 1, 0), jh = min(j + 1, H - 1);
        const int kl = max(k - 1, 0), kh = min(k + 1, D - 1);
        const float sx = ih - il == 2 ? sx2 : sx1, sy = jh - jl == 2 ? sy2 : sy1, sz = kh - kl == 2 ? sz2 : sz1;
        const int64_t base = (int64_t)k * hw + (int64_t)j * W;
        const int64_t xl = base + il, xh = base + ih;
        const int64_t yl = (int64_t)k * hw + (int64_t)jl * W + i, yh = (int64_t)k * hw + (int64_t)jh * W + i;
        const int64_t zl = (int64_t)kl * hw + (int64_t)j * W + i, zh = (int64_t)kh * hw + (int64_t)j * W + i;
        mu_d[q] = (mu_u[xh] - mu_u[xl]) * sx + (mu_v[yh] - mu_v[yl]) * sy + (mu_w[zh] - mu_w[zl]) * sz;
        var_d[q] = (var_u[xh] + var_u[xl]) * (sx * sx) + (var_v[yh] + var_v[yl]) * (sy * sy) +
                   (var_w[zh] + var_w[zl]) * (sz * sz);
    }
}

// one thread per cell (all isovalues); a warp covers 32 consecutive cells of a
// row, aligned to a mask word, so the crossing bits are whole ballots
template <typename OutT>
__global__ void __launch_bounds__(256) map3_kernel(const float* __restrict__ mu_d, const float* __restrict__ var_d,
                                                   int D, int H, int W, const __grid_constant__ IsoParams iso,
                                                   OutT* __restrict__ out, uint32_t* __restrict__ mask, int n_words) {
    const int Wc = W - 1, Hc = H - 1, Dc = D - 1;
    const int64_t rows = (int64_t)Dc * Hc, per_row = (int64_t)n_words * 32;
    const int64_t n = rows * per_row;
    const int lane = threadIdx.x & 31;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q - lane < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = q / per_row;
        const int i = (int)(q - row * per_row);
        const int kc = (int)(row / Hc), jc = (int)(row - (int64_t)kc * Hc);
        const bool ok = q < n && i < Wc;
        float mu[8], sd[8];
        bool zero[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int di = v & 1, dj = (v >> 1) & 1, dk = v >> 2;
            const int64_t o = ((int64_t)min(kc + dk, D - 1) * H + min(jc + dj, H - 1)) * W + min(i + di, W - 1);
            mu[v] = ok ? mu_d[o] : 0.f;
            const float vv = ok ? var_d[o] : 0.f;
            zero[v] = vv == 0.f;
            sd[v] = zero[v] ? 0.f : rsqrtf(2.f * vv);
        }
        for (int k = 0; k < iso.K; ++k) {
            const float c = iso.c[k];
            float pp = 1.f, qq = 1.f;
            int nb = 0;
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const bool below = mu[v] < c;
                nb += below;
                const float2 pq = vertex_pq(mu[v], sd[v], zero[v], c, below);
                pp *= pq.x;
                qq *= pq.y;
            }
            if (ok) out[(((int64_t)k * Dc + kc) * Hc + jc) * Wc + i] = to_out<OutT>(clamp01_nan(1.f - pp - qq));
            if (mask) {
                const uint32_t bal = __ballot_sync(kFull, ok && nb > 0 && nb < 8);
                if (lane == 0 && q < n) mask[(((int64_t)k * Dc + kc) * Hc + jc) * n_words + (i >> 5)] = bal;
            }
        }
    }
}

struct Ring {
    int S;           // plane slots
    int B;           // new statistics planes per slab
    size_t bytes;    // 3 * S * hw * 16
};

// The ring holds S >= 2B + 3 planes, B new planes per slab: the three older planes
// the next cells need, and room for the next slab's statistics to be written
// while the LCP of this slab still reads its planes (the two run concurrently).
Ring ring_for(int D, int H, int W) {
    const size_t plane = (size_t)H * W * 3 * sizeof(float4);
    const int fit = (int)(kL2Budget3 / plane);
    int B = std::max(1, (fit - 3) / 2);
    B = std::min(B, D);
    Ring r;
    r.B = B;
    r.S = 2 * B + 3;
    r.bytes = (size_t)r.S * plane;
    return r;
}

// A second stream per host thread and device for the LCP kernels, and ping-pong
// events for the fork / join with the caller's stream.
struct SideStream {
    cudaStream_t st = nullptr;
    cudaEvent_t ev_stats[2] = {nullptr, nullptr}, ev_lcp[2] = {nullptr, nullptr};
};

lcp_status side_stream(SideStream*& out) {
    thread_local SideStream per_dev[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(LCP_ERR_CUDA, "lcp3d_fused_ws: no device");
    SideStream& ss = per_dev[dev];
    if (!ss.st) {
        if (cudaStreamCreateWithFlags(&ss.st, cudaStreamNonBlocking) != cudaSuccess)
            return fail(LCP_ERR_CUDA, "lcp3d_fused_ws: stream creation failed");
        for (int q = 0; q < 2; ++q)
            if (cudaEventCreateWithFlags(&ss.ev_stats[q], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ss.ev_lcp[q], cudaEventDisableTiming) != cudaSuccess)
                return fail(LCP_ERR_CUDA, "lcp3d_fused_ws: event creation failed");
    }
    out = &ss;
    return LCP_OK;
}

template <int KX, bool MASK, typename OutT>
lcp_status launch_lcp3(const Lcp3Params& p, const IsoParams& ip, cudaStream_t st) {
    const dim3 grid((p.W - 1 + kL3C - 1) / kL3C, (p.H - 1 + kL3R - 1) / kL3R, (p.k_end - p.k_begin + kL3Z - 1) / kL3Z);
    lcp3_kernel<KX, MASK, OutT><<<grid, kL3T, 0, st>>>(p, ip);
    return check_launch("lcp3d_fused_ws (LCP)");
}

template <bool MASK, typename OutT>
lcp_status launch_lcp3_chunk(const Lcp3Params& p, const IsoParams& ip, cudaStream_t st) {
    switch (ip.K) {
        case 1: return launch_lcp3<1, MASK, OutT>(p, ip, st);
        case 2: return launch_lcp3<2, MASK, OutT>(p, ip, st);
        case 4: return launch_lcp3<4, MASK, OutT>(p, ip, st);
        case 8: return launch_lcp3<8, MASK, OutT>(p, ip, st);
    }
    return fail(LCP_ERR_UNSUPPORTED, "lcp3d_fused_ws: isovalue chunk %d", ip.K);
}

template <typename OutT>
lcp_status lcp3_passes(const Lcp3Params& p0, const float* iso, int K, cudaStream_t st) {
    Lcp3Params p = p0;
    int kb = 0;
    while (kb < K) {
        int chunk = 8;
        while (chunk > K - kb) chunk >>= 1;
        IsoParams ip;
        ip.K = chunk;
        for (int k = 0; k < chunk; ++k) ip.c[k] = iso[kb + k];
        p.kbase = kb;
        const lcp_status s = p.mask ? launch_lcp3_chunk<true, OutT>(p, ip, st) : launch_lcp3_chunk<false, OutT>(p, ip, st);
        if (s != LCP_OK) return s;
        kb += chunk;
    }
    return LCP_OK;
}

template <typename T>
lcp_status run3(const void* u, const void* v, const void* w, int M, int D, int H, int W, int64_t stride, int ddof,
                double dx, double dy, double dz, const float* iso, int K, void* out, lcp_dtype out_dtype,
                uint32_t* mask, void* ws, bool vec_ok, cudaStream_t st) {
    const Ring rg = ring_for(D, H, W);
    const int64_t hw = (int64_t)H * W;
    if (mask) {
        const size_t mbytes = (size_t)K * (D - 1) * (H - 1) * ((W - 1 + 31) / 32) * sizeof(uint32_t);
        if (cudaMemsetAsync(mask, 0, mbytes, st) != cudaSuccess) return fail(LCP_ERR_CUDA, "lcp3d_fused_ws: mask clear failed");
    }
    Stats3Params sp;
    sp.c[0] = u;
    sp.c[1] = v;
    sp.c[2] = w;
    sp.stride = stride;
    sp.M = M;
    sp.ddof = ddof;
    sp.hw = hw;
    sp.ring = reinterpret_cast<float4*>(ws);
    sp.S = rg.S;
    Lcp3Params lp;
    lp.ring = sp.ring;
    lp.S = rg.S;
    lp.D = D;
    lp.H = H;
    lp.W = W;
    lp.sx1 = (float)(1.0 / dx);
    lp.sx2 = (float)(0.5 / dx);
    lp.sy1 = (float)(1.0 / dy);
    lp.sy2 = (float)(0.5 / dy);
    lp.sz1 = (float)(1.0 / dz);
    lp.sz2 = (float)(0.5 / dz);
    lp.sx1q = (float)(1.0 / (dx * dx));
    lp.sx2q = (float)(0.25 / (dx * dx));
    lp.sy1q = (float)(1.0 / (dy * dy));
    lp.sy2q = (float)(0.25 / (dy * dy));
    lp.sz1q = (float)(1.0 / (dz * dz));
    lp.sz2q = (float)(0.25 / (dz * dz));
    lp.out = out;
    lp.mask = mask;
    lp.n_words = (W - 1 + 31) / 32;
    lp.kbase = 0;
    // Slab t: statistics of planes [P_t, P_t + B) on the caller's stream, then the LCP of the cells
    // they complete on the side stream.  The statistics of slab t + 1 overwrite ring slots that only
    // the LCP of slab t - 1 still reads, so they wait for that one and run beside the LCP of slab t.
    SideStream* ss = nullptr;
    lcp_status s = side_stream(ss);
    if (s != LCP_OK) return s;
    int P = 0, C = 0, t = 0;
    bool lcp_pending[2] = {false, false};
    while (C < D - 1) {
        const int Pn = std::min(P + rg.B, D);
        if (t >= 2 && lcp_pending[t & 1] && cudaStreamWaitEvent(st, ss->ev_lcp[t & 1], 0) != cudaSuccess)
            return fail(LCP_ERR_CUDA, "lcp3d_fused_ws: stream wait failed");
        sp.n_begin = (int64_t)P * hw;
        sp.n_end = (int64_t)Pn * hw;
        sp.vecload = vec_ok && (sp.n_begin % 4) == 0;
        const int64_t groups = (sp.n_end - sp.n_begin + 3) / 4;
        stats3_kernel<T><<<(unsigned)((groups + kS3T - 1) / kS3T), kS3T, 0, st>>>(sp);
        s = check_launch("lcp3d_fused_ws (statistics)");
        if (s != LCP_OK) return s;
        const int Cn = Pn == D ? D - 1 : std::max(C, Pn - 2);  // cells k need record planes k-1 .. k+2
        lcp_pending[t & 1] = false;
        if (Cn > C) {
            if (cudaEventRecord(ss->ev_stats[t & 1], st) != cudaSuccess ||
                cudaStreamWaitEvent(ss->st, ss->ev_stats[t & 1], 0) != cudaSuccess)
                return fail(LCP_ERR_CUDA, "lcp3d_fused_ws: fork failed");
            lp.k_begin = C;
            lp.k_end = Cn;
            s = out_dtype == LCP_F16 ? lcp3_passes<__half>(lp, iso, K, ss->st) : lcp3_passes<float>(lp, iso, K, ss->st);
            if (s != LCP_OK) return s;
            if (cudaEventRecord(ss->ev_lcp[t & 1], ss->st) != cudaSuccess)
                return fail(LCP_ERR_CUDA, "lcp3d_fused_ws: event record failed");
            lcp_pending[t & 1] = true;
        }
        C = Cn;
        P = Pn;
        ++t;
    }
    // join: the caller's stream waits for the last LCP launches
    for (int q = 0; q < 2; ++q)
        if (lcp_pending[q] && cudaStreamWaitEvent(st, ss->ev_lcp[q], 0) != cudaSuccess)
            return fail(LCP_ERR_CUDA, "lcp3d_fused_ws: join failed");
    return LCP_OK;
}

inline lcp_status check_volume(const char* fn, int D, int H, int W) {
    if (D < 2 || H < 2 || W < 2) return fail(LCP_ERR_ARG, "%s: need D, H, W >= 2", fn);
    if ((int64_t)(H - 1 + kL3R - 1) / kL3R > 65535 || (int64_t)(D - 1 + kL3Z - 1) / kL3Z > 65535)
        return fail(LCP_ERR_UNSUPPORTED, "%s: grid too large", fn);
    return LCP_OK;
}

}  // namespace
}  // namespace lcp

using namespace lcp;

extern "C" size_t lcp3d_workspace_bytes(int M, int D, int H, int W, lcp_dtype in_dtype) {
    (void)M;
    (void)in_dtype;
    if (D < 2 || H < 2 || W < 2) return 0;
    return ring_for(D, H, W).bytes;
}

extern "C" lcp_status lcp3d_fused_ws(const void* u, const void* v, const void* w, lcp_dtype in_dtype, int M, int D,
                                     int H, int W, int64_t member_stride, int ddof, double dx, double dy, double dz,
                                     const float* iso, int K, void* lcp_out, lcp_dtype out_dtype, uint32_t* mask,
                                     void* workspace, size_t workspace_bytes, lcp_stream_t stream) {
    static const char* fn = "lcp3d_fused_ws";
    if (!u || !v || !w) return fail(LCP_ERR_ARG, "%s: u, v and w must be non-NULL", fn);
    if (in_dtype != LCP_F32 && in_dtype != LCP_BF16) return fail(LCP_ERR_ARG, "%s: member dtype must be F32 or BF16", fn);
    lcp_status s = check_volume(fn, D, H, W);
    if (s != LCP_OK) return s;
    if (M < 1 || ddof < 0 || ddof > 1 || M - ddof < 1) return fail(LCP_ERR_ARG, "%s: need M >= 1, ddof in {0, 1}, M - ddof >= 1", fn);
    const int64_t vol = (int64_t)D * H * W;
    if (M > 1 && member_stride < vol) return fail(LCP_ERR_ARG, "%s: member_stride must be >= D*H*W", fn);
    if ((s = check_iso(fn, iso, K)) != LCP_OK) return s;
    if ((s = check_spacing(fn, dx, dy)) != LCP_OK) return s;
    if (!(dz > 0.0) || !std::isfinite(dz)) return fail(LCP_ERR_ARG, "%s: dz must be positive and finite", fn);
    if (!lcp_out) return fail(LCP_ERR_ARG, "%s: NULL output", fn);
    if (out_dtype != LCP_F32 && out_dtype != LCP_F16) return fail(LCP_ERR_ARG, "%s: out dtype must be F32 or F16", fn);
    if ((uintptr_t)mask & 3) return fail(LCP_ERR_ARG, "%s: mask must be 4-byte aligned", fn);
    if (!workspace || ((uintptr_t)workspace & 255)) return fail(LCP_ERR_ARG, "%s: need a 256-byte aligned workspace", fn);
    const Ring rg = ring_for(D, H, W);
    if (workspace_bytes < rg.bytes) return fail(LCP_ERR_ARG, "%s: workspace too small (%zu < %zu bytes)", fn, workspace_bytes, rg.bytes);
    const int64_t stride = M > 1 ? member_stride : vol;
    const size_t align = in_dtype == LCP_F32 ? 16 : 8;
    const bool vec_ok = ((uintptr_t)u % align) == 0 && ((uintptr_t)v % align) == 0 && ((uintptr_t)w % align) == 0 &&
                        stride % 4 == 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (in_dtype == LCP_F32)
        return run3<float>(u, v, w, M, D, H, W, stride, ddof, dx, dy, dz, iso, K, lcp_out, out_dtype, mask, workspace,
                           vec_ok, st);
    return run3<__nv_bfloat16>(u, v, w, M, D, H, W, stride, ddof, dx, dy, dz, iso, K, lcp_out, out_dtype, mask,
                               workspace, vec_ok, st);
}

extern "C" lcp_status lcp3d_divergence(const float* mu_u, const float* var_u, const float* mu_v, const float* var_v,
                                       const float* mu_w, const float* var_w, int D, int H, int W, double dx, double dy,
                                       double dz, float* mu_d, float* var_d, lcp_stream_t stream) {
    static const char* fn = "lcp3d_divergence";
    if (!mu_u || !var_u || !mu_v || !var_v || !mu_w || !var_w || !mu_d || !var_d)
        return fail(LCP_ERR_ARG, "%s: NULL pointer", fn);
    lcp_status s = check_volume(fn, D, H, W);
    if (s != LCP_OK) return s;
    if ((s = check_spacing(fn, dx, dy)) != LCP_OK) return s;
    if (!(dz > 0.0) || !std::isfinite(dz)) return fail(LCP_ERR_ARG, "%s: dz must be positive and finite", fn);
    const int64_t n = (int64_t)D * H * W;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16);
    div3_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(mu_u, var_u, mu_v, var_v, mu_w, var_w, D, H, W,
                                                        (float)(1.0 / dx), (float)(0.5 / dx), (float)(1.0 / dy),
                                                        (float)(0.5 / dy), (float)(1.0 / dz), (float)(0.5 / dz), mu_d,
                                                        var_d);
    return check_launch(fn);
}

extern "C" lcp_status lcp3d_map(const float* mu_d, const float* var_d, int D, int H, int W, const float* iso, int K,
                                void* lcp_out, lcp_dtype out_dtype, uint32_t* mask, lcp_stream_t stream) {
    static const char* fn = "lcp3d_map";
    if (!mu_d || !var_d || !lcp_out) return fail(LCP_ERR_ARG, "%s: NULL pointer", fn);
    lcp_status s = check_volume(fn, D, H, W);
    if (s != LCP_OK) return s;
    if ((s = check_iso(fn, iso, K)) != LCP_OK) return s;
    if (K > kMaxIsoPerLaunch) return fail(LCP_ERR_UNSUPPORTED, "%s: K <= %d", fn, kMaxIsoPerLaunch);
    if (out_dtype != LCP_F32 && out_dtype != LCP_F16) return fail(LCP_ERR_ARG, "%s: out dtype must be F32 or F16", fn);
    if ((uintptr_t)mask & 3) return fail(LCP_ERR_ARG, "%s: mask must be 4-byte aligned", fn);
    IsoParams ip;
    ip.K = K;
    for (int k = 0; k < K; ++k) ip.c[k] = iso[k];
    const int n_words = (W - 1 + 31) / 32;
    const int64_t n = (int64_t)(D - 1) * (H - 1) * n_words * 32;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16);
    cudaStream_t st = (cudaStream_t)stream;
    if (out_dtype == LCP_F16)
        map3_kernel<__half><<<grid, 256, 0, st>>>(mu_d, var_d, D, H, W, ip, (__half*)lcp_out, mask, n_words);
    else
        map3_kernel<float><<<grid, 256, 0, st>>>(mu_d, var_d, D, H, W, ip, (float*)lcp_out, mask, n_words);
    return check_launch(fn);
}
