// Learned surrogate: moments of the members, cumulants of the vertex
// divergence under the empirical model, per-cell features, and a
// 17 -> 64 -> 64 -> 1 network trained and evaluated on the tensor cores
// (mma.sync m16n8k16, BF16 operands, FP32 accumulation).
//
// Register layouts of mma.sync.m16n8k16 (gid = lane / 4, tig = lane % 4):
//   A (16 x 16, row-major):  a0 = A[gid][2 tig .. +1],     a1 = A[gid+8][2 tig ..],
//                            a2 = A[gid][8 + 2 tig ..],    a3 = A[gid+8][8 + 2 tig ..]
//   B (16 x 8, k x n):       b0 = B[2 tig .. +1][gid],     b1 = B[8 + 2 tig .. +1][gid]
//   C (16 x 8, fp32):        c0, c1 = C[gid][2 tig .. +1], c2, c3 = C[gid+8][2 tig .. +1]
// so the C fragments of two adjacent 8-column tiles are exactly the A fragment
// of the next layer's 16-wide k-step (no shared-memory round trip between
// layers).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstddef>
#include <mutex>

#include "lcp_common.cuh"

namespace lcp {
namespace {

constexpr int kHid = 64;
constexpr int kFS = LCP_MLP_FEAT_STRIDE;  // 32 bf16 per feature row
constexpr int kOffW1 = 0, kOffB1 = 2048, kOffW2 = 2112, kOffB2 = 6208, kOffW3 = 6272, kOffB3 = 6336;
constexpr int kW1S = 40;  // shared-memory row strides (bf16) chosen so that fragment loads hit 32 banks
constexpr int kW2S = 72;

// ---- 1. moments ---------------------------------------------------------------
// Shifted power sums about member 0, then the central moments by the binomial
// expansion: with delta = S1/M and e_p = S_p/M,
//   m2 = e2 - delta^2,  m3 = e3 - 3 delta e2 + 2 delta^3,
//   m4 = e4 - 4 delta e3 + 6 delta^2 e2 - 3 delta^4.
template <typename T, int VEC>
__global__ void __launch_bounds__(256) moments_kernel(const T* __restrict__ u, const T* __restrict__ v, int M,
                                                     int64_t stride, int64_t n_vert, int vec_ok, float4* mom) {
    using L = Loader<T, VEC>;
    const float fm = (float)M;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g * VEC < n_vert;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n0 = g * VEC;
        const int cnt = (int)min((int64_t)VEC, n_vert - n0);
        const bool vec = vec_ok && cnt == VEC;
        for (int comp = 0; comp < 2; ++comp) {
            const T* x = comp ? v : u;
            float x0[VEC], s[4][VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                x0[e] = 0.f;
                s[0][e] = s[1][e] = s[2][e] = s[3][e] = 0.f;
            }
            if (vec) {
                L::cvt(L::load(x + n0), x0);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (e < cnt) Loader<T, 1>::cvt(Loader<T, 1>::load(x + n0 + e), &x0[e]);
            }
            for (int m = 1; m < M; ++m) {
                float a[VEC];
                if (vec) {
                    L::cvt(L::load(x + (int64_t)m * stride + n0), a);
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        a[e] = 0.f;
                        if (e < cnt) Loader<T, 1>::cvt(Loader<T, 1>::load(x + (int64_t)m * stride + n0 + e), &a[e]);
                    }
                }
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const float d = a[e] - x0[e], d2 = d * d;
                    s[0][e] += d;
                    s[1][e] += d2;
                    s[2][e] = fmaf(d2, d, s[2][e]);
                    s[3][e] = fmaf(d2, d2, s[3][e]);
                }
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                if (e >= cnt) break;
                const float dl = s[0][e] / fm, e2 = s[1][e] / fm, e3 = s[2][e] / fm, e4 = s[3][e] / fm;
                const float dl2 = dl * dl;
                float m2 = e2 - dl2;
                float m3 = e3 - 3.f * dl * e2 + 2.f * dl2 * dl;
                float m4 = e4 - 4.f * dl * e3 + 6.f * dl2 * e2 - 3.f * dl2 * dl2;
                m2 = m2 < 0.f ? 0.f : m2;  // NaN stays NaN
                m4 = m4 < 0.f ? 0.f : m4;
                mom[(int64_t)comp * n_vert + n0 + e] = make_float4(x0[e] + dl, m2, m3, m4);
            }
        }
    }
}

// ---- 2. cumulants of the vertex divergence ------------------------------------
// k_n(D) = a^n k_n(U_hi) + (-a)^n k_n(U_lo) + b^n k_n(V_hi) + (-b)^n k_n(V_lo),
// a = 1/(2 dx) inside and 1/dx on the first/last column (b likewise along y),
// with k1 = mean, k2 = m2, k3 = m3, k4 = m4 - 3 m2^2 of each term.
__device__ __forceinline__ float4 vertex_cumulants(const float4* __restrict__ mu, const float4* __restrict__ mv,
                                                   int H, int W, int j, int i, const Spacing& sp) {
    const int ilo = max(i - 1, 0), ihi = min(i + 1, W - 1), jlo = max(j - 1, 0), jhi = min(j + 1, H - 1);
    const float a = (ihi - ilo == 2) ? sp.sx2 : sp.sx1, b = (jhi - jlo == 2) ? sp.sy2 : sp.sy1;
    const float4 A = __ldg(mu + (int64_t)j * W + ihi), B = __ldg(mu + (int64_t)j * W + ilo);
    const float4 C = __ldg(mv + (int64_t)jhi * W + i), D = __ldg(mv + (int64_t)jlo * W + i);
    const float a2 = a * a, b2 = b * b;
    float4 k;
    k.x = fmaf(a, A.x - B.x, b * (C.x - D.x));
    k.y = fmaf(a2, A.y + B.y, b2 * (C.y + D.y));
    k.z = fmaf(a2 * a, A.z - B.z, b2 * b * (C.z - D.z));
    const float ka = (A.w - 3.f * A.y * A.y) + (B.w - 3.f * B.y * B.y);
    const float kb = (C.w - 3.f * C.y * C.y) + (D.w - 3.f * D.y * D.y);
    k.w = fmaf(a2 * a2, ka, b2 * b2 * kb);
    return k;
}

// Isovalue-independent part of a cell's features.
struct CellPart {
    float mu[4], sig[4], inv_sig[4], ratio[4], skew[4], kurt[4];
    VertexG g[4];  // the closed form's per-vertex scale (feature 16)
};

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

__device__ __forceinline__ CellPart cell_part(const float4 (&k)[4]) {
    CellPart p;
    float msum = 0.f;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        p.mu[v] = k[v].x;
        const float var = fmaxf(k[v].y, 0.f);
        p.sig[v] = sqrtf(var);
        p.inv_sig[v] = p.sig[v] > 0.f ? 1.0f / p.sig[v] : 0.f;
        p.g[v] = vertex_g(k[v].x, var);
        msum += p.sig[v];
    }
    const float mean_sig = 0.25f * msum;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float s = p.sig[v];
        p.ratio[v] = mean_sig > 0.f ? s / mean_sig : 1.f;
        if (s > 0.f) {
            const float s2 = s * s;
            p.skew[v] = clampf(k[v].z / (s2 * s), -5.f, 5.f);
            p.kurt[v] = clampf(k[v].w / (s2 * s2), -2.f, 10.f);
        } else {
            p.skew[v] = 0.f;
            p.kurt[v] = 0.f;
        }
    }
    return p;
}

// The network's prior: the logit of the independent-Gaussian LCP, clamped to
// [1e-6, 1 - 1e-6] (|logit| <= 13.8); the output layer adds it to its own sum.
__device__ __forceinline__ float prior_logit(float g) {
    const float p = fminf(fmaxf(g, 1e-6f), 1.0f - 1e-6f);
    return __logf(p) - __logf(1.0f - p);
}

// The 17 features of (cell, c) as 16 words of bf16 pairs (features 17..31
// zero); returns the prior (fp32).
__device__ __forceinline__ float cell_feature_words(const CellPart& p, float c, uint32_t (&w)[kFS / 2]) {
    float f[kFS];
#pragma unroll
    for (int q = 0; q < kFS; ++q) f[q] = 0.f;
    float pb = 1.f, qb = 1.f;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float d = c - p.mu[v];
        f[4 * v + 0] = p.sig[v] > 0.f ? clampf(d * p.inv_sig[v], -8.f, 8.f) : (d > 0.f ? 8.f : (d < 0.f ? -8.f : 0.f));
        f[4 * v + 1] = p.ratio[v];
        f[4 * v + 2] = p.skew[v];
        f[4 * v + 3] = p.kurt[v];
        float pv, qv;
        below_above(p.g[v], c, pv, qv);
        pb *= pv;
        qb *= qv;
    }
    f[16] = 1.f - pb - qb;
#pragma unroll
    for (int q = 0; q < kFS / 2; ++q) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * q], f[2 * q + 1]);
        w[q] = *reinterpret_cast<const uint32_t*>(&h);
    }
    return prior_logit(f[16]);
}

// The features into a contiguous 32-wide bf16 row (16-byte aligned); returns the prior.
__device__ __forceinline__ float cell_features(const CellPart& p, float c, __nv_bfloat16* row) {
    uint32_t w[kFS / 2];
    const float pr = cell_feature_words(p, c, w);
    uint4* out = reinterpret_cast<uint4*>(row);
#pragma unroll
    for (int q = 0; q < kFS / 8; ++q) out[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    return pr;
}

__global__ void __launch_bounds__(256) features_kernel(const float4* __restrict__ mom, int H, int W, Spacing sp,
                                                      const __grid_constant__ IsoParams iso, __nv_bfloat16* feat,
                                                      float* prior) {
    const int Hc = H - 1, Wc = W - 1;
    const int64_t n_cells = (int64_t)Hc * Wc, n_vert = (int64_t)H * W;
    for (int64_t cidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; cidx < n_cells;
         cidx += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(cidx / Wc), i = (int)(cidx - (int64_t)j * Wc);
        float4 k[4];
        k[0] = vertex_cumulants(mom, mom + n_vert, H, W, j, i, sp);
        k[1] = vertex_cumulants(mom, mom + n_vert, H, W, j, i + 1, sp);
        k[2] = vertex_cumulants(mom, mom + n_vert, H, W, j + 1, i, sp);
        k[3] = vertex_cumulants(mom, mom + n_vert, H, W, j + 1, i + 1, sp);
        const CellPart p = cell_part(k);
        for (int q = 0; q < iso.K; ++q) {
            const int64_t r = (int64_t)q * n_cells + cidx;
            const float pr = cell_features(p, iso.c[q], feat + r * kFS);
            if (prior) prior[r] = pr;
        }
    }
}

// ---- 3. tensor-core building blocks -------------------------------------------
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Four 8x8 bf16 matrices; lane l supplies the row address of matrix l / 8.
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack_bf16(uint32_t w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
}
__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sigmoid(float z) { return 1.0f / (1.0f + __expf(-z)); }

// Network weights in shared memory, BF16 operands and FP32 vectors.
struct NetSmem {
    __align__(16) __nv_bfloat16 W1[kHid * kW1S];  // [n][k]
    __align__(16) __nv_bfloat16 W2[kHid * kW2S];  // [n][k]
    __align__(16) float b1[kHid];
    float b2[kHid], w3[kHid];
    float b3;
};

__device__ void load_net(const float* __restrict__ prm, NetSmem& s, __nv_bfloat16* W2t /* [k][n], or null */) {
    for (int q = threadIdx.x; q < kHid * kFS; q += blockDim.x) {
        const int n = q / kFS, k = q - n * kFS;
        s.W1[n * kW1S + k] = __float2bfloat16_rn(k < 17 ? prm[kOffW1 + q] : 0.f);
    }
    for (int q = threadIdx.x; q < kHid * kHid; q += blockDim.x) {
        const int n = q >> 6, k = q & 63;
        const __nv_bfloat16 w = __float2bfloat16_rn(prm[kOffW2 + q]);
        s.W2[n * kW2S + k] = w;
        if (W2t) W2t[k * kW2S + n] = w;
    }
    for (int q = threadIdx.x; q < kHid; q += blockDim.x) {
        s.b1[q] = prm[kOffB1 + q];
        s.b2[q] = prm[kOffB2 + q];
        s.w3[q] = prm[kOffW3 + q];
    }
    if (threadIdx.x == 0) s.b3 = prm[kOffB3];
}

// One warp, 16 rows: layers 1 and 2 from the A fragments of the input (two
// 16-feature k-steps).  Leaves h1 as bf16 A fragments (four 16-unit k-steps)
// and h2 in C-fragment layout (fp32).
__device__ __forceinline__ void forward16(const NetSmem& s, const uint32_t (&x)[2][4], uint32_t (&h1)[4][4],
                                          float (&h2)[8][4], int gid, int tig) {
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float bl = s.b1[8 * nt + 2 * tig], bh = s.b1[8 * nt + 2 * tig + 1];
        acc[nt][0] = bl; acc[nt][1] = bh; acc[nt][2] = bl; acc[nt][3] = bh;
    }
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const __nv_bfloat16* w = s.W1 + (8 * nt + gid) * kW1S + 16 * ks + 2 * tig;
            mma16816(acc[nt], x[ks], *reinterpret_cast<const uint32_t*>(w), *reinterpret_cast<const uint32_t*>(w + 8));
        }
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        const int a = 2 * ks, b = 2 * ks + 1;
        h1[ks][0] = pack_bf16(tanh_fast(acc[a][0]), tanh_fast(acc[a][1]));
        h1[ks][1] = pack_bf16(tanh_fast(acc[a][2]), tanh_fast(acc[a][3]));
        h1[ks][2] = pack_bf16(tanh_fast(acc[b][0]), tanh_fast(acc[b][1]));
        h1[ks][3] = pack_bf16(tanh_fast(acc[b][2]), tanh_fast(acc[b][3]));
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float bl = s.b2[8 * nt + 2 * tig], bh = s.b2[8 * nt + 2 * tig + 1];
        h2[nt][0] = bl; h2[nt][1] = bh; h2[nt][2] = bl; h2[nt][3] = bh;
    }
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const __nv_bfloat16* w = s.W2 + (8 * nt + gid) * kW2S + 16 * ks + 2 * tig;
            mma16816(h2[nt], h1[ks], *reinterpret_cast<const uint32_t*>(w), *reinterpret_cast<const uint32_t*>(w + 8));
        }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) h2[nt][e] = tanh_fast(h2[nt][e]);
}

// Output pre-activation of rows gid and gid + 8 (complete in all four lanes of the group).
__device__ __forceinline__ float2 output16(const NetSmem& s, const float (&h2)[8][4], int tig) {
    float lo = 0.f, hi = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float w0 = s.w3[8 * nt + 2 * tig], w1 = s.w3[8 * nt + 2 * tig + 1];
        lo = fmaf(h2[nt][0], w0, fmaf(h2[nt][1], w1, lo));
        hi = fmaf(h2[nt][2], w0, fmaf(h2[nt][3], w1, hi));
    }
    lo += __shfl_xor_sync(0xFFFFFFFFu, lo, 1);
    hi += __shfl_xor_sync(0xFFFFFFFFu, hi, 1);
    lo += __shfl_xor_sync(0xFFFFFFFFu, lo, 2);
    hi += __shfl_xor_sync(0xFFFFFFFFu, hi, 2);
    return make_float2(lo + s.b3, hi + s.b3);
}

// A fragments of a 16-row x 32-feature tile held row-major in shared memory
// (row stride kW1S bf16): matrices (rows 0-7 | 8-15) x (k 0-7 | 8-15) per k-step.
__device__ __forceinline__ void load_x_frags(const __nv_bfloat16* tile, uint32_t (&x)[2][4], int lane) {
    const int r = (lane & 7) + ((lane >> 3) & 1) * 8, c = (lane >> 4) * 8;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) ldsm_x4(x[ks], tile + r * kW1S + 16 * ks + c);
}

// ---- 4. forward over feature rows ---------------------------------------------
constexpr int kMT = 128;  // threads per CTA of the network kernels (4 warps)

__global__ void __launch_bounds__(kMT) mlp_forward_kernel(const float* __restrict__ prm,
                                                         const __nv_bfloat16* __restrict__ feat,
                                                         const float* __restrict__ prior, int64_t n,
                                                         float* __restrict__ y) {
    __shared__ NetSmem s;
    __shared__ __align__(16) __nv_bfloat16 xs[kMT / 32][16 * kW1S];
    load_net(prm, s, nullptr);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gid = lane >> 2, tig = lane & 3;
    __nv_bfloat16* tile = xs[warp];
    for (int64_t r0 = ((int64_t)blockIdx.x * (kMT / 32) + warp) * 16; r0 < n;
         r0 += (int64_t)gridDim.x * (kMT / 32) * 16) {
        // stage 16 rows (64 B each): lane covers half a row
        {
            const int r = lane >> 1, h = lane & 1;
            uint4 a = make_uint4(0, 0, 0, 0), b = a;
            if (r0 + r < n) {
                const uint4* src = reinterpret_cast<const uint4*>(feat + (r0 + r) * kFS) + 2 * h;
                a = __ldg(src);
                b = __ldg(src + 1);
            }
            uint4* dst = reinterpret_cast<uint4*>(tile + r * kW1S + 16 * h);
            dst[0] = a;
            dst[1] = b;
        }
        __syncwarp();
        uint32_t x[2][4], h1[4][4];
        float h2[8][4];
        load_x_frags(tile, x, lane);
        forward16(s, x, h1, h2, gid, tig);
        const float2 z = output16(s, h2, tig);
        if (tig == 0) {
            if (r0 + gid < n) y[r0 + gid] = sigmoid(z.x + (prior ? __ldg(prior + r0 + gid) : 0.f));
            if (r0 + gid + 8 < n) y[r0 + gid + 8] = sigmoid(z.y + (prior ? __ldg(prior + r0 + gid + 8) : 0.f));
        }
        __syncwarp();
    }
}

// ---- 5. fused inference from moments ------------------------------------------
// CTA: 4 cell rows x 32 cell columns, one warp per cell row, one lane per cell.
// The cumulants of the tile's 5 x 33 vertices are computed once into shared
// memory; per isovalue each lane writes its cell's feature row, and the warp
// evaluates its 32 rows as two 16-row tensor-core tiles.
constexpr int kIR = 4, kIC = 32;

template <typename OutT>
__global__ void __launch_bounds__(kMT) mlp_infer_kernel(const float4* __restrict__ mom, int H, int W, Spacing sp,
                                                       const __grid_constant__ IsoParams iso,
                                                       const float* __restrict__ prm, OutT* __restrict__ out) {
    __shared__ NetSmem s;
    __shared__ float4 kap[(kIR + 1) * (kIC + 1)];
    __shared__ __align__(16) __nv_bfloat16 xs[kMT / 32][32 * kW1S];
    load_net(prm, s, nullptr);
    const int Hc = H - 1, Wc = W - 1;
    const int a = blockIdx.y * kIR, c0 = blockIdx.x * kIC;
    const int64_t n_vert = (int64_t)H * W;
    for (int q = threadIdx.x; q < (kIR + 1) * (kIC + 1); q += blockDim.x) {
        const int rr = q / (kIC + 1), cc = q - rr * (kIC + 1);
        const int j = min(a + rr, H - 1), i = min(c0 + cc, W - 1);
        kap[q] = vertex_cumulants(mom, mom + n_vert, H, W, j, i, sp);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gid = lane >> 2, tig = lane & 3;
    const int j = a + warp, i = c0 + lane;
    const bool ok = j < Hc && i < Wc;
    float4 k4[4];
    k4[0] = kap[warp * (kIC + 1) + lane];
    k4[1] = kap[warp * (kIC + 1) + lane + 1];
    k4[2] = kap[(warp + 1) * (kIC + 1) + lane];
    k4[3] = kap[(warp + 1) * (kIC + 1) + lane + 1];
    const CellPart part = cell_part(k4);
    __nv_bfloat16* tile = xs[warp];
    const int64_t plane = (int64_t)Hc * Wc;
    for (int q = 0; q < iso.K; ++q) {
        const float pr = cell_features(part, iso.c[q], tile + lane * kW1S);
        __syncwarp();
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            uint32_t x[2][4], h1[4][4];
            float h2[8][4];
            load_x_frags(tile + 16 * mt * kW1S, x, lane);
            forward16(s, x, h1, h2, gid, tig);
            const float2 z = output16(s, h2, tig);
            const float plo = __shfl_sync(0xFFFFFFFFu, pr, 16 * mt + gid);
            const float phi = __shfl_sync(0xFFFFFFFFu, pr, 16 * mt + gid + 8);
            if (tig == 0 && j < Hc) {
                const int i0 = c0 + 16 * mt + gid;
                OutT* o = out + (int64_t)q * plane + (int64_t)j * Wc;
                if (i0 < Wc) o[i0] = to_out<OutT>(sigmoid(z.x + plo));
                if (i0 + 8 < Wc) o[i0 + 8] = to_out<OutT>(sigmoid(z.y + phi));
            }
        }
        __syncwarp();
    }
    (void)ok;
}

// ---- 5b. fused inference on the 5th-generation tensor cores (tcgen05) ---------
// Per CTA a block of 4 x 32 cells, as above; per isovalue its 128 feature rows
// form one M = 128 tile.  Each thread owns one row (= one TMEM lane): it writes
// the row's features into shared memory in the canonical K-major layout
// (8-row x 16-byte core matrices), one elected thread issues the layer's
// tcgen05.mma (K = 16 per instruction, FP32 accumulators in TMEM, operands
// read through shared-memory descriptors) and commits to an mbarrier, and each
// thread reads its row of the accumulators back with tcgen05.ld for the
// epilogue (bias, tanh, the next layer's operand, and finally the output dot
// product, prior and sigmoid).
//
// Shared-memory descriptor (64 bits): start address >> 4 in bits 0-13, leading
// (K-direction) byte offset between core matrices >> 4 in bits 16-29, stride
// (M/N-direction) byte offset between 8-row groups >> 4 in bits 32-45, the
// descriptor version 1 in bits 46-47, no swizzle (bits 61-63 = 0).
// Instruction descriptor (32 bits, kind::f16): D format F32 (bits 4-5 = 1), A
// and B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kTmemCols = 64;  // D1, then D2 (D1 is read out before layer 2 is issued)
constexpr long long kTcWaitBudget = 2000000000ll;  // clock cycles (~1 s) before an mbarrier wait gives up
__device__ uint32_t g_sur_status = 0;

struct TcSmem {
    __align__(1024) __nv_bfloat16 W1[kHid * kFS];  // B operand of layer 1: N = 64 units x K = 32 features
    __align__(1024) __nv_bfloat16 W2[kHid * kHid];  // B operand of layer 2: N = 64 x K = 64

    // A operands: layer 1 (128 rows x 32 features, the first 8 KB) and then layer 2
    // (128 rows x 64 units) in the same bytes: h1 is written after layer 1's
    // MMAs have completed, the next features after layer 2's
    __align__(1024) __nv_bfloat16 A[128 * kHid];
    float4 kap[(kIR + 1) * (kIC + 1)];
    float b1[kHid], b2[kHid], w3[kHid];
    __align__(8) uint64_t mbar;
    uint32_t tmem;
    int abort_flag;  // set when an mbarrier wait gave up; read by all threads after a barrier
};

// Byte offset of element (row, k) in a K-major canonical tile with `kg` core
// matrices along K: core matrix (row / 8, k / 8) at ((row / 8) kg + k / 8) 128.
__host__ __device__ constexpr uint32_t canon_off(int row, int k, int kg) {
    return (uint32_t)(((row >> 3) * kg + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

constexpr uint32_t kIdescM128N64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdescM128N64), "r"(accumulate));
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded wait for the mbarrier phase `parity`; false (and the status bit) when
// it gives up.  The clock is read every 64 tries.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    const long long t0 = clock64();
    for (int it = 1;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 0 && clock64() - t0 > kTcWaitBudget) {
            atomicOr(&g_sur_status, 1u);
            return false;
        }
    }
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ uint32_t tanh_bf16x2(float lo, float hi) {
    uint32_t x = pack_bf16(lo, hi), y;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}

constexpr int kTcCtasPerSm = 5;

template <typename OutT>
__global__ void __launch_bounds__(kMT, kTcCtasPerSm) mlp_infer_tc_kernel(const float4* __restrict__ mom, int H, int W, Spacing sp,
                                                             const __grid_constant__ IsoParams iso,
                                                             const float* __restrict__ prm, OutT* __restrict__ out) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    // the dynamic window starts 16-byte aligned; round it up to 1024 for the tiles
    TcSmem& S = *reinterpret_cast<TcSmem*>(tc_raw + ((1024 - (smem_addr(tc_raw) & 1023)) & 1023));
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // weights into the canonical layouts (bf16), vectors as fp32
    for (int q = t; q < kHid * kFS; q += kMT) {
        const int n = q / kFS, k = q - n * kFS;
        *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(S.W1) + canon_off(n, k, kFS / 8)) =
            __float2bfloat16_rn(k < 17 ? prm[kOffW1 + q] : 0.f);
    }
    for (int q = t; q < kHid * kHid; q += kMT) {
        const int n = q >> 6, k = q & 63;
        *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(S.W2) + canon_off(n, k, kHid / 8)) =
            __float2bfloat16_rn(prm[kOffW2 + q]);
    }
    for (int q = t; q < kHid; q += kMT) {
        S.b1[q] = prm[kOffB1 + q];
        S.b2[q] = prm[kOffB2 + q];
        S.w3[q] = prm[kOffW3 + q];
    }
    if (t == 0) {
        S.abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {  // TMEM: 64 FP32 columns x 128 lanes, the accumulator of either layer
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&S.tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const int Hc = H - 1, Wc = W - 1;
    const int64_t n_vert = (int64_t)H * W;
    const uint32_t mbar = smem_addr(&S.mbar);
    const uint32_t a0 = smem_addr(S.A), a1 = a0, w1 = smem_addr(S.W1), w2 = smem_addr(S.W2);
    const float b3 = prm[kOffB3];
    const int64_t plane = (int64_t)Hc * Wc;
    const int nbx = (Wc + kIC - 1) / kIC, nblocks = nbx * ((Hc + kIR - 1) / kIR);
    uint32_t phase = 0;
    volatile int* abort_flag = &S.abort_flag;
    tc_fence_before();
    __syncthreads();  // TMEM address, mbarrier and weights are ready
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    // persistent: the CTA walks cell blocks of 4 x 32 cells
    for (int blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
        const int a = (blk / nbx) * kIR, c0 = (blk % nbx) * kIC;
        for (int q = t; q < (kIR + 1) * (kIC + 1); q += kMT) {
            const int rr = q / (kIC + 1), cc = q - rr * (kIC + 1);
            S.kap[q] = vertex_cumulants(mom, mom + n_vert, H, W, min(a + rr, H - 1), min(c0 + cc, W - 1), sp);
        }
        __syncthreads();
        const int j = a + warp, i = c0 + lane;
        float4 k4[4];
        k4[0] = S.kap[warp * (kIC + 1) + lane];
        k4[1] = S.kap[warp * (kIC + 1) + lane + 1];
        k4[2] = S.kap[(warp + 1) * (kIC + 1) + lane];
        k4[3] = S.kap[(warp + 1) * (kIC + 1) + lane + 1];
        const CellPart part = cell_part(k4);
        for (int q = 0; q < iso.K; ++q) {
            // features of row t into A0
            uint32_t fw[kFS / 2];
            const float pr = cell_feature_words(part, iso.c[q], fw);
#pragma unroll
            for (int g = 0; g < kFS / 8; ++g)
                *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(S.A) + canon_off(t, 8 * g, kFS / 8)) =
                    make_uint4(fw[4 * g], fw[4 * g + 1], fw[4 * g + 2], fw[4 * g + 3]);
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (*abort_flag) break;  // uniform: read after the barrier, written only before one
            if (t == 0) {  // layer 1: D1 = A0 W1^T (K = 32 in two steps)
#pragma unroll
                for (int s = 0; s < 2; ++s)
                    tc_mma(tmem, smem_desc(a0 + 256 * s, 128, 512), smem_desc(w1 + 256 * s, 128, 512), s);
                tc_commit(mbar);
            }
            if (!mbar_wait(mbar, phase)) *abort_flag = 1;
            phase ^= 1u;
            tc_fence_after();
            // h1 = tanh(D1 + b1) as bf16 into A1
#pragma unroll
            for (int cg = 0; cg < 4; ++cg) {
                float z[16];
                tmem_ld16(lane_base + 16 * cg, z);
                uint32_t hw[8];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    hw[e] = tanh_bf16x2(z[2 * e] + S.b1[16 * cg + 2 * e], z[2 * e + 1] + S.b1[16 * cg + 2 * e + 1]);
                *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(S.A) + canon_off(t, 16 * cg, kHid / 8)) =
                    make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(S.A) + canon_off(t, 16 * cg + 8, kHid / 8)) =
                    make_uint4(hw[4], hw[5], hw[6], hw[7]);
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (*abort_flag) break;
            if (t == 0) {  // layer 2: D2 = A1 W2^T (K = 64 in four steps)
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    tc_mma(tmem, smem_desc(a1 + 256 * s, 128, 1024), smem_desc(w2 + 256 * s, 128, 1024), s);
                tc_commit(mbar);
            }
            if (!mbar_wait(mbar, phase)) *abort_flag = 1;
            phase ^= 1u;
            tc_fence_after();
            // output: b3 + prior + w3 . tanh(D2), the tanh two units at a time (bf16x2), the dot product in fp32
            float z3 = b3 + pr;
#pragma unroll
            for (int cg = 0; cg < 4; ++cg) {
                float z[16];
                tmem_ld16(lane_base + 16 * cg, z);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float2 h = unpack_bf16(
                        tanh_bf16x2(z[2 * e] + S.b2[16 * cg + 2 * e], z[2 * e + 1] + S.b2[16 * cg + 2 * e + 1]));
                    z3 = fmaf(h.x, S.w3[16 * cg + 2 * e], fmaf(h.y, S.w3[16 * cg + 2 * e + 1], z3));
                }
            }
            if (j < Hc && i < Wc) out[(int64_t)q * plane + (int64_t)j * Wc + i] = to_out<OutT>(sigmoid(z3));
            tc_fence_before();  // this iteration's TMEM reads are ordered before the next MMA
        }
        __syncthreads();  // every thread is done with this block's cumulants, and the flag is settled
        if (*abort_flag) break;  // uniform: read after the barrier
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

constexpr size_t kTcSmemBytes = sizeof(TcSmem) + 1024;

// ---- 6. backward: gradient of the mean squared error ---------------------------
// Per iteration a CTA takes 64 rows (16 per warp).  Each warp runs the forward
// pass, the output and hidden-layer deltas (dA1 = dZ2 W2^T on the tensor cores,
// dZ2 in registers as its A fragments), and stages X, h1, dZ1, dZ2 (bf16) in
// shared memory; the CTA then accumulates the weight gradients
// dW2 = dZ2^T h1 and dW1 = dZ1^T X as contractions over the 64 rows
// (ldmatrix .trans supplies the transposed operands), in registers across
// iterations, and adds them to the output once at the end.
struct BwdSmem {
    NetSmem net;
    __align__(16) __nv_bfloat16 W2t[kHid * kW2S];  // [k][n] = W2[n][k]
    __align__(16) __nv_bfloat16 xs[64 * kW1S];
    __align__(16) __nv_bfloat16 h1s[64 * kW2S];
    __align__(16) __nv_bfloat16 d1s[64 * kW2S];
    __align__(16) __nv_bfloat16 d2s[64 * kW2S];
    // per-warp partial sums (each written by one warp only, summed in warp order at the end), so the
    // block's result does not depend on the order in which its warps run
    __align__(16) float db1[kMT / 32][kHid];
    float db2[kMT / 32][kHid], dw3[kMT / 32][kHid];
    float db3[kMT / 32], loss[kMT / 32];
};

static_assert(offsetof(BwdSmem, xs) % 16 == 0 && offsetof(BwdSmem, h1s) % 16 == 0 &&
                  offsetof(BwdSmem, d1s) % 16 == 0 && offsetof(BwdSmem, d2s) % 16 == 0,
              "ldmatrix rows must be 16-byte aligned");
static_assert((kW1S * 2) % 16 == 0 && (kW2S * 2) % 16 == 0, "row strides must keep 16-byte alignment");

__device__ __forceinline__ void st_pair(__nv_bfloat16* base, int row, int col, int stride, uint32_t w) {
    *reinterpret_cast<uint32_t*>(base + row * stride + col) = w;
}

// Column sums over the 8 row groups of a warp (lanes with equal tig).
__device__ __forceinline__ float sum_over_gid(float x) {
    x += __shfl_xor_sync(0xFFFFFFFFu, x, 4);
    x += __shfl_xor_sync(0xFFFFFFFFu, x, 8);
    x += __shfl_xor_sync(0xFFFFFFFFu, x, 16);
    return x;
}

// One CTA's gradient sums go either straight into grad (atomic adds, scaled by
// 1/n) or, for the deterministic variant, unscaled into its own row `part` of
// [gridDim.x][kPartStride] floats (every entry written), which
// bwd_reduce_kernel then sums over the CTAs in CTA order.
constexpr int kPartStride = LCP_MLP_NPARAMS + 4;  // the parameters, then the loss (16-byte rows)

template <bool DET>
__global__ void __launch_bounds__(kMT) mlp_backward_kernel(const float* __restrict__ prm,
                                                          const __nv_bfloat16* __restrict__ feat,
                                                          const float* __restrict__ prior,
                                                          const float* __restrict__ target, int64_t n,
                                                          float* __restrict__ grad, float* __restrict__ loss,
                                                          float* __restrict__ parts) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem& S = *reinterpret_cast<BwdSmem*>(smem_raw);
    load_net(prm, S.net, S.W2t);
    for (int q = threadIdx.x; q < (kMT / 32) * kHid; q += blockDim.x) {
        (&S.db1[0][0])[q] = 0.f;
        (&S.db2[0][0])[q] = 0.f;
        (&S.dw3[0][0])[q] = 0.f;
    }
    if (threadIdx.x < kMT / 32) S.db3[threadIdx.x] = S.loss[threadIdx.x] = 0.f;
    __syncthreads();
    const NetSmem& s = S.net;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gid = lane >> 2, tig = lane & 3;
    const float inv_n = 1.0f / (float)n;
    float gW2[8][4], gW1[4][4];
#pragma unroll
    for (int a = 0; a < 8; ++a) gW2[a][0] = gW2[a][1] = gW2[a][2] = gW2[a][3] = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) gW1[a][0] = gW1[a][1] = gW1[a][2] = gW1[a][3] = 0.f;
    const int rw = 16 * warp;  // this warp's rows inside the staged 64

    for (int64_t base = (int64_t)blockIdx.x * 64; base < n; base += (int64_t)gridDim.x * 64) {
        const int64_t r0 = base + rw;
        {  // stage X
            const int r = lane >> 1, h = lane & 1;
            uint4 a = make_uint4(0, 0, 0, 0), b = a;
            if (r0 + r < n) {
                const uint4* src = reinterpret_cast<const uint4*>(feat + (r0 + r) * kFS) + 2 * h;
                a = __ldg(src);
                b = __ldg(src + 1);
            }
            uint4* dst = reinterpret_cast<uint4*>(S.xs + (rw + r) * kW1S + 16 * h);
            dst[0] = a;
            dst[1] = b;
        }
        __syncwarp();
        uint32_t x[2][4], h1[4][4];
        float h2[8][4];
        load_x_frags(S.xs + rw * kW1S, x, lane);
        forward16(s, x, h1, h2, gid, tig);
        const float2 z = output16(s, h2, tig);
        const bool vlo = r0 + gid < n, vhi = r0 + gid + 8 < n;
        const float plo = (prior && vlo) ? __ldg(prior + r0 + gid) : 0.f;
        const float phi = (prior && vhi) ? __ldg(prior + r0 + gid + 8) : 0.f;
        const float ylo = sigmoid(z.x + plo), yhi = sigmoid(z.y + phi);
        const float tlo = vlo ? __ldg(target + r0 + gid) : 0.f, thi = vhi ? __ldg(target + r0 + gid + 8) : 0.f;
        // d(sum of squared errors)/dz3 = 2 (y - t) y (1 - y); the 1/n of the mean is applied once at the end
        const float dlo = vlo ? 2.f * (ylo - tlo) * ylo * (1.f - ylo) : 0.f;
        const float dhi = vhi ? 2.f * (yhi - thi) * yhi * (1.f - yhi) : 0.f;
        {  // the warp's sums over its 16 rows (each row once: the lanes with tig == 0), fixed order
            const float e = tig == 0 ? (vlo ? (ylo - tlo) * (ylo - tlo) : 0.f) + (vhi ? (yhi - thi) * (yhi - thi) : 0.f)
                                     : 0.f;
            const float dd = tig == 0 ? dlo + dhi : 0.f;
            const float es = sum_over_gid(e), ds = sum_over_gid(dd);
            if (lane == 0) {
                S.loss[warp] += es;
                S.db3[warp] += ds;
            }
        }
        // stage h1 (its A fragments are C fragments of 8-column tiles 2ks, 2ks+1)
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            st_pair(S.h1s, rw + gid, 16 * ks + 2 * tig, kW2S, h1[ks][0]);
            st_pair(S.h1s, rw + gid + 8, 16 * ks + 2 * tig, kW2S, h1[ks][1]);
            st_pair(S.h1s, rw + gid, 16 * ks + 8 + 2 * tig, kW2S, h1[ks][2]);
            st_pair(S.h1s, rw + gid + 8, 16 * ks + 8 + 2 * tig, kW2S, h1[ks][3]);
        }
        // dZ2 = dz3 w3 (1 - h2^2); dw3 += h2^T dz3; db2 += column sums of dZ2
        uint32_t d2[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float dz[4];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int col = 8 * nt + 2 * tig + e;
                const float w = s.w3[col];
                dz[e] = dlo * w * (1.f - h2[nt][e] * h2[nt][e]);
                dz[2 + e] = dhi * w * (1.f - h2[nt][2 + e] * h2[nt][2 + e]);
                const float gw3 = sum_over_gid(h2[nt][e] * dlo + h2[nt][2 + e] * dhi);
                const float gb2 = sum_over_gid(dz[e] + dz[2 + e]);
                if (gid == 0) {  // one lane per column of this warp
                    S.dw3[warp][col] += gw3;
                    S.db2[warp][col] += gb2;
                }
            }
            const uint32_t lo = pack_bf16(dz[0], dz[1]), hi = pack_bf16(dz[2], dz[3]);
            d2[nt >> 1][(nt & 1) * 2 + 0] = lo;
            d2[nt >> 1][(nt & 1) * 2 + 1] = hi;
            st_pair(S.d2s, rw + gid, 8 * nt + 2 * tig, kW2S, lo);
            st_pair(S.d2s, rw + gid + 8, 8 * nt + 2 * tig, kW2S, hi);
        }
        // dA1 = dZ2 W2^T; B(k = output unit, n = input unit) = W2t[n][k]
        float da[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) da[nt][0] = da[nt][1] = da[nt][2] = da[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const __nv_bfloat16* w = S.W2t + (8 * nt + gid) * kW2S + 16 * ks + 2 * tig;
                mma16816(da[nt], d2[ks], *reinterpret_cast<const uint32_t*>(w),
                         *reinterpret_cast<const uint32_t*>(w + 8));
            }
        // dZ1 = dA1 (1 - h1^2); db1 += column sums
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float2 hl = unpack_bf16(h1[nt >> 1][(nt & 1) * 2 + 0]);
            const float2 hh = unpack_bf16(h1[nt >> 1][(nt & 1) * 2 + 1]);
            const float z0 = da[nt][0] * (1.f - hl.x * hl.x), z1 = da[nt][1] * (1.f - hl.y * hl.y);
            const float z2 = da[nt][2] * (1.f - hh.x * hh.x), z3 = da[nt][3] * (1.f - hh.y * hh.y);
            st_pair(S.d1s, rw + gid, 8 * nt + 2 * tig, kW2S, pack_bf16(z0, z1));
            st_pair(S.d1s, rw + gid + 8, 8 * nt + 2 * tig, kW2S, pack_bf16(z2, z3));
            const float g0 = sum_over_gid(z0 + z2), g1 = sum_over_gid(z1 + z3);
            if (gid == 0) {
                S.db1[warp][8 * nt + 2 * tig] += g0;
                S.db1[warp][8 * nt + 2 * tig + 1] += g1;
            }
        }
        __syncthreads();
        // weight gradients over the 64 staged rows: this warp's 16 output rows
        const int o0 = 16 * warp;
        const int ar = (lane & 7) + ((lane >> 4) & 1) * 8, ac = ((lane >> 3) & 1) * 8;  // A^T operand addressing
        const int br = (lane & 7) + ((lane >> 3) & 1) * 8, bc = (lane >> 4) * 8;        // B operand addressing
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t a2[4], a1[4];
            ldsm_x4_t(a2, S.d2s + (16 * kk + ar) * kW2S + o0 + ac);
            ldsm_x4_t(a1, S.d1s + (16 * kk + ar) * kW2S + o0 + ac);
#pragma unroll
            for (int np = 0; np < 4; ++np) {  // dW2: input units in pairs of 8-column tiles
                uint32_t b[4];
                ldsm_x4_t(b, S.h1s + (16 * kk + br) * kW2S + 16 * np + bc);
                mma16816(gW2[2 * np], a2, b[0], b[1]);
                mma16816(gW2[2 * np + 1], a2, b[2], b[3]);
            }
#pragma unroll
            for (int np = 0; np < 2; ++np) {  // dW1: features 0-15, 16-31
                uint32_t b[4];
                ldsm_x4_t(b, S.xs + (16 * kk + br) * kW1S + 16 * np + bc);
                mma16816(gW1[2 * np], a1, b[0], b[1]);
                mma16816(gW1[2 * np + 1], a1, b[2], b[3]);
            }
        }
        __syncthreads();
    }
    // this CTA's sums: the weight matrices from this warp's registers (its own 16 output rows), the
    // vectors from the per-warp partials in warp order
    float* const row = DET ? parts + (int64_t)blockIdx.x * kPartStride : nullptr;
    auto put = [&](int idx, float val) {
        if (DET) row[idx] = val;
        else atomicAdd(grad + idx, val * inv_n);
    };
    const int o0 = 16 * warp;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int col = 8 * nt + 2 * tig + e;
            put(kOffW2 + (o0 + gid) * kHid + col, gW2[nt][e]);
            put(kOffW2 + (o0 + gid + 8) * kHid + col, gW2[nt][2 + e]);
        }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int col = 8 * nt + 2 * tig + e;
            if (col < 17) {
                put(kOffW1 + (o0 + gid) * kFS + col, gW1[nt][e]);
                put(kOffW1 + (o0 + gid + 8) * kFS + col, gW1[nt][2 + e]);
            } else if (DET) {  // the zero columns of W1: every entry of the row is written
                row[kOffW1 + (o0 + gid) * kFS + col] = 0.f;
                row[kOffW1 + (o0 + gid + 8) * kFS + col] = 0.f;
            }
        }
    __syncthreads();
    for (int q = threadIdx.x; q < kHid; q += blockDim.x) {
        float a = 0.f, b = 0.f, c = 0.f;
#pragma unroll
        for (int w = 0; w < kMT / 32; ++w) {
            a += S.db1[w][q];
            b += S.db2[w][q];
            c += S.dw3[w][q];
        }
        put(kOffB1 + q, a);
        put(kOffB2 + q, b);
        put(kOffW3 + q, c);
    }
    if (threadIdx.x == 0) {
        float a = 0.f, l = 0.f;
#pragma unroll
        for (int w = 0; w < kMT / 32; ++w) {
            a += S.db3[w];
            l += S.loss[w];
        }
        put(kOffB3, a);
        if (DET) {
            for (int q = kOffB3 + 1; q < LCP_MLP_NPARAMS; ++q) row[q] = 0.f;  // padding
            row[LCP_MLP_NPARAMS] = l;
        } else if (loss) {
            atomicAdd(loss, l * inv_n);
        }
    }
}

// grad[q] = (sum over CTAs, in CTA order, of their partial q) / n; the loss likewise.
__global__ void bwd_reduce_kernel(const float* __restrict__ parts, int nparts, float inv_n, float* __restrict__ grad,
                                  float* __restrict__ loss) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q <= LCP_MLP_NPARAMS; q += gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int b = 0; b < nparts; ++b) acc += parts[(int64_t)b * kPartStride + q];
        if (q < LCP_MLP_NPARAMS) grad[q] = acc * inv_n;
        else if (loss) *loss = acc * inv_n;
    }
}

// ---- 7. Adam ---------------------------------------------------------------------
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.f - b1) * gq;
        const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        p[q] -= lr * (mq * c1) / (sqrtf(vq * c2) + eps);
    }
}

}  // namespace

uint32_t read_sur_status(bool reset) {
    uint32_t f = 0;
    cudaMemcpyFromSymbol(&f, g_sur_status, sizeof(f));
    if (reset) {
        const uint32_t z = 0;
        cudaMemcpyToSymbol(g_sur_status, &z, sizeof(z));
    }
    return f;
}

}  // namespace lcp

// ---- host ------------------------------------------------------------------------
using namespace lcp;

namespace {

lcp_status check_iso_host(const char* fn, const float* iso, int K, IsoParams& ip) {
    if (!iso) return fail(LCP_ERR_ARG, "%s: iso must be a non-NULL host array", fn);
    if (K < 1 || K > kMaxIsoPerLaunch) return fail(LCP_ERR_ARG, "%s: need 1 <= K <= %d", fn, kMaxIsoPerLaunch);
    ip.K = K;
    for (int k = 0; k < K; ++k) ip.c[k] = iso[k];
    return LCP_OK;
}

int grid_for(int64_t work, int per_block, int cap_per_sm) {
    const int64_t b = (work + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms() * cap_per_sm));
}

}  // namespace

extern "C" lcp_status lcp_moments(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                                  int64_t member_stride, float* mom, lcp_stream_t stream) {
    lcp_status s = check_members("lcp_moments", u, v, in_dtype, M, H, W, member_stride, 0);
    if (s != LCP_OK) return s;
    if (!mom || !aligned16(mom)) return fail(LCP_ERR_ARG, "lcp_moments: mom must be a 16-byte aligned device array");
    const int64_t nv = (int64_t)H * W;
    const int64_t stride = M > 1 ? member_stride : nv;
    float4* out = reinterpret_cast<float4*>(mom);
    cudaStream_t st = (cudaStream_t)stream;
    const bool in16 = aligned16(u) && aligned16(v);
    if (in_dtype == LCP_F32) {
        moments_kernel<float, 4><<<grid_for((nv + 3) / 4, 256, 8), 256, 0, st>>>(
            (const float*)u, (const float*)v, M, stride, nv, in16 && stride % 4 == 0, out);
    } else {
        moments_kernel<__nv_bfloat16, 8><<<grid_for((nv + 7) / 8, 256, 8), 256, 0, st>>>(
            (const __nv_bfloat16*)u, (const __nv_bfloat16*)v, M, stride, nv, in16 && stride % 8 == 0, out);
    }
    return check_launch("lcp_moments");
}

extern "C" lcp_status lcp_surrogate_features(const float* mom, int H, int W, double dx, double dy, const float* iso,
                                             int K, void* feat, float* prior, lcp_stream_t stream) {
    if (H < 2 || W < 2) return fail(LCP_ERR_ARG, "lcp_surrogate_features: need H, W >= 2");
    lcp_status s = check_spacing("lcp_surrogate_features", dx, dy);
    if (s != LCP_OK) return s;
    IsoParams ip;
    if ((s = check_iso_host("lcp_surrogate_features", iso, K, ip)) != LCP_OK) return s;
    if (!mom || !aligned16(mom) || !feat || !aligned16(feat))
        return fail(LCP_ERR_ARG, "lcp_surrogate_features: mom and feat must be 16-byte aligned device arrays");
    const int64_t cells = (int64_t)(H - 1) * (W - 1);
    features_kernel<<<grid_for(cells, 256, 8), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(mom), H, W, make_spacing(dx, dy), ip, (__nv_bfloat16*)feat, prior);
    return check_launch("lcp_surrogate_features");
}

extern "C" lcp_status lcp_mlp_forward(const float* params, const void* feat, const float* prior, int64_t n, float* y,
                                      lcp_stream_t stream) {
    if (!params || !feat || !y || n < 1 || !aligned16(feat))
        return fail(LCP_ERR_ARG, "lcp_mlp_forward: NULL/misaligned pointer or n < 1");
    mlp_forward_kernel<<<grid_for(n, 64, 8), kMT, 0, (cudaStream_t)stream>>>(
        params, (const __nv_bfloat16*)feat, prior, n, y);
    return check_launch("lcp_mlp_forward");
}

namespace {
// Shared-memory size of both backward variants, set once per device.
lcp_status prepare_backward(const char* fn) {
    static std::mutex mu;
    static bool set[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return fail(LCP_ERR_CUDA, "%s: no usable current device", fn);
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!set[dev]) {
        if (cudaFuncSetAttribute(mlp_backward_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(BwdSmem)) != cudaSuccess ||
            cudaFuncSetAttribute(mlp_backward_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(BwdSmem)) != cudaSuccess) {
            cudaGetLastError();
            return fail(LCP_ERR_CUDA, "%s: %zu bytes of shared memory not available", fn, sizeof(BwdSmem));
        }
        set[dev] = true;
    }
    return LCP_OK;
}

lcp_status check_backward(const char* fn, const float* params, const void* feat, const float* target, float* grad,
                          int64_t n) {
    if (!params || !feat || !target || !grad || n < 1 || !aligned16(feat))
        return fail(LCP_ERR_ARG, "%s: NULL/misaligned pointer or n < 1", fn);
    return LCP_OK;
}
}  // namespace

extern "C" lcp_status lcp_mlp_backward(const float* params, const void* feat, const float* prior, const float* target,
                                       int64_t n, float* grad, float* loss, lcp_stream_t stream) {
    static const char* fn = "lcp_mlp_backward";
    lcp_status s = check_backward(fn, params, feat, target, grad, n);
    if (s != LCP_OK || (s = prepare_backward(fn)) != LCP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(grad, 0, LCP_MLP_NPARAMS * sizeof(float), st) != cudaSuccess ||
        (loss && cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess)) {
        cudaGetLastError();
        return fail(LCP_ERR_CUDA, "%s: clearing the outputs failed", fn);
    }
    mlp_backward_kernel<false><<<grid_for(n, 64, 2), kMT, sizeof(BwdSmem), st>>>(
        params, (const __nv_bfloat16*)feat, prior, target, n, grad, loss, nullptr);
    return check_launch(fn);
}

extern "C" size_t lcp_mlp_backward_workspace_bytes(int64_t n) {
    if (n < 1) return 0;
    return (size_t)grid_for(n, 64, 2) * kPartStride * sizeof(float);
}

extern "C" lcp_status lcp_mlp_backward_ws(const float* params, const void* feat, const float* prior,
                                          const float* target, int64_t n, float* grad, float* loss, void* workspace,
                                          size_t workspace_bytes, lcp_stream_t stream) {
    static const char* fn = "lcp_mlp_backward_ws";
    lcp_status s = check_backward(fn, params, feat, target, grad, n);
    if (s != LCP_OK) return s;
    const int grid = grid_for(n, 64, 2);
    const size_t need = (size_t)grid * kPartStride * sizeof(float);
    if (!workspace || !aligned16(workspace) || workspace_bytes < need)
        return fail(LCP_ERR_ARG, "%s: need a 16-byte aligned workspace of %zu bytes", fn, need);
    if ((s = prepare_backward(fn)) != LCP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float* parts = reinterpret_cast<float*>(workspace);
    mlp_backward_kernel<true><<<grid, kMT, sizeof(BwdSmem), st>>>(params, (const __nv_bfloat16*)feat, prior, target,
                                                                    n, grad, loss, parts);
    if ((s = check_launch(fn)) != LCP_OK) return s;
    bwd_reduce_kernel<<<(LCP_MLP_NPARAMS + 1 + 255) / 256, 256, 0, st>>>(parts, grid, 1.0f / (float)n, grad, loss);
    return check_launch(fn);
}

extern "C" lcp_status lcp_adam_step(float* params, const float* grad, float* m, float* v, int64_t n, int t, float lr,
                                    float beta1, float beta2, float eps, lcp_stream_t stream) {
    if (!params || !grad || !m || !v || n < 1 || t < 1)
        return fail(LCP_ERR_ARG, "lcp_adam_step: NULL pointer, n < 1 or t < 1");
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f))
        return fail(LCP_ERR_ARG, "lcp_adam_step: need 0 <= beta < 1 and eps >= 0");
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)t)));
    adam_kernel<<<grid_for(n, 256, 4), 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, n, lr, beta1, beta2, eps,
                                                                        c1, c2);
    return check_launch("lcp_adam_step");
}

extern "C" lcp_status lcp_mlp_infer(const float* mom, int H, int W, double dx, double dy, const float* iso, int K,
                                    const float* params, void* lcp_out, lcp_dtype out_dtype, lcp_stream_t stream) {
    if (H < 2 || W < 2) return fail(LCP_ERR_ARG, "lcp_mlp_infer: need H, W >= 2");
    lcp_status s = check_spacing("lcp_mlp_infer", dx, dy);
    if (s != LCP_OK) return s;
    IsoParams ip;
    if ((s = check_iso_host("lcp_mlp_infer", iso, K, ip)) != LCP_OK) return s;
    if (!mom || !aligned16(mom) || !params || !lcp_out)
        return fail(LCP_ERR_ARG, "lcp_mlp_infer: NULL or misaligned pointer");
    if (out_dtype != LCP_F32 && out_dtype != LCP_F16) return fail(LCP_ERR_ARG, "lcp_mlp_infer: out dtype must be F32 or F16");
    const int64_t nblocks = (int64_t)((W - 1 + kIC - 1) / kIC) * ((H - 1 + kIR - 1) / kIR);
    if (nblocks > INT_MAX) return fail(LCP_ERR_UNSUPPORTED, "lcp_mlp_infer: grid too large");
    const float4* m4 = reinterpret_cast<const float4*>(mom);
    const Spacing sp = make_spacing(dx, dy);
    {
        static std::mutex mu;
        static bool set[64] = {false};
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
            cudaGetLastError();
            return fail(LCP_ERR_CUDA, "lcp_mlp_infer: no usable current device");
        }
        std::lock_guard<std::mutex> lk(mu);
        if (!set[dev]) {
            // the full shared-memory carveout, so that the occupancy below counts every resident CTA
            if (cudaFuncSetAttribute(mlp_infer_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTcSmemBytes) != cudaSuccess ||
                cudaFuncSetAttribute(mlp_infer_tc_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTcSmemBytes) != cudaSuccess ||
                cudaFuncSetAttribute(mlp_infer_tc_kernel<float>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
                cudaFuncSetAttribute(mlp_infer_tc_kernel<__half>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess) {
                cudaGetLastError();
                return fail(LCP_ERR_CUDA, "lcp_mlp_infer: %zu bytes of shared memory not available", kTcSmemBytes);
            }
            set[dev] = true;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    // persistent: kTcCtasPerSm CTAs per SM (the kernel's launch bounds; its
    // registers, shared memory and 64 TMEM columns each allow that many), each
    // walking cell blocks; CTAs beyond what fits wait for a slot (no CTA waits
    // on another)
    const int grid = (int)std::min<int64_t>(nblocks, (int64_t)kTcCtasPerSm * num_sms());
    if (out_dtype == LCP_F16)
        mlp_infer_tc_kernel<__half><<<grid, kMT, kTcSmemBytes, st>>>(m4, H, W, sp, ip, params, (__half*)lcp_out);
    else
        mlp_infer_tc_kernel<float><<<grid, kMT, kTcSmemBytes, st>>>(m4, H, W, sp, ip, params, (float*)lcp_out);
    return check_launch("lcp_mlp_infer");
}
