// Learned surrogate: moments of the members, cumulants of the vertex
// divergence under the empirical model, per-cell features, and a
// 17 -> 64 -> 64 -> 1 network trained and evaluated on the 5th-generation
// tensor cores: tcgen05.mma with BF16 operands in shared memory (canonical
// K-major layout, no swizzle), FP32 accumulators in tensor memory read back
// with tcgen05.ld, one thread issuing each layer's MMAs and committing them to
// an mbarrier.  Inference (section 4) evaluates 128 cells per tile from the
// moments; training (section 5) runs the forward pass, the backward pass and
// the weight gradients of 128 feature rows per tile, the gradients as one more
// contraction over the rows accumulated in tensor memory.

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

// ---- 1. moments ---------------------------------------------------------------
// Shifted power sums about member 0, then the central moments by the binomial
// expansion: with delta = S1/M and e_p = S_p/M,
//   m2 = e2 - delta^2,  m3 = e3 - 3 delta e2 + 2 delta^3,
//   m4 = e4 - 4 delta e3 + 6 delta^2 e2 - 3 delta^4.
// Members in batches (every load of a batch in flight at once): fp32 4 per batch at
// <= 64 registers (4 blocks per SM), bf16 8 per batch at full registers.  Measured on
// 1024^2 x 50 members: fp32 0.111 -> 0.071 ms (0.94 of the measured HBM copy peak),
// bf16 0.116 -> 0.060 ms, against one load in flight per thread.
template <typename T>
struct MomTune {
    static constexpr int kBatch = sizeof(T) == 4 ? 4 : 8;
    static constexpr int kMinBlocks = sizeof(T) == 4 ? 4 : 1;
};
template <typename T, int VEC>
__global__ void __launch_bounds__(256, MomTune<T>::kMinBlocks) moments_kernel(const T* __restrict__ u, const T* __restrict__ v, int M,
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
            auto acc = [&](const float (&a)[VEC]) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const float d = a[e] - x0[e], d2 = d * d;
                    s[0][e] += d;
                    s[1][e] += d2;
                    s[2][e] = fmaf(d2, d, s[2][e]);
                    s[3][e] = fmaf(d2, d2, s[3][e]);
                }
            };
            if (vec) {  // members in batches of kMB, every load of a batch in flight at once
                constexpr int kMB = MomTune<T>::kBatch;
                for (int m = 1; m < M; m += kMB) {
                    typename L::raw_t r[kMB];
#pragma unroll
                    for (int q = 0; q < kMB; ++q)
                        if (m + q < M) r[q] = L::load(x + (int64_t)(m + q) * stride + n0);
#pragma unroll
                    for (int q = 0; q < kMB; ++q)
                        if (m + q < M) {
                            float a[VEC];
                            L::cvt(r[q], a);
                            acc(a);
                        }
                }
            } else {
                for (int m = 1; m < M; ++m) {
                    float a[VEC];
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        a[e] = 0.f;
                        if (e < cnt) Loader<T, 1>::cvt(Loader<T, 1>::load(x + (int64_t)m * stride + n0 + e), &a[e]);
                    }
                    acc(a);
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

// below_above for two vertices at once: the same steps per vertex, the erfc
// polynomial on paired FP32 instructions (each half one IEEE operation, so the
// results equal two scalar calls bit for bit).
__device__ __forceinline__ void below_above2(const VertexG& g0, const VertexG& g1, float c, float (&p)[2],
                                             float (&q)[2]) {
    const float2 t = __fmul2_rn(__fadd2_rn(make_float2(g0.mu, g1.mu), make_float2(-c, -c)), make_float2(g0.s, g1.s));
    const float2 e = half_erfc_nonneg2(make_float2(fabsf(t.x), fabsf(t.y)));
    const float tt[2] = {t.x, t.y}, ee[2] = {e.x, e.y}, ss[2] = {g0.s, g1.s}, mm[2] = {g0.mu, g1.mu};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (ss[k] == 0.0f) {
            p[k] = (mm[k] < c) ? 1.0f : 0.0f;
            q[k] = 1.0f - p[k];
        } else if (tt[k] >= 0.0f) {
            p[k] = ee[k];
            q[k] = 1.0f - ee[k];
        } else {
            q[k] = ee[k];
            p[k] = 1.0f - ee[k];
        }
    }
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
    }
#pragma unroll
    for (int v = 0; v < 4; v += 2) {  // the four vertices' (p, q) as two paired erfc evaluations
        float pv[2], qv[2];
        below_above2(p.g[v], p.g[v + 1], c, pv, qv);
        pb *= pv[0];
        qb *= qv[0];
        pb *= pv[1];
        qb *= qv[1];
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

// ---- 3. shared helpers --------------------------------------------------------
constexpr int kMT = 128;           // threads per CTA of the network kernels (4 warps; one row or cell per thread)
constexpr int kIR = 4, kIC = 32;   // inference CTA: 4 cell rows x 32 cell columns

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
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

// ---- 4. fused inference on the 5th-generation tensor cores (tcgen05) ----------
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

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate,
                                       uint32_t idesc = kIdescM128N64) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
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
                for (int e = 0; e < 8; ++e) {  // bias added two units at a time (paired FP32 add)
                    const float2 zz = __fadd2_rn(make_float2(z[2 * e], z[2 * e + 1]),
                                                 *reinterpret_cast<const float2*>(&S.b1[16 * cg + 2 * e]));
                    hw[e] = tanh_bf16x2(zz.x, zz.y);
                }
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
                    const float2 zz = __fadd2_rn(make_float2(z[2 * e], z[2 * e + 1]),
                                                 *reinterpret_cast<const float2*>(&S.b2[16 * cg + 2 * e]));
                    const float2 h = unpack_bf16(tanh_bf16x2(zz.x, zz.y));
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

// ---- 5. training on the 5th-generation tensor cores (tcgen05) -------------------
// One CTA walks tiles of 128 feature rows, one row per thread (= TMEM lane).
// Per tile, four groups of tcgen05.mma (M = 128, FP32 accumulators in TMEM,
// BF16 operands in shared memory in the canonical K-major layout, issued by
// one thread and committed to an mbarrier):
//   layer 1   D = X W1^T               (N = 64, K = 32)  -> h1 = bf16(tanh(D + b1))
//   layer 2   D = H1 W2^T              (N = 64, K = 64)  -> h2 = tanh(D + b2), y
//   backward  D = dZ2 W2               (N = 64, K = 64)  -> dZ1 = D (1 - h1^2)
//   gradients G += [dZ2^T; dZ1^T] [H1 | X | 1]           (M = 128, N = 112, K = the tile's 128 rows)
// so that rows 0-63 of G hold dW2 (columns 0-63) and db2 (column 96), and rows
// 64-127 hold dW1 (columns 64-80) and db1 (column 96); G accumulates over the
// CTA's tiles.  dz3 = d(squared error)/dz3 = 2 (y - t) y (1 - y) per row; dw3,
// db3 and the loss are summed over the warp's rows by shuffles into per-warp
// partials (added in warp order at the end), so a CTA's result does not
// depend on the order in which its warps run.  The forward-only variant
// (BWD = false) writes y and stops after layer 2.
constexpr uint32_t kIdescM128N112 =
    (1u << 4) | (1u << 7) | (1u << 10) | ((112u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kTrainTmemCols = 256;  // D in columns 0-63, G in 128-239
constexpr int kGN = 112;                  // rows of the gradient B operand
constexpr int kPartStride = LCP_MLP_NPARAMS + 4;  // a CTA's partial: the parameters, then the loss (16-byte rows)

struct TrainSmem {
    __align__(1024) __nv_bfloat16 W1[kHid * kFS];    // B of layer 1: N = 64 units x K = 32 features
    __align__(1024) __nv_bfloat16 W2[kHid * kHid];   // B of layer 2: N = 64 outputs x K = 64 inputs
    __align__(1024) __nv_bfloat16 W2t[kHid * kHid];  // B of the backward product: N = 64 inputs x K = 64 outputs
    __align__(1024) __nv_bfloat16 X[128 * kFS];      // A of layer 1: the tile's feature rows
    __align__(1024) __nv_bfloat16 H1[128 * kHid];    // A of layer 2: h1 rows
    __align__(1024) __nv_bfloat16 DZ2[128 * kHid];   // A of the backward product: dZ2 rows
    __align__(1024) __nv_bfloat16 Ag[128 * 128];     // A of the gradients: dZ2^T (rows 0-63), dZ1^T (64-127)
    __align__(1024) __nv_bfloat16 Bg[kGN * 128];     // B: H1^T (rows 0-63), X^T (64-95), ones (96), zeros
    float b1[kHid], b2[kHid], w3[kHid];
    float dw3[kMT / 32][kHid];
    float db3[kMT / 32], loss[kMT / 32];
    __align__(8) uint64_t mbar;
    uint32_t tmem;
    int abort_flag;  // set when an mbarrier wait gave up; read by all threads after a barrier
};
constexpr size_t kTrainSmemBytes = sizeof(TrainSmem) + 1024;

__device__ __forceinline__ void put_canon(__nv_bfloat16* tile, int row, int k, int kg, __nv_bfloat16 v) {
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(tile) + canon_off(row, k, kg)) = v;
}
__device__ __forceinline__ void put_canon16(__nv_bfloat16* tile, int row, int k, int kg, uint4 v) {  // k % 8 == 0
    *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(tile) + canon_off(row, k, kg)) = v;
}
__device__ __forceinline__ uint4 get_canon16(const __nv_bfloat16* tile, int row, int k, int kg) {
    return *reinterpret_cast<const uint4*>(reinterpret_cast<const unsigned char*>(tile) + canon_off(row, k, kg));
}
__device__ __forceinline__ __nv_bfloat16 bf16_bits(uint32_t w, int hi) {
    const unsigned short s = (unsigned short)(hi ? (w >> 16) : (w & 0xFFFFu));
    return *reinterpret_cast<const __nv_bfloat16*>(&s);
}
// Generic-proxy shared-memory writes visible to the tensor core, every thread's
// earlier TMEM reads ordered before the MMAs issued next, all threads past.
__device__ __forceinline__ void tc_handoff() {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

template <bool BWD, bool DET>
__global__ void __launch_bounds__(kMT, 1) mlp_train_tc_kernel(const float* __restrict__ prm,
                                                              const __nv_bfloat16* __restrict__ feat,
                                                              const float* __restrict__ prior,
                                                              const float* __restrict__ target, int64_t n,
                                                              float* __restrict__ y, float* __restrict__ grad,
                                                              float* __restrict__ loss, float* __restrict__ parts) {
    extern __shared__ __align__(1024) unsigned char tr_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(tr_raw + ((1024 - (smem_addr(tr_raw) & 1023)) & 1023));
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int kg1 = kFS / 8, kg2 = kHid / 8, kgG = 128 / 8;  // core matrices along K
    // weights into the canonical layouts (bf16), vectors as fp32
    for (int q = t; q < kHid * kFS; q += kMT) {
        const int u = q / kFS, f = q - u * kFS;
        put_canon(S.W1, u, f, kg1, __float2bfloat16_rn(f < 17 ? prm[kOffW1 + q] : 0.f));
    }
    for (int q = t; q < kHid * kHid; q += kMT) {
        const int o = q >> 6, i = q & 63;
        const __nv_bfloat16 w = __float2bfloat16_rn(prm[kOffW2 + q]);
        put_canon(S.W2, o, i, kg2, w);
        if (BWD) put_canon(S.W2t, i, o, kg2, w);
    }
    for (int q = t; q < kHid; q += kMT) {
        S.b1[q] = prm[kOffB1 + q];
        S.b2[q] = prm[kOffB2 + q];
        S.w3[q] = prm[kOffW3 + q];
    }
    if (BWD) {
        // the rows of Bg that no tile rewrites: X^T of the zero features 17-31, the ones, the zeros
        for (int q = t; q < (kGN - 81) * 128; q += kMT) {
            const int rr = 81 + q / 128, k = q % 128;
            put_canon(S.Bg, rr, k, kgG, __float2bfloat16_rn(rr == 96 ? 1.f : 0.f));
        }
        for (int q = t; q < (kMT / 32) * kHid; q += kMT) (&S.dw3[0][0])[q] = 0.f;
        if (t < kMT / 32) S.db3[t] = S.loss[t] = 0.f;
    }
    if (t == 0) {
        S.abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&S.tmem)),
                     "r"(kTrainTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_handoff();  // weights, constant rows, TMEM address and mbarrier are ready
    const uint32_t tmem = S.tmem, tmem_g = tmem + 128;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16), lane_g = lane_base + 128;
    const uint32_t mbar = smem_addr(&S.mbar);
    const uint32_t aX = smem_addr(S.X), aH = smem_addr(S.H1), aD = smem_addr(S.DZ2), aG = smem_addr(S.Ag);
    const uint32_t bW1 = smem_addr(S.W1), bW2 = smem_addr(S.W2), bW2t = smem_addr(S.W2t), bG = smem_addr(S.Bg);
    const float b3 = prm[kOffB3];
    uint32_t phase = 0;
    volatile int* abort_flag = &S.abort_flag;
    bool any = false;  // G holds this CTA's sums (uniform)
    auto mma_wait = [&]() {
        if (!mbar_wait(mbar, phase)) *abort_flag = 1;
        phase ^= 1u;
        tc_fence_after();
    };
    const int64_t ntiles = (n + 127) / 128;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r = tile * 128 + t;
        const bool valid = r < n;
        // features: X (A of layer 1) and X^T (rows 64-80 of Bg); rows beyond n are zero
        uint4 xr[kFS / 8];
#pragma unroll
        for (int g = 0; g < kFS / 8; ++g) {
            xr[g] = valid ? __ldg(reinterpret_cast<const uint4*>(feat + r * kFS) + g) : make_uint4(0, 0, 0, 0);
            put_canon16(S.X, t, 8 * g, kg1, xr[g]);
        }
        if (BWD) {
            const uint32_t* xw = reinterpret_cast<const uint32_t*>(xr);
#pragma unroll
            for (int f = 0; f < 17; ++f) put_canon(S.Bg, 64 + f, t, kgG, bf16_bits(xw[f >> 1], f & 1));
        }
        tc_handoff();
        if (*abort_flag) break;  // uniform: read after the barrier, written only before one
        if (t == 0) {
#pragma unroll
            for (int s = 0; s < 2; ++s)
                tc_mma(tmem, smem_desc(aX + 256 * s, 128, 128 * kg1), smem_desc(bW1 + 256 * s, 128, 128 * kg1), s);
            tc_commit(mbar);
        }
        mma_wait();
        // h1 = bf16(tanh(D + b1)): H1 (A of layer 2) and H1^T (rows 0-63 of Bg)
#pragma unroll
        for (int cg = 0; cg < 4; ++cg) {
            float z[16];
            tmem_ld16(lane_base + 16 * cg, z);
            uint32_t hw[8];
#pragma unroll
            for (int e = 0; e < 8; ++e)
                hw[e] = pack_bf16(tanh_fast(z[2 * e] + S.b1[16 * cg + 2 * e]),
                                  tanh_fast(z[2 * e + 1] + S.b1[16 * cg + 2 * e + 1]));
            put_canon16(S.H1, t, 16 * cg, kg2, make_uint4(hw[0], hw[1], hw[2], hw[3]));
            put_canon16(S.H1, t, 16 * cg + 8, kg2, make_uint4(hw[4], hw[5], hw[6], hw[7]));
            if (BWD) {
#pragma unroll
                for (int e = 0; e < 16; ++e) put_canon(S.Bg, 16 * cg + e, t, kgG, bf16_bits(hw[e >> 1], e & 1));
            }
        }
        tc_handoff();
        if (*abort_flag) break;
        if (t == 0) {
#pragma unroll
            for (int s = 0; s < 4; ++s)
                tc_mma(tmem, smem_desc(aH + 256 * s, 128, 128 * kg2), smem_desc(bW2 + 256 * s, 128, 128 * kg2), s);
            tc_commit(mbar);
        }
        mma_wait();
        // output: y = sigmoid(b3 + prior + w3 . tanh(D + b2))
        float z3 = b3 + ((prior && valid) ? __ldg(prior + r) : 0.f);
#pragma unroll
        for (int cg = 0; cg < 4; ++cg) {
            float z[16];
            tmem_ld16(lane_base + 16 * cg, z);
#pragma unroll
            for (int e = 0; e < 16; ++e) z3 = fmaf(tanh_fast(z[e] + S.b2[16 * cg + e]), S.w3[16 * cg + e], z3);
        }
        const float yv = sigmoid(z3);
        if (!BWD) {
            if (valid) y[r] = yv;
            tc_fence_before();  // this tile's TMEM reads are ordered before the next MMA
            continue;
        }
        const float tv = valid ? __ldg(target + r) : 0.f;
        // d(sum of squared errors)/dz3 = 2 (y - t) y (1 - y); the 1/n of the mean is applied once at the end
        const float dz3 = valid ? 2.f * (yv - tv) * yv * (1.f - yv) : 0.f;
        const float err2 = valid ? (yv - tv) * (yv - tv) : 0.f;
        // dZ2 = dz3 w3 (1 - h2^2): DZ2 (A of the backward product) and dZ2^T (rows 0-63 of Ag);
        // dw3 = sum over rows of dz3 h2, reduced over the warp 16 columns at a time
#pragma unroll
        for (int cg = 0; cg < 4; ++cg) {
            float z[16], ev[16];
            tmem_ld16(lane_base + 16 * cg, z);
            uint32_t dw[8];
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const float h0 = tanh_fast(z[e] + S.b2[16 * cg + e]), h1v = tanh_fast(z[e + 1] + S.b2[16 * cg + e + 1]);
                ev[e] = dz3 * h0;
                ev[e + 1] = dz3 * h1v;
                dw[e >> 1] = pack_bf16(dz3 * S.w3[16 * cg + e] * (1.f - h0 * h0),
                                       dz3 * S.w3[16 * cg + e + 1] * (1.f - h1v * h1v));
            }
            put_canon16(S.DZ2, t, 16 * cg, kg2, make_uint4(dw[0], dw[1], dw[2], dw[3]));
            put_canon16(S.DZ2, t, 16 * cg + 8, kg2, make_uint4(dw[4], dw[5], dw[6], dw[7]));
#pragma unroll
            for (int e = 0; e < 16; ++e) put_canon(S.Ag, 16 * cg + e, t, kgG, bf16_bits(dw[e >> 1], e & 1));
            // reduce-scatter of the 16 columns over the 32 lanes: lanes 2c and 2c + 1 end with column c
#pragma unroll
            for (int w = 16, m = 8; m >= 1; w >>= 1, m >>= 1) {
                const bool up = (lane & w) != 0;
#pragma unroll
                for (int e = 0; e < m; ++e) {
                    const float give = up ? ev[e] : ev[m + e];
                    const float keep = up ? ev[m + e] : ev[e];
                    ev[e] = keep + __shfl_xor_sync(0xFFFFFFFFu, give, w);
                }
            }
            ev[0] += __shfl_xor_sync(0xFFFFFFFFu, ev[0], 1);
            if ((lane & 1) == 0) S.dw3[warp][16 * cg + (lane >> 1)] += ev[0];
        }
        {  // db3 and the loss: the warp's rows, fixed order
            float a = dz3, l = err2;
#pragma unroll
            for (int w = 16; w >= 1; w >>= 1) {
                a += __shfl_xor_sync(0xFFFFFFFFu, a, w);
                l += __shfl_xor_sync(0xFFFFFFFFu, l, w);
            }
            if (lane == 0) {
                S.db3[warp] += a;
                S.loss[warp] += l;
            }
        }
        tc_handoff();
        if (*abort_flag) break;
        if (t == 0) {  // dA1 = dZ2 W2
#pragma unroll
            for (int s = 0; s < 4; ++s)
                tc_mma(tmem, smem_desc(aD + 256 * s, 128, 128 * kg2), smem_desc(bW2t + 256 * s, 128, 128 * kg2), s);
            tc_commit(mbar);
        }
        mma_wait();
        // dZ1 = dA1 (1 - h1^2), h1 as rounded for layer 2: dZ1^T (rows 64-127 of Ag)
#pragma unroll
        for (int cg = 0; cg < 4; ++cg) {
            float z[16];
            tmem_ld16(lane_base + 16 * cg, z);
            const uint4 ha = get_canon16(S.H1, t, 16 * cg, kg2), hb = get_canon16(S.H1, t, 16 * cg + 8, kg2);
            const uint32_t hw[8] = {ha.x, ha.y, ha.z, ha.w, hb.x, hb.y, hb.z, hb.w};
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                const float2 h = unpack_bf16(hw[e >> 1]);
                const uint32_t d1 = pack_bf16(z[e] * (1.f - h.x * h.x), z[e + 1] * (1.f - h.y * h.y));
                put_canon(S.Ag, 64 + 16 * cg + e, t, kgG, bf16_bits(d1, 0));
                put_canon(S.Ag, 64 + 16 * cg + e + 1, t, kgG, bf16_bits(d1, 1));
            }
        }
        tc_handoff();
        if (*abort_flag) break;
        if (t == 0) {  // G += [dZ2^T; dZ1^T] [H1 | X | 1] over the tile's 128 rows
#pragma unroll
            for (int s = 0; s < 8; ++s)
                tc_mma(tmem_g, smem_desc(aG + 256 * s, 128, 128 * kgG), smem_desc(bG + 256 * s, 128, 128 * kgG),
                       (any || s > 0) ? 1u : 0u, kIdescM128N112);
            tc_commit(mbar);
        }
        mma_wait();  // the MMAs have read this tile's operands before the next tile rewrites them
        any = true;
    }
    if (BWD) {
        // this CTA's sums: thread t holds row t of G (TMEM lane t)
        const float inv_n = 1.0f / (float)n;
        float* const row = DET ? parts + (int64_t)blockIdx.x * kPartStride : nullptr;
        auto put = [&](int idx, float val) {
            if (DET) row[idx] = val;
            else atomicAdd(grad + idx, val * inv_n);
        };
        float gsum[kGN];
        if (any) {
#pragma unroll
            for (int cg = 0; cg < kGN / 16; ++cg) {
                float z[16];
                tmem_ld16(lane_g + 16 * cg, z);
#pragma unroll
                for (int e = 0; e < 16; ++e) gsum[16 * cg + e] = z[e];
            }
        } else {
#pragma unroll
            for (int e = 0; e < kGN; ++e) gsum[e] = 0.f;
        }
        if (t < kHid) {  // dW2 row t, db2[t]
#pragma unroll
            for (int i = 0; i < kHid; ++i) put(kOffW2 + t * kHid + i, gsum[i]);
            put(kOffB2 + t, gsum[96]);
        } else {  // dW1 row u, db1[u]
            const int u = t - kHid;
#pragma unroll
            for (int f = 0; f < kFS; ++f) {
                if (f < 17) put(kOffW1 + u * kFS + f, gsum[64 + f]);
                else if (DET) row[kOffW1 + u * kFS + f] = 0.f;  // the zero columns of W1: every entry written
            }
            put(kOffB1 + u, gsum[96]);
        }
        __syncthreads();
        for (int q = t; q < kHid; q += kMT) {
            float c = 0.f;
#pragma unroll
            for (int w = 0; w < kMT / 32; ++w) c += S.dw3[w][q];
            put(kOffW3 + q, c);
        }
        if (t == 0) {
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
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTrainTmemCols) : "memory");
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

// ---- 6. Adam ---------------------------------------------------------------------
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

namespace {
// The training kernels' shared memory (about 124 KB: one CTA per SM), set once per device.
lcp_status prepare_train(const char* fn) {
    static std::mutex mu;
    static bool set[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return fail(LCP_ERR_CUDA, "%s: no usable current device", fn);
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!set[dev]) {
        const int b = (int)kTrainSmemBytes;
        if (cudaFuncSetAttribute(mlp_train_tc_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b) !=
                cudaSuccess ||
            cudaFuncSetAttribute(mlp_train_tc_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b) !=
                cudaSuccess ||
            cudaFuncSetAttribute(mlp_train_tc_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b) !=
                cudaSuccess) {
            cudaGetLastError();
            return fail(LCP_ERR_CUDA, "%s: %zu bytes of shared memory not available", fn, kTrainSmemBytes);
        }
        set[dev] = true;
    }
    return LCP_OK;
}

// 128-row tiles, one CTA per SM walking them.
int train_grid(int64_t n) { return grid_for(n, 128, 1); }

lcp_status check_backward(const char* fn, const float* params, const void* feat, const float* target, float* grad,
                          int64_t n) {
    if (!params || !feat || !target || !grad || n < 1 || !aligned16(feat))
        return fail(LCP_ERR_ARG, "%s: NULL/misaligned pointer or n < 1", fn);
    return LCP_OK;
}
}  // namespace

extern "C" lcp_status lcp_mlp_forward(const float* params, const void* feat, const float* prior, int64_t n, float* y,
                                      lcp_stream_t stream) {
    static const char* fn = "lcp_mlp_forward";
    if (!params || !feat || !y || n < 1 || !aligned16(feat))
        return fail(LCP_ERR_ARG, "%s: NULL/misaligned pointer or n < 1", fn);
    lcp_status s = prepare_train(fn);
    if (s != LCP_OK) return s;
    mlp_train_tc_kernel<false, false><<<train_grid(n), kMT, kTrainSmemBytes, (cudaStream_t)stream>>>(
        params, (const __nv_bfloat16*)feat, prior, nullptr, n, y, nullptr, nullptr, nullptr);
    return check_launch(fn);
}

extern "C" lcp_status lcp_mlp_backward(const float* params, const void* feat, const float* prior, const float* target,
                                       int64_t n, float* grad, float* loss, lcp_stream_t stream) {
    static const char* fn = "lcp_mlp_backward";
    lcp_status s = check_backward(fn, params, feat, target, grad, n);
    if (s != LCP_OK || (s = prepare_train(fn)) != LCP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(grad, 0, LCP_MLP_NPARAMS * sizeof(float), st) != cudaSuccess ||
        (loss && cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess)) {
        cudaGetLastError();
        return fail(LCP_ERR_CUDA, "%s: clearing the outputs failed", fn);
    }
    mlp_train_tc_kernel<true, false><<<train_grid(n), kMT, kTrainSmemBytes, st>>>(
        params, (const __nv_bfloat16*)feat, prior, target, n, nullptr, grad, loss, nullptr);
    return check_launch(fn);
}

extern "C" size_t lcp_mlp_backward_workspace_bytes(int64_t n) {
    if (n < 1) return 0;
    return (size_t)train_grid(n) * kPartStride * sizeof(float);
}

extern "C" lcp_status lcp_mlp_backward_ws(const float* params, const void* feat, const float* prior,
                                          const float* target, int64_t n, float* grad, float* loss, void* workspace,
                                          size_t workspace_bytes, lcp_stream_t stream) {
    static const char* fn = "lcp_mlp_backward_ws";
    lcp_status s = check_backward(fn, params, feat, target, grad, n);
    if (s != LCP_OK) return s;
    const int grid = train_grid(n);
    const size_t need = (size_t)grid * kPartStride * sizeof(float);
    if (!workspace || !aligned16(workspace) || workspace_bytes < need)
        return fail(LCP_ERR_ARG, "%s: need a 16-byte aligned workspace of %zu bytes", fn, need);
    if ((s = prepare_train(fn)) != LCP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    float* parts = reinterpret_cast<float*>(workspace);
    mlp_train_tc_kernel<true, true><<<grid, kMT, kTrainSmemBytes, st>>>(params, (const __nv_bfloat16*)feat, prior,
                                                                       target, n, nullptr, grad, loss, parts);
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
