// lcp_fused, TMA pipeline variant (sm_103a): the same computation as the
// register-streaming kernel in fused.cu (statistics, Eqs. 2/3, LCP), with the
// member stream moved off the threads and onto the Tensor Memory Accelerator.
//
// Warp specialisation.  One producer warp walks the same row sequence as the
// CTA's march and, for every (row, chunk of MB members), issues 3D TMA copies
// (cp.async.bulk.tensor, box = window columns x 1 row x MB members) of u and v
// into a ring of NSTAGE shared-memory stages, signalling an mbarrier with the
// transaction byte count.  Five consumer warps reduce each stage into shifted
// sums, release it, and between rows evaluate the divergence Gaussian and the
// cells' LCP while the producer already streams the next rows: HBM never waits
// for the ALU phase and no thread holds loads in registers.
//
// Tile.  TW = 256 cell columns; the shared-memory window spans one 16-byte
// column group beyond each side (x must start on a 16-byte boundary), so u at
// c0 - 1 and c0 + TW + 1 come with the same copies.  Two boxes per member row
// (each at most 256 elements wide) cover the window.  Rows outside the band
// (the one-row v halo above and below) skip the u copies.
//
// Every wait is bounded: a wait that exceeds its clock budget raises the CTA's
// abort flag and the library's device status word; from then on the CTA's
// waits return at once, the loops run to their ends without touching
// shared memory that a copy may still target, and the producer finally
// waits (bounded) for the copies it issued.
#include <cuda.h>

#include <mutex>

#include "lcp_common.cuh"

namespace lcp {

__device__ unsigned int g_fused_status;  // bit 0: a bounded wait gave up

namespace {

constexpr int TW = 256;        // cell columns per tile
constexpr int MB = 8;          // members per stage
constexpr int NSTAGE = 4;      // stages in the ring
constexpr int NCONS = 160;     // consumer threads (5 warps)
constexpr int NTHREADS = NCONS + 32;
constexpr int kOwnG = TW / 4;  // own 4-column groups = div threads per isovalue split
constexpr int kMaxKPass = 32;
constexpr long long kWaitBudget = 4000000000ll;  // clock cycles (~2 s) before a wait gives up

template <typename T>
struct TGeom {
    static constexpr int ESZ = sizeof(T);
    static constexpr int WOFF = 16 / ESZ;          // window starts at c0 - WOFF (16-byte aligned)
    static constexpr int NCOLW = TW + 2 * WOFF;    // window columns
    static constexpr int NG = NCOLW / 4;           // 4-column groups in the window
    static constexpr int G0 = WOFF / 4;            // first own group
    static constexpr int BXA = NCOLW / 2;          // box A width (elements)
    static constexpr int BXB = NCOLW - BXA;        // box B width
    static constexpr int COMP_BYTES = MB * NCOLW * ESZ;
    static constexpr int STAGE_BYTES = 2 * COMP_BYTES;
    static_assert(BXA <= 256 && BXB <= 256, "TMA box dims are at most 256");
    static_assert((BXA * ESZ) % 16 == 0 && (BXB * ESZ) % 16 == 0, "TMA box rows are 16-byte multiples");
    static_assert((MB * BXA * ESZ) % 128 == 0 && COMP_BYTES % 128 == 0, "TMA destinations 128-byte aligned");
    static_assert(2 * NG <= NCONS, "two member splits of the window fit the consumers");
};

struct TmaParams {
    int M, H, W, ddof;
    Spacing sp;
    void* out;
    uint32_t* mask;
    int n_words;
    int n_ty;
    int kbase;
};

struct Maps {
    CUtensorMap ua, ub, va, vb;
};

// ---- PTX wrappers --------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; returns false (and raises the abort flag) if the budget runs out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile uint32_t* abort) {
    if (*abort) return false;
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (*abort) return false;
        if (clock64() - t0 > kWaitBudget) {
            *abort = 1u;
            atomicOr(&g_fused_status, 1u);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

template <typename T>
__device__ __forceinline__ void load4(const T* p, float* x);
template <>
__device__ __forceinline__ void load4<float>(const float* p, float* x) {
    const float4 r = *reinterpret_cast<const float4*>(p);
    x[0] = r.x; x[1] = r.y; x[2] = r.z; x[3] = r.w;
}
template <>
__device__ __forceinline__ void load4<__nv_bfloat16>(const __nv_bfloat16* p, float* x) {
    const uint2 r = *reinterpret_cast<const uint2*>(p);
    x[0] = __uint_as_float(r.x << 16); x[1] = __uint_as_float(r.x & 0xFFFF0000u);
    x[2] = __uint_as_float(r.y << 16); x[3] = __uint_as_float(r.y & 0xFFFF0000u);
}

// ---- kernel ---------------------------------------------------------------
template <typename T, typename OutT>
__global__ void __launch_bounds__(NTHREADS, 1)
    fused_tma_kernel(const __grid_constant__ Maps maps, const __grid_constant__ TmaParams p,
                     const __grid_constant__ IsoParams iso) {
    using G = TGeom<T>;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int K = iso.K;
    const int kslots = (K + 1) / 2;
    // carve-up
    unsigned char* stages = smem;
    uint64_t* full = reinterpret_cast<uint64_t*>(stages + NSTAGE * G::STAGE_BYTES);
    uint64_t* empty = full + NSTAGE;
    uint32_t* abort_flag = reinterpret_cast<uint32_t*>(empty + NSTAGE);
    float* part1 = reinterpret_cast<float*>(abort_flag + 4);  // [NG][16] split-1 partial sums
    float* ru = part1 + G::NG * 16;                           // [3 planes][2 slots][NCOLW]
    float* rv = ru + 6 * G::NCOLW;                            // [3 planes][3 slots][NCOLW]
    float* pp = rv + 9 * G::NCOLW;                            // [kslots][2][kOwnG][4]
    float* pq = pp + kslots * 2 * kOwnG * 4;
    uint32_t* pb = reinterpret_cast<uint32_t*>(pq + kslots * 2 * kOwnG * 4);
    volatile uint32_t* abortv = abort_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int H = p.H, W = p.W, M = p.M, Hc = H - 1, Wc = W - 1;
    const int c0 = blockIdx.x * TW;
    const int ty = blockIdx.y;
    const int r0 = (int)(((int64_t)ty * Hc) / p.n_ty);
    const int r1 = (int)(((int64_t)(ty + 1) * Hc) / p.n_ty);
    const bool down = (ty & 1) == 0;
    const int jfirst = down ? max(r0 - 1, 0) : min(r1 + 1, H - 1);
    const int jlast = down ? min(r1 + 1, H - 1) : max(r0 - 1, 0);
    const int nsteps = (down ? jlast - jfirst : jfirst - jlast) + 1;
    const int nq = (M + MB - 1) / MB;

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), NCONS / 32);
        }
        *abort_flag = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == NCONS / 32) {
        // ============================ producer ============================
        if (lane == 0) {
            int n = 0;
            for (int step = 0; step < nsteps; ++step) {
                const int j = down ? jfirst + step : jfirst - step;
                const bool needU = j >= r0 && j <= r1;
                for (int q = 0; q < nq; ++q, ++n) {
                    const int st = n % NSTAGE;
                    const uint32_t par = ((n / NSTAGE) & 1) ^ 1;
                    if (!mbar_wait(smem_u32(&empty[st]), par, abortv)) continue;
                    const uint32_t fb = smem_u32(&full[st]);
                    mbar_expect_tx(fb, needU ? G::STAGE_BYTES : G::COMP_BYTES);
                    const uint32_t dst = smem_u32(stages + st * G::STAGE_BYTES);
                    const int x = c0 - G::WOFF;
                    if (needU) {
                        tma_load_3d(dst, &maps.ua, x, j, q * MB, fb);
                        tma_load_3d(dst + MB * G::BXA * G::ESZ, &maps.ub, x + G::BXA, j, q * MB, fb);
                    }
                    tma_load_3d(dst + G::COMP_BYTES, &maps.va, x, j, q * MB, fb);
                    tma_load_3d(dst + G::COMP_BYTES + MB * G::BXA * G::ESZ, &maps.vb, x + G::BXA, j, q * MB, fb);
                }
            }
            if (*abortv) {  // drain: let every issued copy land before the CTA exits
                const int total = n;
                for (int k = (total > NSTAGE ? total - NSTAGE : 0); k < total; ++k) {
                    const uint32_t fb = smem_u32(&full[k % NSTAGE]);
                    const long long t0 = clock64();
                    while (!mbar_try(fb, (k / NSTAGE) & 1) && clock64() - t0 < kWaitBudget) {
                    }
                }
            }
        }
        return;
    }

    // ============================== consumers ==============================
    const bool stat_thread = tid < 2 * G::NG;
    const int ss = tid / G::NG;  // member split of the stage (0: first half, 1: second half)
    const int g = tid % G::NG;   // window column group
    const int mlo = ss * (MB / 2), mhi = mlo + MB / 2;
    const int ga = g * 4;        // first window column of the group
    const bool inA = ga < G::BXA;
    const float fm = (float)M, fdof = (float)(M - p.ddof);

    bool have_prev = false;
    int n = 0;
    for (int step = 0; step < nsteps; ++step) {
        const int j = down ? jfirst + step : jfirst - step;
        const bool needU = j >= r0 && j <= r1;
        float x0u[4] = {0.f, 0.f, 0.f, 0.f}, x0v[4] = {0.f, 0.f, 0.f, 0.f};
        float s1u[4] = {0.f, 0.f, 0.f, 0.f}, s2u[4] = {0.f, 0.f, 0.f, 0.f};
        float s1v[4] = {0.f, 0.f, 0.f, 0.f}, s2v[4] = {0.f, 0.f, 0.f, 0.f};
        for (int q = 0; q < nq; ++q, ++n) {
            const int st = n % NSTAGE;
            const bool ok = mbar_wait(smem_u32(&full[st]), (n / NSTAGE) & 1, abortv);
            if (ok && stat_thread) {
                const T* ub = reinterpret_cast<const T*>(stages + st * G::STAGE_BYTES);
                const T* vb = reinterpret_cast<const T*>(stages + st * G::STAGE_BYTES + G::COMP_BYTES);
                // element (member i, window column c) of a component block
                auto at = [&](const T* base, int i) {
                    return inA ? base + i * G::BXA + ga : base + MB * G::BXA + i * G::BXB + (ga - G::BXA);
                };
                if (q == 0) {
                    if (needU) load4<T>(at(ub, 0), x0u);
                    load4<T>(at(vb, 0), x0v);
                }
                const int mvalid = M - q * MB;
#pragma unroll
                for (int i = mlo; i < mhi; ++i) {
                    if (i < mvalid) {
                        float a[4], b[4];
                        if (needU) {
                            load4<T>(at(ub, i), a);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float d = a[e] - x0u[e];
                                s1u[e] += d;
                                s2u[e] = fmaf(d, d, s2u[e]);
                            }
                        }
                        load4<T>(at(vb, i), b);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float d = b[e] - x0v[e];
                            s1v[e] += d;
                            s2v[e] = fmaf(d, d, s2v[e]);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0 && ok) mbar_arrive(smem_u32(&empty[st]));
        }
        // combine the two member splits into (x0, delta, var) rings
        if (stat_thread && ss == 1) {
            float* pt = part1 + g * 16;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                pt[e] = s1u[e]; pt[4 + e] = s2u[e]; pt[8 + e] = s1v[e]; pt[12 + e] = s2v[e];
            }
        }
        named_sync(1, NCONS);
        if (stat_thread && ss == 0) {
            const float* pt = part1 + g * 16;
            const int su = j & 1, sv = j % 3;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float a1 = s1u[e] + pt[e], a2 = s2u[e] + pt[4 + e];
                const float b1 = s1v[e] + pt[8 + e], b2 = s2v[e] + pt[12 + e];
                const float du = a1 / fm, dv = b1 / fm;
                float vu = (a2 - a1 * du) / fdof, vv = (b2 - b1 * dv) / fdof;
                if (vu < 0.f) vu = 0.f;
                if (vv < 0.f) vv = 0.f;
                const int col = ga + e;
                if (needU) {
                    ru[(0 * 2 + su) * G::NCOLW + col] = x0u[e];
                    ru[(1 * 2 + su) * G::NCOLW + col] = du;
                    ru[(2 * 2 + su) * G::NCOLW + col] = vu;
                }
                rv[(0 * 3 + sv) * G::NCOLW + col] = x0v[e];
                rv[(1 * 3 + sv) * G::NCOLW + col] = dv;
                rv[(2 * 3 + sv) * G::NCOLW + col] = vv;
            }
        }
        named_sync(1, NCONS);
        // divergence rows completed by row j, then their cells
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
            if (tid < 2 * kOwnG) {
                const int ks = tid / kOwnG;  // isovalue split
                const int og = tid % kOwnG;  // own group: cells c0 + 4 og .. + 3
                const int su = d & 1;
                const int jlo = d > 0 ? d - 1 : 0, jhi = d < H - 1 ? d + 1 : H - 1;
                const float sy = (jhi - jlo == 2) ? p.sp.sy2 : p.sp.sy1;
                const float syq = (jhi - jlo == 2) ? p.sp.sy2q : p.sp.sy1q;
                const int vlo = jlo % 3, vhi = jhi % 3;
                float mu[5], var[5];
#pragma unroll
                for (int e = 0; e <= 4; ++e) {
                    const int ic = min(c0 + 4 * og + e, W - 1);
                    const int ilo = ic > 0 ? ic - 1 : 0, ihi = ic < W - 1 ? ic + 1 : W - 1;
                    const float sx = (ihi - ilo == 2) ? p.sp.sx2 : p.sp.sx1;
                    const float sxq = (ihi - ilo == 2) ? p.sp.sx2q : p.sp.sx1q;
                    const int base = c0 - G::WOFF;
                    const int lcl = ilo - base, lch = ihi - base, lc = ic - base;
                    const float* rx0 = ru + (0 * 2 + su) * G::NCOLW;
                    const float* rdl = ru + (1 * 2 + su) * G::NCOLW;
                    const float* rvr = ru + (2 * 2 + su) * G::NCOLW;
                    const float du = (rx0[lch] - rx0[lcl]) + (rdl[lch] - rdl[lcl]);
                    const float dv = (rv[(0 * 3 + vhi) * G::NCOLW + lc] - rv[(0 * 3 + vlo) * G::NCOLW + lc]) +
                                     (rv[(1 * 3 + vhi) * G::NCOLW + lc] - rv[(1 * 3 + vlo) * G::NCOLW + lc]);
                    const float vu = rvr[lch] + rvr[lcl];
                    const float vv = rv[(2 * 3 + vhi) * G::NCOLW + lc] + rv[(2 * 3 + vlo) * G::NCOLW + lc];
                    mu[e] = fmaf(du, sx, dv * sy);
                    var[e] = fmaf(vu, sxq, vv * syq);
                }
                const int cr = down ? d - 1 : d;
                const int cbase = c0 + 4 * og;
                for (int t = 0, k = ks; k < K; ++t, k += 2) {
                    const float c = iso.c[k];
                    float pr[5], qr[5];
                    uint32_t bits = 0;
#pragma unroll
                    for (int e = 0; e <= 4; ++e) {
                        below_above(mu[e], var[e], c, pr[e], qr[e]);
                        bits |= (uint32_t)(mu[e] < c) << e;
                    }
                    float ph[4], qh[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        ph[e] = pr[e] * pr[e + 1];
                        qh[e] = qr[e] * qr[e + 1];
                    }
                    const int slot = (t * 2 + ks) * kOwnG + og;
                    float4* PP = reinterpret_cast<float4*>(pp) + slot;
                    float4* PQ = reinterpret_cast<float4*>(pq) + slot;
                    if (have_prev) {
                        const float4 a = *PP, b = *PQ;
                        const float pa[4] = {a.x, a.y, a.z, a.w}, qa[4] = {b.x, b.y, b.z, b.w};
                        const uint32_t bp = pb[slot];
                        const int64_t obase = ((int64_t)(p.kbase + k) * Hc + cr) * Wc;
                        OutT* out = reinterpret_cast<OutT*>(p.out);
                        uint32_t nib = 0;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int col = cbase + e;
                            if (col < Wc) {
                                const float lcp = 1.0f - pa[e] * ph[e] - qa[e] * qh[e];
                                out[obase + col] = to_out<OutT>(clamp01(lcp));
                                const uint32_t four = ((bp >> e) & 3u) | (((bits >> e) & 3u) << 2);
                                nib |= (uint32_t)(four != 0u && four != 15u) << e;
                            }
                        }
                        if (p.mask) {
                            uint32_t val = nib << (4 * (lane & 7));
                            val |= __shfl_xor_sync(0xFFFFFFFFu, val, 1);
                            val |= __shfl_xor_sync(0xFFFFFFFFu, val, 2);
                            val |= __shfl_xor_sync(0xFFFFFFFFu, val, 4);
                            const int word = cbase >> 5;
                            if ((lane & 7) == 0 && word < p.n_words)
                                p.mask[((int64_t)(p.kbase + k) * Hc + cr) * p.n_words + word] = val;
                        }
                    }
                    *PP = make_float4(ph[0], ph[1], ph[2], ph[3]);
                    *PQ = make_float4(qh[0], qh[1], qh[2], qh[3]);
                    pb[slot] = bits;
                }
            }
            have_prev = true;
        }
    }
}

// ---- host ------------------------------------------------------------------
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}

template <typename T>
bool make_map(CUtensorMap* m, const void* base, int W, int H, int M, int64_t stride, int box_x) {
    EncodeFn enc = encode_fn();
    if (!enc) return false;
    const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)M};
    const cuuint64_t strides[2] = {(cuuint64_t)W * sizeof(T), (cuuint64_t)stride * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, 1u, (cuuint32_t)MB};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return enc(m, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, typename OutT>
lcp_status launch(const void* u, const void* v, int64_t stride, TmaParams p, const float* iso, int K,
                  cudaStream_t st) {
    using G = TGeom<T>;
    Maps maps;
    if (!make_map<T>(&maps.ua, u, p.W, p.H, p.M, stride, G::BXA) ||
        !make_map<T>(&maps.ub, u, p.W, p.H, p.M, stride, G::BXB) ||
        !make_map<T>(&maps.va, v, p.W, p.H, p.M, stride, G::BXA) ||
        !make_map<T>(&maps.vb, v, p.W, p.H, p.M, stride, G::BXB))
        return LCP_ERR_UNSUPPORTED;
    auto kern = fused_tma_kernel<T, OutT>;
    const int kmax_pass = K < kMaxKPass ? K : kMaxKPass;
    const int kslots = (kmax_pass + 1) / 2;
    const size_t smem = (size_t)NSTAGE * G::STAGE_BYTES + 2 * NSTAGE * 8 + 16 +
                        4 * ((size_t)G::NG * 16 + 15 * G::NCOLW + (size_t)kslots * 2 * kOwnG * 9);
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
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTHREADS, smem) != cudaSuccess || per_sm < 1)
        return fail(LCP_ERR_CUDA, "lcp_fused: TMA kernel does not fit on an SM (smem %zu)", smem);
    const int Hc = p.H - 1, Wc = p.W - 1;
    const int n_tx = (Wc + TW - 1) / TW;
    long n_ty = (long)per_sm * num_sms() / n_tx;
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
        kern<<<grid, NTHREADS, smem, st>>>(maps, p, ip);
        lcp_status s = check_launch("lcp_fused (TMA)");
        if (s != LCP_OK) return s;
    }
    return LCP_OK;
}

}  // namespace

// Runs the TMA variant if the layout allows it (16-byte aligned planes, row and
// member strides multiples of 16 bytes); LCP_ERR_UNSUPPORTED means "use the
// register-streaming kernel" and has enqueued nothing.
lcp_status fused_tma(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W, int64_t stride, int ddof,
                     double dx, double dy, const float* iso, int K, void* out, lcp_dtype out_dtype, uint32_t* mask,
                     cudaStream_t st) {
    const int esz = in_dtype == LCP_F32 ? 4 : 2;
    if (!aligned16(u) || !aligned16(v) || ((int64_t)W * esz) % 16 || (stride * esz) % 16) return LCP_ERR_UNSUPPORTED;
    if (H > (1 << 30) || M > (1 << 30)) return LCP_ERR_UNSUPPORTED;
    TmaParams p;
    p.M = M; p.H = H; p.W = W; p.ddof = ddof;
    p.sp = make_spacing(dx, dy);
    p.out = out;
    p.mask = mask;
    p.n_words = (W - 1 + 31) / 32;
    p.n_ty = 1;
    p.kbase = 0;
    const bool f16 = out_dtype == LCP_F16;
    if (in_dtype == LCP_F32)
        return f16 ? launch<float, __half>(u, v, stride, p, iso, K, st) : launch<float, float>(u, v, stride, p, iso, K, st);
    return f16 ? launch<__nv_bfloat16, __half>(u, v, stride, p, iso, K, st)
               : launch<__nv_bfloat16, float>(u, v, stride, p, iso, K, st);
}

}  // namespace lcp

namespace lcp {
uint32_t read_tma_status(bool reset) {
    uint32_t f = 0;
    cudaMemcpyFromSymbol(&f, g_fused_status, sizeof(f));
    if (reset) {
        const uint32_t z = 0;
        cudaMemcpyToSymbol(g_fused_status, &z, sizeof(z));
    }
    return f;
}
}  // namespace lcp
