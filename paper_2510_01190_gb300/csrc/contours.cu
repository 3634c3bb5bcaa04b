// Isocontour segments (marching squares) of a scalar field -- the mean-field
// divergence of Fig. 1a / Fig. 3c -- or of every member's divergence -- the
// spaghetti plot of Fig. 1b -- compacted into one segment list in key order in
// a single pass.
//
// A tile of 256 threads takes a ticket (its position in start order) and 992
// consecutive items (cells, or member cells); in round e lane l < 31 of warp w
// takes item 124 w + 31 e + l, so that the segments of one round fill one
// contiguous output range in lane order and the warp's stores coalesce; the
// right corners of a cell are the next lane's left ones, by shuffle (lane 31
// evaluates the 32nd corner column).  Per
// cell the "below" bits of each corner for all isovalues form one mask, the
// crossing edges are the XORs of neighbouring masks, and a cell has half as
// many segments as crossing edges, so counting needs no per-isovalue case
// analysis.  The tile counts its segments, scans the counts, and finds its
// output offset by
// decoupled look-back (Merrill and Garland, "Single-pass Parallel Prefix Scan
// with Decoupled Look-back", 2016): it publishes its aggregate, and warp 0
// reads the flags of the 32 preceding tiles at a time until it meets one that
// holds an inclusive prefix.  Every tile it waits for took its ticket earlier,
// so it is running and publishes without waiting itself; each wait is still
// bounded (lcp_set_wait_budget, ~2 s of clock by default), after which the tile counts the missing flag as 0,
// sets a bit in the library's device status and carries on.  Then each warp
// lays a round's segments out in shared memory as small descriptors in their
// final order, shares them evenly among its lanes (a cell can have up to 2K
// segments, so per-cell emission would leave most lanes idle) and writes them
// with contiguous streaming stores (evict-first: the output must not push the
// members out of L2): in key order, the same on every run.
//
// The member divergence uses Eq. 1 in fp32 with each operation rounded to
// nearest in a fixed order (within 5 u (|gx| + |gy|) of the exact value, u =
// 2^-24, gx and gy its two terms), and the saddle decider's centre value
// ((f0 + f1) + (f2 + f3)) / 4 is formed in fp32 the same way, so the results
// are deterministic and differ from the exact marching squares only where a
// corner or a saddle centre lies within that rounding of the isovalue.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "lcp_common.cuh"

namespace lcp {

__device__ unsigned int g_contour_status;  // bit 0: a look-back wait gave up

namespace {

constexpr int kCT = 256;                 // threads per tile
constexpr int kCI = 4;                   // rounds per tile
constexpr int kIW = 31;                  // items per warp and round (lane 31 supplies the 32nd corner column)
constexpr int kWin = 512;                // segment descriptors staged per warp and window
constexpr int64_t kTile = (kCT / 32) * kCI * kIW;
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr unsigned long long kAgg = 1ull << 62, kPre = 2ull << 62, kVal = (1ull << 62) - 1;

struct ContourParams {
    const float* f;          // field mode: [H][W]
    const void* u;           // member mode
    const void* v;
    int64_t stride;
    int M, H, W, K;
    float sx1, sx2, sy1, sy2;
    int64_t n_items;         // cells (x members)
    float4* seg;
    long long* key;
    int64_t capacity;
    unsigned long long* count;
    unsigned long long* flags;  // [tiles] look-back words (zeroed before the launch)
    unsigned int* ticket;
    long long budget;           // clock cycles before a look-back wait gives up
};

__device__ __forceinline__ unsigned long long ld_acq64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ float ldv(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p) {
    return __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p)) << 16);
}

// value at vertex (i, j) of item set m: the field, or member m's fp32 divergence
// (clamped neighbours: the one-sided stencil at the edges)
template <int MODE>
__device__ __forceinline__ float corner(const ContourParams& p, int64_t m, int j, int i) {
    const int64_t o = (int64_t)j * p.W + i;
    if (MODE == 0) return __ldg(p.f + o);
    using T = typename std::conditional<MODE == 1, float, __nv_bfloat16>::type;
    const int64_t base = m * p.stride + o;
    const T* up = reinterpret_cast<const T*>(p.u) + base;
    const T* vp = reinterpret_cast<const T*>(p.v) + base;
    const int dl = i > 0 ? -1 : 0, dh = i < p.W - 1 ? 1 : 0;
    const int dd = j > 0 ? -p.W : 0, du = j < p.H - 1 ? p.W : 0;
    const float sx = dh - dl == 2 ? p.sx2 : p.sx1, sy = du - dd == 2 * p.W ? p.sy2 : p.sy1;
    const float gx = __fmul_rn(__fsub_rn(ldv(up + dh), ldv(up + dl)), sx);
    const float gy = __fmul_rn(__fsub_rn(ldv(vp + du), ldv(vp + dd)), sy);
    return __fadd_rn(gx, gy);
}

// crossing point of edge e of cell (i, j), interpolated from the edge's
// lower-coordinate vertex; selects instead of branches, so that lanes on
// different edges do not diverge.  E0: v0 -> v1 (+x), E1: v1 -> v2 (+y),
// E2: v3 -> v2 (+x), E3: v0 -> v3 (+y).
__device__ __forceinline__ float2 edge_point(const float (&f)[4], int e, float c, float fi, float fj) {
    const float from = e == 1 ? f[1] : (e == 2 ? f[3] : f[0]);
    const float to = e == 3 ? f[3] : (e == 0 ? f[1] : f[2]);
    const float t = __fdividef(__fsub_rn(c, from), __fsub_rn(to, from));
    const bool horiz = (e & 1) == 0;
    const float x0 = fi + (e == 1 ? 1.f : 0.f), y0 = fj + (e == 2 ? 1.f : 0.f);  // exact (grid indices < 2^24)
    return horiz ? make_float2(__fadd_rn(x0, t), y0) : make_float2(x0, __fadd_rn(y0, t));
}

// decode item n into (set m, row j, column i)
__device__ __forceinline__ void decode(int64_t n, int64_t per_m, int Wc, int64_t& m, int& j, int& i) {
    m = n / per_m;
    const int64_t r = n - m * per_m;
    j = (int)(r / Wc);
    i = (int)(r - (int64_t)j * Wc);
}

// the four corners of item (m, j, i) of this lane: the left ones (v0, v3) its
// own, the right ones (v1, v2) the next lane's left ones unless that lane holds
// another row (or nothing), in which case own_right asks for them here
template <int MODE>
__device__ __forceinline__ void corners(const ContourParams& p, bool load_left, bool own_right, int64_t m, int j, int i,
                                        float (&f)[4]) {
    float a = 0.f, d = 0.f;
    if (load_left) {
        a = corner<MODE>(p, m, j, i);
        d = corner<MODE>(p, m, j + 1, i);
    }
    float b = __shfl_down_sync(kFull, a, 1), c = __shfl_down_sync(kFull, d, 1);
    if (own_right) {
        b = corner<MODE>(p, m, j, i + 1);
        c = corner<MODE>(p, m, j + 1, i + 1);
    }
    f[0] = a;
    f[1] = b;
    f[2] = c;
    f[3] = d;
}

// per-isovalue "below" bits of the four corners, and the edges that cross (as
// K-bit masks, MT = 32 or 64 bits: bit k of e[0] set when E0 crosses isovalue k,
// and so on); the isovalues come from shared memory, where lanes may index them
// divergently
template <typename MT>
__device__ __forceinline__ void edge_masks(const float (&f)[4], const float* iso, int K, MT (&bm)[4], MT (&e)[4]) {
#pragma unroll
    for (int v = 0; v < 4; ++v) bm[v] = 0;
    MT bit = 1;
    for (int k = 0; k < K; ++k, bit <<= 1) {
        const float c = iso[k];
#pragma unroll
        for (int v = 0; v < 4; ++v) bm[v] |= f[v] < c ? bit : (MT)0;
    }
    e[0] = bm[0] ^ bm[1];
    e[1] = bm[1] ^ bm[2];
    e[2] = bm[3] ^ bm[2];
    e[3] = bm[0] ^ bm[3];
}

// a cell's two isovalue masks (with a crossing, saddles) as kept in shared memory
template <typename MT>
struct MaskPair;
template <>
struct MaskPair<uint32_t> {
    using T = uint2;
    static __device__ __forceinline__ T pack(uint32_t a, uint32_t s) { return make_uint2(a, s); }
};
template <>
struct MaskPair<unsigned long long> {
    using T = ulonglong2;
    static __device__ __forceinline__ T pack(unsigned long long a, unsigned long long s) { return make_ulonglong2(a, s); }
};

__device__ __forceinline__ int popc_m(uint32_t x) { return __popc(x); }
__device__ __forceinline__ int popc_m(unsigned long long x) { return __popcll(x); }
__device__ __forceinline__ int ffs_m(uint32_t x) { return __ffs(x); }
__device__ __forceinline__ int ffs_m(unsigned long long x) { return __ffsll((long long)x); }

// a tile's scratch, in dynamic shared memory
template <typename MT>
struct ContourSmem {
    float4 cf[kCI][kCT];                       // corners of each lane's cell, per round
    typename MaskPair<MT>::T cm[kCI][kCT];     // its masks: isovalues with a crossing, saddles
    float2 cij[kCI][kCT];                      // its (i, j) as floats
    int lex[kCI][kCT];                         // lane offset within its warp's round
    int desc[kCT / 32][kWin];                  // a warp's window: (owner lane, isovalue, sub-segment)
    int rtot[kCI][kCT / 32];                   // segments of a warp's round
    int warp[kCT / 32];
    float iso[kMaxIsoPerLaunch];
    unsigned long long excl;
    unsigned int tile;
};

template <int MODE, typename MT>
__global__ void __launch_bounds__(kCT) contour_kernel(const __grid_constant__ ContourParams p,
                                                      const __grid_constant__ IsoParams iso) {
    extern __shared__ __align__(16) unsigned char contour_smem[];
    ContourSmem<MT>& S = *reinterpret_cast<ContourSmem<MT>*>(contour_smem);
    unsigned int& s_tile = S.tile;
    int* const s_warp = S.warp;
    unsigned long long& s_excl = S.excl;
    auto& s_lex = S.lex;
    auto& s_rtot = S.rtot;
    auto& s_desc = S.desc;
    auto& s_cf = S.cf;
    auto& s_cij = S.cij;
    auto& s_cm = S.cm;
    float* const s_iso = S.iso;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t < iso.K) s_iso[t] = iso.c[t];
    if (t == 0) s_tile = atomicAdd(p.ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int Wc = p.W - 1, Hc = p.H - 1;
    const int64_t per_m = (int64_t)Hc * Wc;
    // warp w owns items [wbase, wbase + 31 kCI); round e gives lane l < 31 item wbase + 31 e + l, so
    // that a round's segments fill one contiguous output range in lane order and its stores coalesce;
    // lane 31 evaluates the next item's left corners, the right corners of lane 30's cell
    const int64_t wbase = tile * kTile + (int64_t)warp * kIW * kCI;
    const bool item_lane = lane < kIW;
    int64_t m0 = 0;
    int j0 = 0, i0 = 0;
    decode(wbase + lane, per_m, Wc, m0, j0, i0);
    auto advance = [&](int64_t& m, int& j, int& i) {
        i += kIW;
        while (i >= Wc) {
            i -= Wc;
            if (++j == Hc) {
                j = 0;
                ++m;
            }
        }
    };
    // phase 1: segment counts (a cell has half as many segments as crossing edges)
    int wtot = 0;
    {
        int64_t m = m0;
        int j = j0, i = i0;
#pragma unroll
        for (int e = 0; e < kCI; ++e) {
            if (e > 0) advance(m, j, i);
            const int64_t n = wbase + kIW * e + lane;
            const bool in_range = n < p.n_items;
            const bool valid = item_lane && in_range;
            float f[4];
            corners<MODE>(p, in_range, valid && (i == Wc - 1 || n + 1 >= p.n_items), m, j, i, f);
            int cnt = 0;
            MT act = 0, sad = 0;
            if (valid && !(isnan(f[0]) || isnan(f[1]) || isnan(f[2]) || isnan(f[3]))) {
                MT bm[4], em[4];
                edge_masks(f, s_iso, p.K, bm, em);
                act = em[0] | em[1] | em[2] | em[3];  // isovalues with a crossing
                sad = em[0] & em[1] & em[2] & em[3];  // ... with all four edges crossing
                cnt = popc_m(act) + popc_m(sad);      // one segment each, two for a saddle
            }
            s_cf[e][t] = make_float4(f[0], f[1], f[2], f[3]);
            s_cij[e][t] = make_float2((float)i, (float)j);
            s_cm[e][t] = MaskPair<MT>::pack(act, sad);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            s_lex[e][t] = incl - cnt;
            const int rt = __shfl_sync(kFull, incl, 31);
            if (lane == 0) s_rtot[e][warp] = rt;
            wtot += rt;
        }
    }
    if (lane == 0) s_warp[warp] = wtot;
    __syncthreads();
    if (warp == 0) {
        const int wv = lane < kCT / 32 ? s_warp[lane] : 0;
        int wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += y;
        }
        const unsigned long long agg = (unsigned long long)__shfl_sync(kFull, wi, kCT / 32 - 1);
        if (lane < kCT / 32) s_warp[lane] = wi - wv;  // exclusive warp offsets
        // decoupled look-back
        unsigned long long excl = 0;
        if (lane == 0) st_rel64(p.flags + tile, (tile == 0 ? kPre : kAgg) | agg);
        if (tile > 0) {
            int64_t base = tile - 1;
            for (;;) {
                const int64_t q = base - lane;
                unsigned long long fl = kPre;  // before the first tile: an inclusive prefix of 0
                if (q >= 0) {
                    const long long t0 = clock64();
                    fl = ld_acq64(p.flags + q);
                    while ((fl >> 62) == 0) {
                        if (clock64() - t0 > p.budget) {
                            atomicOr(&g_contour_status, 1u);
                            fl = kPre;
                            break;
                        }
                        __nanosleep(64);
                        fl = ld_acq64(p.flags + q);
                    }
                }
                const unsigned pre = __ballot_sync(kFull, (fl >> 62) == 2);
                unsigned long long val = fl & kVal;
                if (pre && lane > __ffs(pre) - 1) val = 0;  // lanes past the nearest prefix
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(kFull, val, o);
                excl += val;
                if (pre) break;
                base -= 32;
            }
            if (lane == 0) st_rel64(p.flags + tile, kPre | (excl + agg));
        }
        if (lane == 0) {
            s_excl = excl;
            if ((tile + 1) * kTile >= p.n_items) *p.count = excl + agg;  // the last tile knows the total
        }
    }
    __syncthreads();
    // phase 3: the segments in key order, round by round, from the cells kept in shared memory.  Each
    // lane writes one small descriptor per segment at the segment's final position in the warp's
    // window; then the lanes share the window's segments evenly, compute them and store them
    // contiguously (streaming stores).
    int64_t rbase = (int64_t)s_excl + s_warp[warp];
#pragma unroll 1
    for (int e = 0; e < kCI; ++e) {
        const int rt = s_rtot[e][warp];
        const int64_t round_base = rbase;
        rbase += rt;
        if (rt == 0) continue;  // uniform: no lane of this warp has a segment in this round
        const int lex = s_lex[e][t];
        const MT active0 = s_cm[e][t].x, saddles = s_cm[e][t].y;
        const int cnt = popc_m(active0) + popc_m(saddles);
        const long long kb_round = (long long)(wbase + kIW * e) * p.K * 2;  // key of lane 0's item, isovalue 0
        for (int w0 = 0; w0 < rt; w0 += kWin) {
            if (cnt > 0 && lex < w0 + kWin && lex + cnt > w0) {
                MT active = active0;
                int idx = lex;
                while (active && idx < w0 + kWin) {
                    const MT low = active & (~active + 1);
                    active ^= low;
                    const int k = ffs_m(low) - 1;
                    const int d = (lane << 8) | (k << 1);
                    if (idx >= w0) s_desc[warp][idx - w0] = d;
                    ++idx;
                    if (saddles & low) {
                        if (idx >= w0 && idx < w0 + kWin) s_desc[warp][idx - w0] = d | 1;
                        ++idx;
                    }
                }
            }
            __syncwarp();
            const int n_win = min(kWin, rt - w0);
            for (int q = lane; q < n_win; q += 32) {
                const int d = s_desc[warp][q];
                const int owner = d >> 8, k = (d >> 1) & 127, sub = d & 1;
                const float4 cf = s_cf[e][warp * 32 + owner];
                const float g[4] = {cf.x, cf.y, cf.z, cf.w};
                const float2 ij = s_cij[e][warp * 32 + owner];
                const float c = s_iso[k];
                const int b0 = g[0] < c, b1 = g[1] < c, b2 = g[2] < c, b3 = g[3] < c;
                const int cross = (b0 ^ b1) | ((b1 ^ b2) << 1) | ((b3 ^ b2) << 2) | ((b0 ^ b3) << 3);
                // one segment joins the lowest and the highest crossing edge; a saddle (all four)
                // pairs them by the fp32 centre value
                int ea = __ffs(cross) - 1, eb = 31 - __clz(cross);
                if (cross == 15) {
                    const float cen = __fmul_rn(__fadd_rn(__fadd_rn(g[0], g[1]), __fadd_rn(g[2], g[3])), 0.25f);
                    const bool with_v0 = (cen < c) == (b0 != 0);
                    ea = sub ? (with_v0 ? 2 : 1) : 0;
                    eb = sub ? (with_v0 ? 3 : 2) : (with_v0 ? 1 : 3);
                }
                const int64_t gq = round_base + w0 + q;
                if (gq < p.capacity) {
                    const float2 a = edge_point(g, ea, c, ij.x, ij.y), b = edge_point(g, eb, c, ij.x, ij.y);
                    __stcs(p.seg + gq, make_float4(a.x, a.y, b.x, b.y));
                    // the key of item n = ((m (H-1) + j) (W-1) + i): (n K + k) 2 + sub
                    if (p.key) __stcs(p.key + gq, kb_round + (long long)((owner * p.K + k) * 2 + sub));
                }
            }
            __syncwarp();
        }
    }
}

template <int MODE, typename MT>
lcp_status launch_contour(const ContourParams& p, const IsoParams& ip, int64_t tiles, cudaStream_t st) {
    constexpr size_t smem = sizeof(ContourSmem<MT>);
    static std::mutex mu;
    static bool set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && !set[dev]) {
            if (cudaFuncSetAttribute(contour_kernel<MODE, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess) {
                cudaGetLastError();
                return fail(LCP_ERR_CUDA, "contours: %zu bytes of shared memory not available", smem);
            }
            set[dev] = true;
        }
    }
    contour_kernel<MODE, MT><<<(unsigned)tiles, kCT, smem, st>>>(p, ip);
    return LCP_OK;
}

// skip_first (the failure-path probe only): the ticket starts at 1, so tile 0
// never runs and the grid has one block fewer.
lcp_status run_contours(int mode, const ContourParams& p0, const float* iso, int K, void* ws, size_t ws_bytes,
                        cudaStream_t st, const char* fn, bool skip_first = false) {
    ContourParams p = p0;
    p.budget = wait_budget_cycles();
    const int64_t tiles = (p.n_items + kTile - 1) / kTile;
    if (skip_first && tiles < 2) return fail(LCP_ERR_ARG, "%s: needs at least two tiles (%lld cells)", fn, (long long)kTile + 1);
    const size_t need = 256 + (size_t)std::max<int64_t>(tiles, 1) * 8;
    if (!ws || ((uintptr_t)ws & 255)) return fail(LCP_ERR_ARG, "%s: need a 256-byte aligned workspace", fn);
    if (ws_bytes < need) return fail(LCP_ERR_ARG, "%s: workspace too small (%zu < %zu bytes)", fn, ws_bytes, need);
    if (tiles > 0x7FFFFFFFll) return fail(LCP_ERR_UNSUPPORTED, "%s: too many cells", fn);
    p.ticket = reinterpret_cast<unsigned int*>(ws);
    p.flags = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ws) + 256);
    if (cudaMemsetAsync(ws, 0, need, st) != cudaSuccess) return fail(LCP_ERR_CUDA, "%s: workspace clear failed", fn);
    if (skip_first && cudaMemsetAsync(ws, 1, 1, st) != cudaSuccess)  // ticket = 1 (little-endian low byte)
        return fail(LCP_ERR_CUDA, "%s: ticket set failed", fn);
    const int64_t blocks = skip_first ? tiles - 1 : tiles;
    if (tiles == 0) {
        if (cudaMemsetAsync(p.count, 0, sizeof(unsigned long long), st) != cudaSuccess)
            return fail(LCP_ERR_CUDA, "%s: count clear failed", fn);
        return LCP_OK;
    }
    IsoParams ip;
    ip.K = K;
    for (int k = 0; k < K; ++k) ip.c[k] = iso[k];
    p.K = K;
    const bool narrow = K <= 32;  // 32-bit isovalue masks
    lcp_status s = LCP_OK;
    switch (mode) {
        case 0:
            s = narrow ? launch_contour<0, uint32_t>(p, ip, blocks, st) : launch_contour<0, unsigned long long>(p, ip, blocks, st);
            break;
        case 1:
            s = narrow ? launch_contour<1, uint32_t>(p, ip, blocks, st) : launch_contour<1, unsigned long long>(p, ip, blocks, st);
            break;
        default:
            s = narrow ? launch_contour<2, uint32_t>(p, ip, blocks, st) : launch_contour<2, unsigned long long>(p, ip, blocks, st);
            break;
    }
    if (s != LCP_OK) return s;
    return check_launch(fn);
}

inline lcp_status check_contour_out(const char* fn, int H, int W, const float* iso, int K, float* seg,
                                    int64_t capacity, unsigned long long* count) {
    if (H >= (1 << 24) || W >= (1 << 24)) return fail(LCP_ERR_UNSUPPORTED, "%s: H, W < 2^24 (fp32 coordinates)", fn);
    lcp_status s = check_iso(fn, iso, K);
    if (s != LCP_OK) return s;
    if (K > kMaxIsoPerLaunch) return fail(LCP_ERR_UNSUPPORTED, "%s: K <= %d", fn, kMaxIsoPerLaunch);
    if (capacity < 0 || (capacity > 0 && !seg)) return fail(LCP_ERR_ARG, "%s: need capacity >= 0 and seg for capacity > 0", fn);
    if ((uintptr_t)seg & 15) return fail(LCP_ERR_ARG, "%s: seg must be 16-byte aligned", fn);
    if (!count || ((uintptr_t)count & 7)) return fail(LCP_ERR_ARG, "%s: need an 8-byte aligned device count", fn);
    return LCP_OK;
}

}  // namespace

uint32_t read_contour_status(bool reset) {
    uint32_t f = 0;
    cudaMemcpyFromSymbol(&f, g_contour_status, sizeof(f));
    if (reset) {
        const uint32_t z = 0;
        cudaMemcpyToSymbol(g_contour_status, &z, sizeof(z));
    }
    return f;
}

}  // namespace lcp

using namespace lcp;

extern "C" size_t lcp_contours_workspace_bytes(int M, int H, int W) {
    if (M < 1 || H < 2 || W < 2) return 0;
    const int64_t items = (int64_t)M * (H - 1) * (W - 1);
    return 256 + (size_t)std::max<int64_t>((items + kTile - 1) / kTile, 1) * 8;
}

namespace {
lcp_status field_contours(const char* fn, bool skip_first, const float* field, int H, int W, const float* iso, int K,
                          float* seg, long long* key, int64_t capacity, unsigned long long* count, void* workspace,
                          size_t workspace_bytes, lcp_stream_t stream) {
    if (!field) return fail(LCP_ERR_ARG, "%s: NULL field", fn);
    if (H < 2 || W < 2) return fail(LCP_ERR_ARG, "%s: need H, W >= 2", fn);
    lcp_status s = check_contour_out(fn, H, W, iso, K, seg, capacity, count);
    if (s != LCP_OK) return s;
    ContourParams p = {};
    p.f = field;
    p.M = 1;
    p.H = H;
    p.W = W;
    p.n_items = (int64_t)(H - 1) * (W - 1);
    p.seg = reinterpret_cast<float4*>(seg);
    p.key = key;
    p.capacity = capacity;
    p.count = count;
    return run_contours(0, p, iso, K, workspace, workspace_bytes, (cudaStream_t)stream, fn, skip_first);
}
}  // namespace

extern "C" lcp_status lcp_contours(const float* field, int H, int W, const float* iso, int K, float* seg, long long* key,
                                   int64_t capacity, unsigned long long* count, void* workspace, size_t workspace_bytes,
                                   lcp_stream_t stream) {
    return field_contours("lcp_contours", false, field, H, W, iso, K, seg, key, capacity, count, workspace,
                          workspace_bytes, stream);
}

extern "C" lcp_status lcp_test_stalled_lookback(const float* field, int H, int W, const float* iso, int K, float* seg,
                                                long long* key, int64_t capacity, unsigned long long* count,
                                                void* workspace, size_t workspace_bytes, lcp_stream_t stream) {
    return field_contours("lcp_test_stalled_lookback", true, field, H, W, iso, K, seg, key, capacity, count, workspace,
                          workspace_bytes, stream);
}

extern "C" lcp_status lcp_member_contours(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                                          int64_t member_stride, double dx, double dy, const float* iso, int K,
                                          float* seg, long long* key, int64_t capacity, unsigned long long* count,
                                          void* workspace, size_t workspace_bytes, lcp_stream_t stream) {
    static const char* fn = "lcp_member_contours";
    lcp_status s = check_members(fn, u, v, in_dtype, M, H, W, member_stride, 0);
    if (s != LCP_OK) return s;
    if ((s = check_spacing(fn, dx, dy)) != LCP_OK) return s;
    if ((s = check_contour_out(fn, H, W, iso, K, seg, capacity, count)) != LCP_OK) return s;
    ContourParams p = {};
    p.u = u;
    p.v = v;
    p.stride = M > 1 ? member_stride : (int64_t)H * W;
    p.M = M;
    p.H = H;
    p.W = W;
    p.sx1 = (float)(1.0 / dx);
    p.sx2 = (float)(0.5 / dx);
    p.sy1 = (float)(1.0 / dy);
    p.sy2 = (float)(0.5 / dy);
    p.n_items = (int64_t)M * (H - 1) * (W - 1);
    p.seg = reinterpret_cast<float4*>(seg);
    p.key = key;
    p.capacity = capacity;
    p.count = count;
    return run_contours(in_dtype == LCP_F32 ? 1 : 2, p, iso, K, workspace, workspace_bytes, (cudaStream_t)stream, fn);
}
