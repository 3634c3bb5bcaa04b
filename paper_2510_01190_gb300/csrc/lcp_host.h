// Host-side helpers of liblcp_gb300: error plumbing, argument checks and the
// internal entry points one translation unit calls in another.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lcp.h"

namespace lcp {

// ---------------------------------------------------------------------------
// Error plumbing (thread-local message behind lcp_last_error)
// ---------------------------------------------------------------------------
lcp_status fail(lcp_status s, const char* fmt, ...);
lcp_status check_launch(const char* what);  // cudaGetLastError after a launch
int num_sms();                              // SM count of the current device (cached per device)
bool aligned16(const void* p);

// Argument checks shared by the entry points that read member planes.
inline lcp_status check_members(const char* fn, const void* u, const void* v, lcp_dtype dt, int M, int H, int W,
                                int64_t stride, int ddof) {
    if (!u || !v) return fail(LCP_ERR_ARG, "%s: u and v must be non-NULL device pointers", fn);
    if (dt != LCP_F32 && dt != LCP_BF16) return fail(LCP_ERR_ARG, "%s: member dtype must be LCP_F32 or LCP_BF16", fn);
    if (H < 2 || W < 2) return fail(LCP_ERR_ARG, "%s: need H >= 2 and W >= 2 (got %d x %d)", fn, H, W);
    if (M < 1) return fail(LCP_ERR_ARG, "%s: need M >= 1 (got %d)", fn, M);
    if (ddof != 0 && ddof != 1) return fail(LCP_ERR_ARG, "%s: ddof must be 0 or 1", fn);
    if (M - ddof < 1) return fail(LCP_ERR_ARG, "%s: need M - ddof >= 1", fn);
    if (M > 1 && stride < (int64_t)H * W) return fail(LCP_ERR_ARG, "%s: member_stride < H*W", fn);
    const size_t esz = dt == LCP_F32 ? 4 : 2;
    if (((uintptr_t)u | (uintptr_t)v) % esz) return fail(LCP_ERR_ARG, "%s: member pointers misaligned", fn);
    return LCP_OK;
}

inline lcp_status check_iso(const char* fn, const float* iso, int K) {
    if (!iso) return fail(LCP_ERR_ARG, "%s: iso must be a non-NULL host array", fn);
    if (K < 1 || K > LCP_MAX_ISOVALUES) return fail(LCP_ERR_ARG, "%s: need 1 <= K <= %d", fn, LCP_MAX_ISOVALUES);
    return LCP_OK;
}

// TMA-pipeline variant of lcp_fused (fused_tma.cu).  Returns
// LCP_ERR_UNSUPPORTED, having enqueued nothing, when the layout does not allow
// TMA (alignment / strides); the caller then uses the register-streaming kernel.
lcp_status fused_tma(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W, int64_t stride, int ddof,
                     double dx, double dy, const float* iso, int K, void* out, lcp_dtype out_dtype, uint32_t* mask,
                     cudaStream_t st);

// Clock-cycle budget of the bounded device waits that take it as a launch
// parameter (the workspace path's waits for statistics rows, the contour
// look-back): lcp_set_wait_budget's value, else the default (~2 s at 2 GHz).
constexpr long long kDefaultWaitBudget = 4000000000ll;
long long wait_budget_cycles();

// Device status words of the kernels with bounded waits (one per translation
// unit: device globals are not shared across units without relocatable code).
uint32_t read_tma_status(bool reset);  // TMA row-march pipeline (mbarrier waits)
uint32_t read_ws_status(bool reset);   // workspace path (LCP blocks waiting on statistics rows)
uint32_t read_contour_status(bool reset);  // contour compaction (decoupled look-back waits)
uint32_t read_sur_status(bool reset);      // learned-surrogate inference (tcgen05 mbarrier waits)

// Workspace of lcp_fused_ws: bands of `band_rows` cell rows (within a 96 MB L2
// budget and the workspace given, at least 8 rows); a counter header of
// ctr_bytes, then two record planes (u, v) of plane_bytes each.  A record is
// float4 (x0, delta, var, 0) per vertex and component: member 0, the FP32 mean
// of the members shifted by member 0, and the variance.
struct WsGeometry {
    int band_rows;
    size_t ctr_bytes, plane_bytes, total;
};
WsGeometry ws_geometry(int H, int W, size_t cap);  // bands that fit `cap` bytes of workspace
// Eqs. 2/3 and the LCP of cell rows [r0, r1) (plus the mask) from such record
// planes, whose row 0 is grid row row0 and which hold rows max(r0-1, 0) ..
// min(r1+1, H-1); launched in stream order after the kernel that wrote them.
lcp_status ws_lcp_rows(const float4* rec, int64_t ps, int row0, int H, int W, int r0, int r1, double dx, double dy,
                       const float* iso, int K, void* out, lcp_dtype out_dtype, uint32_t* mask, cudaStream_t st);

inline lcp_status check_spacing(const char* fn, double dx, double dy) {
    if (!(dx > 0.0) || !(dy > 0.0) || dx > 1e30 || dy > 1e30)
        return fail(LCP_ERR_ARG, "%s: dx and dy must be finite and > 0", fn);
    return LCP_OK;
}

}  // namespace lcp
