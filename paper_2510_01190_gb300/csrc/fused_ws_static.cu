// lcp_fused_static_ws: the workspace path (lcp_fused_ws) with its scratch in a
// fixed, file-scope device array instead of memory the caller allocates.
//
// Some callers cannot allocate device memory at the call site: plain C hosts
// that hold no device allocator of their own, and steady-state loops that must
// not pay cudaMalloc's implicit device synchronisation or risk its failure
// under memory pressure half-way through a run.  This entry point needs no
// allocation at all: the scratch is reserved when the module is loaded, and
// every call only looks up the array's address (host-side bookkeeping once the
// module is loaded) and launches work on the caller's stream.
#include "lcp_common.cuh"

namespace {

// Maximum scratch, 64 MiB.  Record rows take 32 bytes per vertex, so the
// bands shrink to fit it: a 721 x 1440 grid still runs in one band (33.2 MB),
// an 8192-wide grid in 248-row bands (65.8 MB) instead of the 376-row bands
// (99.3 MB) that lcp_fused_workspace_bytes gives it; grids wider than about
// 190,000 vertices do not fit even the smallest band (8 cell rows + halo).
constexpr size_t kStaticWsBytes = (size_t)64 << 20;

static __device__ __align__(256) unsigned char g_static_ws[kStaticWsBytes];

// Device address of g_static_ws on the current device.  Looked up on every
// call rather than cached, so that a context re-created after
// cudaDeviceReset (which may load the module at another address) is never
// handed a stale pointer.
void* static_ws_ptr(lcp_status* s) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        *s = lcp::fail(LCP_ERR_CUDA, "lcp_fused_static_ws: scratch address lookup failed: %s", cudaGetErrorString(e));
        return nullptr;
    }
    *s = LCP_OK;
    return p;
}

}  // namespace

extern "C" lcp_status lcp_fused_static_ws(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                                          int64_t member_stride, int ddof, double dx, double dy, const float* iso,
                                          int K, void* lcp_out, lcp_dtype out_dtype, uint32_t* mask,
                                          lcp_stream_t stream) {
    if (H < 2 || W < 2 || M < 1)
        return lcp::fail(LCP_ERR_ARG, "lcp_fused_static_ws: need M >= 1, H >= 2, W >= 2 (got %d, %d, %d)", M, H, W);
    // the row bands shrink to fit the static scratch; lcp_fused_ws rejects grids whose
    // smallest band does not fit
    lcp_status s = LCP_OK;
    void* ws = static_ws_ptr(&s);
    if (!ws) return s;
    // The only state that must start at zero, the per-band completion counters
    // at the head of the scratch, is cleared on `stream` by the workspace path
    // before each band; the record planes are written before they are read.
    return lcp_fused_ws(u, v, in_dtype, M, H, W, member_stride, ddof, dx, dy, iso, K, lcp_out, out_dtype, mask, ws,
                        kStaticWsBytes, stream);
}
