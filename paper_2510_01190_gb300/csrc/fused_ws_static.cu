// lcp_fused_static_ws: the workspace path (lcp_fused_ws) with its scratch in a
// fixed, file-scope device array instead of memory the caller allocates.
//
// Some callers cannot allocate device memory at the call site: plain C hosts
// that hold no device allocator of their own, and steady-state loops that must
// not pay cudaMalloc's implicit device synchronisation or risk its failure
// under memory pressure half-way through a run.  This entry point needs no
// allocation at all: the scratch is reserved when the module is loaded, its
// address is looked up once per device, and every call after that only
// launches work on the caller's stream.
#include <mutex>

#include "lcp_common.cuh"

namespace {

// Maximum scratch, 64 MiB: covers every grid whose workspace stays in the
// L2-sized band layout with W up to about 190,000 vertices (a 721 x 1440 grid
// needs 33.2 MB, an 8192 x 8192 grid 49.0 MB).
constexpr size_t kStaticWsBytes = (size_t)64 << 20;

static __device__ __align__(256) unsigned char g_static_ws[kStaticWsBytes];

constexpr int kMaxDevices = 64;

// Per-device address of g_static_ws, looked up on the first call made with
// that device current.
void* static_ws_ptr(int dev, lcp_status* s) {
    static std::mutex mu;
    static void* ptr[kMaxDevices] = {nullptr};
    std::lock_guard<std::mutex> lk(mu);
    if (!ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            *s = lcp::fail(LCP_ERR_CUDA, "lcp_fused_static_ws: scratch address lookup failed: %s",
                           cudaGetErrorString(e));
            return nullptr;
        }
        ptr[dev] = p;
    }
    *s = LCP_OK;
    return ptr[dev];
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
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return lcp::fail(LCP_ERR_CUDA, "lcp_fused_static_ws: no usable current device");
    }
    lcp_status s = LCP_OK;
    void* ws = static_ws_ptr(dev, &s);
    if (!ws) return s;
    // The only state that must start at zero, the per-band completion counters
    // at the head of the scratch, is cleared on `stream` by the workspace path
    // before each band; the record planes are written before they are read.
    return lcp_fused_ws(u, v, in_dtype, M, H, W, member_stride, ddof, dx, dy, iso, K, lcp_out, out_dtype, mask, ws,
                        kStaticWsBytes, stream);
}
