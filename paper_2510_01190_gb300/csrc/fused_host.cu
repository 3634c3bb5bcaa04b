// lcp_fused_host: lcp_fused_ws end to end for ensembles and results in host
// memory.  Members that the device can address (device memory, or pinned host
// memory) go straight to lcp_fused_ws, whose statistics kernel reads pinned
// members in place over the CPU-GPU link; the map and mask are computed into
// device staging at the head of the workspace and copied into the caller's
// buffers on the caller's stream.
#include <cstdint>

#include "lcp_common.cuh"

namespace {

// The device staging of the map and the mask words (each rounded up to 256
// bytes), ahead of lcp_fused_ws's records in the workspace.
struct HostLayout {
    size_t map_bytes, mask_bytes, staging;
};
HostLayout host_layout(int H, int W, int K, lcp_dtype out_dtype, bool with_mask) {
    HostLayout h;
    const size_t cells = (size_t)(H - 1) * (size_t)(W - 1);
    h.map_bytes = (size_t)K * cells * (out_dtype == LCP_F16 ? 2 : 4);
    h.mask_bytes = with_mask ? (size_t)K * (size_t)(H - 1) * (size_t)((W - 1 + 31) / 32) * 4 : 0;
    h.staging = ((h.map_bytes + 255) & ~(size_t)255) + ((h.mask_bytes + 255) & ~(size_t)255);
    return h;
}

// Device memory, or host memory the device can address (pinned); not pageable memory.
bool device_addressable(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged ||
           (a.type == cudaMemoryTypeHost && a.devicePointer != nullptr);
}

}  // namespace

extern "C" size_t lcp_fused_host_workspace_bytes(int M, int H, int W, int K, lcp_dtype out_dtype, int with_mask) {
    if (H < 2 || W < 2 || M < 1 || K < 1) return 0;
    return host_layout(H, W, K, out_dtype, with_mask != 0).staging + lcp_fused_workspace_bytes(M, H, W, LCP_F32);
}

extern "C" lcp_status lcp_fused_host(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                                     int64_t member_stride, int ddof, double dx, double dy, const float* iso, int K,
                                     void* lcp_out, lcp_dtype out_dtype, uint32_t* mask, void* workspace,
                                     size_t workspace_bytes, lcp_stream_t stream) {
    using lcp::fail;
    static const char* fn = "lcp_fused_host";
    lcp_status s = lcp::check_members(fn, u, v, in_dtype, M, H, W, member_stride, ddof);
    if (s != LCP_OK) return s;
    if ((s = lcp::check_iso(fn, iso, K)) != LCP_OK) return s;
    if (!lcp_out) return fail(LCP_ERR_ARG, "%s: NULL output", fn);
    if (out_dtype != LCP_F32 && out_dtype != LCP_F16) return fail(LCP_ERR_ARG, "%s: out dtype must be F32 or F16", fn);
    if (!workspace || ((uintptr_t)workspace & 255)) return fail(LCP_ERR_ARG, "%s: need a 256-byte aligned workspace", fn);
    if (!device_addressable(u) || !device_addressable(v))
        return fail(LCP_ERR_ARG, "%s: members must be device memory or pinned host memory", fn);
    const HostLayout hl = host_layout(H, W, K, out_dtype, mask != nullptr);
    if (workspace_bytes <= hl.staging)
        return fail(LCP_ERR_ARG, "%s: workspace too small (%zu bytes; the staging alone needs %zu)", fn,
                    workspace_bytes, hl.staging);
    char* const ws = reinterpret_cast<char*>(workspace);
    void* const map_d = ws;
    uint32_t* const mask_d = mask ? reinterpret_cast<uint32_t*>(ws + ((hl.map_bytes + 255) & ~(size_t)255)) : nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    // the fused path into the staging (its records in the rest of the workspace; smaller bands if it is short)
    s = lcp_fused_ws(u, v, in_dtype, M, H, W, member_stride, ddof, dx, dy, iso, K, map_d, out_dtype, mask_d,
                     ws + hl.staging, workspace_bytes - hl.staging, stream);
    if (s != LCP_OK) return s;
    // the results into the caller's buffers (asynchronous when those are pinned or device memory)
    if (cudaMemcpyAsync(lcp_out, map_d, hl.map_bytes, cudaMemcpyDefault, st) != cudaSuccess ||
        (mask && cudaMemcpyAsync(mask, mask_d, hl.mask_bytes, cudaMemcpyDefault, st) != cudaSuccess)) {
        const cudaError_t e = cudaGetLastError();
        return fail(LCP_ERR_CUDA, "%s: copying the results back failed: %s", fn, cudaGetErrorString(e));
    }
    return LCP_OK;
}
