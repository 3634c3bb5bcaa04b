// Host plumbing of the C ABI: status strings, thread-local error messages,
// device queries, and the raw Philox fill used to test the Monte Carlo generator.
#include <stdarg.h>
#include <stdio.h>

#include <atomic>
#include <mutex>

#include "lcp_common.cuh"

namespace lcp {

static std::atomic<long long> g_wait_budget{0};  // 0: the default

long long wait_budget_cycles() {
    const long long b = g_wait_budget.load(std::memory_order_relaxed);
    return b > 0 ? b : kDefaultWaitBudget;
}

static thread_local char g_last_error[512] = "";

lcp_status fail(lcp_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

lcp_status check_launch(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LCP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return LCP_OK;
}

int num_sms() {
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    std::lock_guard<std::mutex> lk(mu);
    if (cached[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cached[dev] = n;
    }
    return cached[dev];
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// out[4n + r] = word r of Philox-4x32-10(counter (n, c1, off lo, off hi), key (seed lo, seed hi))
__global__ void philox_fill_kernel(uint2 key, uint32_t c1, uint2 off, uint64_t count, uint4* out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t n = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; n < count; n += stride)
        out[n] = philox4x32_10(make_uint4((uint32_t)n, c1, off.x, off.y), key);
}

}  // namespace lcp

using namespace lcp;

extern "C" const char* lcp_status_string(lcp_status s) {
    switch (s) {
        case LCP_OK: return "LCP_OK";
        case LCP_ERR_ARG: return "LCP_ERR_ARG: invalid argument";
        case LCP_ERR_CUDA: return "LCP_ERR_CUDA: CUDA runtime error";
        case LCP_ERR_UNSUPPORTED: return "LCP_ERR_UNSUPPORTED: not implemented for these arguments";
        case LCP_ERR_TIMEOUT: return "LCP_ERR_TIMEOUT: a bounded device wait gave up";
        case LCP_ERR_NUMERIC: return "LCP_ERR_NUMERIC: numerically unusable input";
    }
    return "unknown lcp_status";
}

extern "C" const char* lcp_last_error(void) { return g_last_error; }

extern "C" int lcp_version(void) { return 10000; }

extern "C" long long lcp_set_wait_budget(long long cycles) {
    const long long prev = wait_budget_cycles();
    g_wait_budget.store(cycles > 0 ? cycles : 0, std::memory_order_relaxed);
    return prev;
}

extern "C" lcp_status lcp_philox_fill(uint64_t seed, uint32_t c1, uint64_t offset, int64_t count, uint32_t* out,
                                      lcp_stream_t stream) {
    if (count < 0 || count > (int64_t(1) << 32)) return fail(LCP_ERR_ARG, "lcp_philox_fill: count out of range");
    if (count == 0) return LCP_OK;
    if (!out || !aligned16(out)) return fail(LCP_ERR_ARG, "lcp_philox_fill: out must be a 16-byte aligned device pointer");
    const int threads = 256;
    const int64_t want = (count + threads - 1) / threads;
    const int blocks = (int)(want < 8L * num_sms() ? want : 8L * num_sms());
    philox_fill_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(
        make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), c1,
        make_uint2((uint32_t)offset, (uint32_t)(offset >> 32)), (uint64_t)count, reinterpret_cast<uint4*>(out));
    return check_launch("lcp_philox_fill");
}

extern "C" lcp_status lcp_device_status(uint32_t* flags, int reset) {
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(LCP_ERR_CUDA, "lcp_device_status: device error");
    const uint32_t f = read_tma_status(reset != 0) | read_ws_status(reset != 0) | (read_sur_status(reset != 0) << 1) |
                       (read_contour_status(reset != 0) << 2);
    if (flags) *flags = f;
    return f ? fail(LCP_ERR_TIMEOUT, "a bounded device wait gave up (flags 0x%x)", f) : LCP_OK;
}
