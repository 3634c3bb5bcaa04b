// lcp_divergence: the divergence Gaussian N(mu_d, var_d) at every vertex
// (Sec. 3.1, Eqs. 2 and 3) from per-vertex component statistics.  Eq. 1's
// central differences become first-order one-sided differences on the first
// and last column (row), as Sec. 3.1 states for the boundary.
#include "lcp_common.cuh"

namespace lcp {
namespace {

__global__ void __launch_bounds__(256) divergence_kernel(const float* __restrict__ mu_u, const float* __restrict__ var_u,
                                                         const float* __restrict__ mu_v, const float* __restrict__ var_v,
                                                         int H, int W, Spacing sp, float* __restrict__ mu_d,
                                                         float* __restrict__ var_d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= W) return;
    const int ilo = i > 0 ? i - 1 : 0, ihi = i < W - 1 ? i + 1 : W - 1;
    const int jlo = j > 0 ? j - 1 : 0, jhi = j < H - 1 ? j + 1 : H - 1;
    const float sx = (ihi - ilo == 2) ? sp.sx2 : sp.sx1, sxq = (ihi - ilo == 2) ? sp.sx2q : sp.sx1q;
    const float sy = (jhi - jlo == 2) ? sp.sy2 : sp.sy1, syq = (jhi - jlo == 2) ? sp.sy2q : sp.sy1q;
    const int64_t row = (int64_t)j * W;
    const float du = mu_u[row + ihi] - mu_u[row + ilo];
    const float dv = mu_v[(int64_t)jhi * W + i] - mu_v[(int64_t)jlo * W + i];
    const float vu = var_u[row + ihi] + var_u[row + ilo];
    const float vv = var_v[(int64_t)jhi * W + i] + var_v[(int64_t)jlo * W + i];
    mu_d[row + i] = fmaf(du, sx, dv * sy);
    var_d[row + i] = fmaf(vu, sxq, vv * syq);
}

}  // namespace
}  // namespace lcp

using namespace lcp;

extern "C" lcp_status lcp_divergence(const float* mu_u, const float* var_u, const float* mu_v, const float* var_v,
                                     int H, int W, double dx, double dy, float* mu_d, float* var_d,
                                     lcp_stream_t stream) {
    if (!mu_u || !var_u || !mu_v || !var_v || !mu_d || !var_d)
        return fail(LCP_ERR_ARG, "lcp_divergence: NULL pointer");
    if (H < 2 || W < 2) return fail(LCP_ERR_ARG, "lcp_divergence: need H >= 2 and W >= 2");
    lcp_status s = check_spacing("lcp_divergence", dx, dy);
    if (s != LCP_OK) return s;
    if (H > 65535 * 64) return fail(LCP_ERR_UNSUPPORTED, "lcp_divergence: H too large");
    dim3 grid((W + 255) / 256, H);
    divergence_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(mu_u, var_u, mu_v, var_v, H, W, make_spacing(dx, dy),
                                                               mu_d, var_d);
    return check_launch("lcp_divergence");
}
