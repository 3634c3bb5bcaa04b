// Partition of the closed-form path over several GPUs (host arithmetic only).
//
// The method is per-pixel data parallel (Sec. 3.3): every cell's LCP depends
// only on the statistics of its four vertices and their stencil neighbours
// (Eqs. 2/3).  A grid therefore splits into strips of cell rows with no
// exchange at all: the strip of cells [c0, c1) needs vertex rows c0 .. c1 and,
// for their vertical central differences, the rows c0 - 1 and c1 + 1, so each
// rank re-reads that halo of member rows (one row above, two below in the
// half-open range of vertex rows) and evaluates its strip as a grid of its own.
// The sub-grid's outermost vertex rows then take one-sided differences, which
// is right only where they are the grid's own first or last row; the cell rows
// next to a halo row are computed and dropped.  Independent fields (a batch)
// split by whole fields, balanced by bytes with the longest-processing-time
// rule (largest first, each to the least-loaded rank).
#include <algorithm>
#include <numeric>
#include <vector>

#include "lcp_common.cuh"

using namespace lcp;

extern "C" lcp_status lcp_strip_plan(int H, int nranks, int rank, int* vrow_begin, int* vrow_end, int* cell_begin,
                                     int* cell_end) {
    if (H < 2) return fail(LCP_ERR_ARG, "lcp_strip_plan: need H >= 2");
    if (nranks < 1 || rank < 0 || rank >= nranks) return fail(LCP_ERR_ARG, "lcp_strip_plan: need 0 <= rank < nranks");
    if (!vrow_begin || !vrow_end || !cell_begin || !cell_end) return fail(LCP_ERR_ARG, "lcp_strip_plan: NULL output");
    const int64_t Hc = H - 1;
    const int c0 = (int)(Hc * rank / nranks), c1 = (int)(Hc * (rank + 1) / nranks);
    *cell_begin = c0;
    *cell_end = c1;
    if (c0 == c1) {  // more ranks than cell rows: an empty strip
        *vrow_begin = *vrow_end = c0;
        return LCP_OK;
    }
    *vrow_begin = std::max(c0 - 1, 0);
    *vrow_end = std::min(c1 + 2, H);
    return LCP_OK;
}

extern "C" lcp_status lcp_lpt_assign(const int64_t* cost, int n, int nranks, int* owner, int64_t* load) {
    if (n < 0 || nranks < 1) return fail(LCP_ERR_ARG, "lcp_lpt_assign: need n >= 0 and nranks >= 1");
    if (n > 0 && (!cost || !owner)) return fail(LCP_ERR_ARG, "lcp_lpt_assign: NULL cost or owner");
    for (int i = 0; i < n; ++i)
        if (cost[i] < 0) return fail(LCP_ERR_ARG, "lcp_lpt_assign: negative cost %lld", (long long)cost[i]);
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    // largest first; equal costs in index order, so the plan is the same on every rank
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<int64_t> l(nranks, 0);
    for (int i : order) {
        const int r = (int)(std::min_element(l.begin(), l.end()) - l.begin());  // least loaded, lowest index
        owner[i] = r;
        l[r] += cost[i];
    }
    if (load)
        for (int r = 0; r < nranks; ++r) load[r] = l[r];
    return LCP_OK;
}
