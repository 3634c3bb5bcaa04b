/*
 * lcp.h - C ABI of the GB300 (sm_103a) library for level-crossing-probability
 * (LCP) maps of the local divergence of uncertain 2D vector fields.
 *
 * Method: Ouermi, Li, Moreland, Pugmire, Johnson, Athawale, "Efficient
 * Probabilistic Visualization of Local Divergence of 2D Vector Fields with
 * Independent Gaussian Uncertainty", arXiv 2510.01190.  Sec. 3.1 defines the
 * per-vertex Gaussian model, the divergence stencil (Eq. 1) and the divergence
 * Gaussian (Eqs. 2, 3); its last paragraph feeds that Gaussian to the
 * level-crossing probability of Poethkow et al.  Sec. 3.2 and Sec. 4 define the
 * classical Monte Carlo estimator used as the baseline.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid      H rows x W columns of vertices, H >= 2 and W >= 2.  Vertex (i, j)
 *           has i = x = column, j = y = row; 2D arrays are row-major [H][W].
 * Members   one plane per member and component: element (m, j, i) of u lives at
 *           u[m * member_stride + j * W + i]; member_stride >= H * W.  u is the
 *           x component, v the y component.  Element type LCP_F32 or LCP_BF16.
 * Cells     cell (i, j) has vertices (i,j), (i+1,j), (i,j+1), (i+1,j+1); LCP maps
 *           are [K][H-1][W-1], isovalue-major.
 * Masks     mean-field crossing bits (optional, may be NULL): for isovalue k and
 *           cell row j, ceil((W-1)/32) uint32 words; bit (i % 32) of word i / 32
 *           is set iff cell (i, j) crosses.  Layout [K][H-1][ceil((W-1)/32)].
 * Boundary  Eq. 1 uses central differences; on the first/last column (row) the
 *           library uses the first-order forward/backward difference with step
 *           dx (dy), as Sec. 3.1 states for the boundary.
 * Memory    every array argument is a DEVICE pointer owned by the caller unless
 *           the parameter says "host"; the library allocates no device memory.
 *           fp32 arrays must be 4-byte aligned, bf16/fp16 2-byte aligned; wider
 *           vector loads are used automatically when alignment allows.
 * Streams   every call only validates its arguments and enqueues work on
 *           `stream`; it returns before the GPU finishes.  Errors found on the
 *           host return a negative lcp_status and enqueue nothing; the message
 *           is available from lcp_last_error() on the calling thread.
 * NaN/Inf   NaN or Inf member values propagate to NaN in the statistics of that
 *           vertex and in every divergence/LCP value that touches it; they are
 *           not an error.
 */
#ifndef LCP_GB300_H
#define LCP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* lcp_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    LCP_OK = 0,
    LCP_ERR_ARG = -1,         /* invalid size, pointer, alignment or option */
    LCP_ERR_CUDA = -2,        /* a CUDA runtime call failed (launch, attribute, ...) */
    LCP_ERR_UNSUPPORTED = -3, /* valid request the library does not implement */
    LCP_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    LCP_ERR_NUMERIC = -5      /* reserved: numerically unusable input */
} lcp_status;

typedef enum { LCP_F32 = 0, LCP_BF16 = 1, LCP_F16 = 2, LCP_F64 = 3 } lcp_dtype;

typedef enum { LCP_MC_GAUSS = 0, LCP_MC_EMPIRICAL = 1 } lcp_mc_mode;

#define LCP_MAX_ISOVALUES 256 /* K limit of every entry point */

/* Human-readable name of a status code (static storage). */
const char* lcp_status_string(lcp_status s);

/* Message of the last error returned on the calling thread ("" if none). */
const char* lcp_last_error(void);

/* Library version as 10000 * major + 100 * minor + patch. */
int lcp_version(void);

/*
 * lcp_stats - per-vertex Gaussian model of each component (Sec. 3.1, closing
 * paragraph: mu-hat and sigma-hat^2 are estimated from the ensemble).
 *
 *   mean = (1/M) sum_m x_m,  var = sum_m (x_m - mean)^2 / (M - ddof)
 *
 * computed in FP32 as shifted sums about member 0 (one pass over the members).
 * u, v        members, element type `in_dtype` (LCP_F32 or LCP_BF16)
 * M, H, W     members (M >= 1, M - ddof >= 1), rows, columns
 * member_stride  elements between consecutive members (>= H*W)
 * ddof        0 (population) or 1 (sample variance)
 * mu_u, var_u, mu_v, var_v   outputs, fp32 [H][W]
 * Errors: LCP_ERR_ARG for a NULL pointer, H < 2, W < 2, M < 1, M - ddof < 1,
 * ddof not in {0, 1}, member_stride < H*W, or an unsupported dtype.
 */
lcp_status lcp_stats(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                     int64_t member_stride, int ddof, float* mu_u, float* var_u, float* mu_v,
                     float* var_v, lcp_stream_t stream);

/*
 * lcp_divergence - divergence Gaussian N(mu_d, var_d) at every vertex (Eqs. 2
 * and 3, Sec. 3.1), with the one-sided boundary rule above:
 *   mu_d  = (mu_u[i+] - mu_u[i-]) / ((i+ - i-) dx) + (mu_v[j+] - mu_v[j-]) / ((j+ - j-) dy)
 *   var_d = (var_u[i+] + var_u[i-]) / ((i+ - i-) dx)^2 + (var_v[j+] + var_v[j-]) / ((j+ - j-) dy)^2
 * with i- = max(i-1, 0), i+ = min(i+1, W-1) (j alike).
 * Inputs fp32 [H][W] (from lcp_stats); outputs mu_d, var_d fp32 [H][W].
 * dx, dy > 0 (finite).  Errors: LCP_ERR_ARG for NULL, H < 2, W < 2, dx or dy <= 0.
 */
lcp_status lcp_divergence(const float* mu_u, const float* var_u, const float* mu_v,
                          const float* var_v, int H, int W, double dx, double dy, float* mu_d,
                          float* var_d, lcp_stream_t stream);

/*
 * lcp_map - level-crossing probability of every cell (Sec. 3.1, last
 * paragraph, after Poethkow et al.): with p = P(D < c) = erfc((mu_d - c) /
 * (sigma_d sqrt 2)) / 2 and q = P(D >= c) at the 4 cell vertices, treated as
 * independent,
 *   LCP = 1 - p00 p10 p01 p11 - q00 q10 q01 q11.
 * A vertex with var_d == 0 has p = [mu_d < c], q = 1 - p.
 * mu_d, var_d   fp32 [H][W]
 * iso           HOST array of K isovalues (fp32), 1 <= K <= LCP_MAX_ISOVALUES
 * lcp_out       [K][H-1][W-1] of `out_dtype` (LCP_F32 or LCP_F16)
 * mask          optional mean-field crossing bits (layout above) or NULL
 */
lcp_status lcp_map(const float* mu_d, const float* var_d, int H, int W, const float* iso, int K,
                   void* lcp_out, lcp_dtype out_dtype, uint32_t* mask, lcp_stream_t stream);

/*
 * lcp_fused - lcp_stats -> lcp_divergence -> lcp_map in one kernel pass over
 * the members: each member byte is read from HBM once; statistics, divergence
 * and per-vertex probabilities stay on chip.  Same arguments and results as
 * the three calls in sequence (the mean is kept as member-0 shift plus FP32
 * offset internally, so it is at least as accurate as the unfused path).
 * K > 32 is processed in passes of 32 isovalues.  When the planes are 16-byte
 * aligned and W and member_stride are multiples of 16 bytes, members stream
 * through TMA copies into shared memory; otherwise through vector loads.
 * This is the entry point for callers that cannot provide a workspace;
 * lcp_fused_ws is the fast path (about twice as fast on large grids, 0.10 ms
 * against 0.18 ms on 721 x 1440 x 51) and the more accurate one: lcp_fused
 * forms every stencil in fp32, which keeps the 1e-5 bound while the member-0
 * values across a stencil differ by at most ~16 sigma or lie within a factor
 * of 2 of each other (a common offset of any size), but not for means of
 * large magnitude that change sign across a stencil.
 */
lcp_status lcp_fused(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                     int64_t member_stride, int ddof, double dx, double dy, const float* iso, int K,
                     void* lcp_out, lcp_dtype out_dtype, uint32_t* mask, lcp_stream_t stream);

/*
 * lcp_fused_workspace_bytes / lcp_fused_ws - lcp_fused with a caller-provided
 * device workspace (256-byte aligned, at least lcp_fused_workspace_bytes(M, H,
 * W, in_dtype) bytes).  Same results as lcp_fused.  Each member byte is still
 * read from HBM once: a flat, coalesced statistics stream leaves two 16-byte
 * records per vertex (member-0 shift, shifted mean and variance of u and of v)
 * in the workspace with an L2 keep-resident policy, and a second kernel,
 * launched as its programmatic dependent, evaluates Eqs. 2/3 and the LCP of
 * every cell from there, each of its blocks starting as soon as the records it
 * reads are complete (per-band counters in the workspace, reset by the call
 * with a memset node on `stream`).  Grids whose records exceed about 96 MB run
 * in bands of rows with one halo row each side, so the workspace stays in L2
 * and its size is bounded.  lcp_fused_workspace_bytes is the size for the
 * largest bands; a smaller workspace gives smaller bands (at least 8 cell rows
 * plus the halo, else LCP_ERR_ARG).  Calls sharing one workspace must not
 * overlap in time.  workspace == NULL runs lcp_fused.  With a workspace, u and
 * v may also be pinned host memory that the device can address (cudaHostAlloc
 * under unified addressing): the statistics kernel then reads each member byte
 * once over the CPU-GPU link, with no staging copy; the host planes must stay
 * unchanged until the work on `stream` is complete.
 * Precision: where the member-0 differences across a vertex's stencil exceed 16
 * sigma (means of large magnitude changing sign, say), that vertex's mean is
 * formed again in FP64 and carried as an fp32 pair into the z-scores, so the
 * map stays within 1e-5 of the FP64 definition (Sec. 3.1) whatever the means'
 * magnitude; elsewhere the fp32 stencil already is.
 */
size_t lcp_fused_workspace_bytes(int M, int H, int W, lcp_dtype in_dtype);

/*
 * lcp_fused_band_rows - the cell rows per band that lcp_fused_ws (and
 * lcp_speed_gradient_ws, whose records have the same layout) runs an H x W
 * grid in with `workspace_bytes` of workspace: H - 1 when the grid runs as
 * one band, else a multiple of 8; ceil((H - 1) / rows) bands.  Host-only: no
 * device is touched.  Returns 0 for H < 2 or W < 2, or a workspace smaller
 * than the smallest band needs.
 */
int lcp_fused_band_rows(int H, int W, size_t workspace_bytes);

lcp_status lcp_fused_ws(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                        int64_t member_stride, int ddof, double dx, double dy, const float* iso, int K,
                        void* lcp_out, lcp_dtype out_dtype, uint32_t* mask, void* workspace,
                        size_t workspace_bytes, lcp_stream_t stream);

/*
 * lcp_fused_static_ws - lcp_fused_ws with its scratch in a 64 MiB file-scope
 * device array of the library instead of a caller workspace, so that the call
 * allocates no memory: for callers that hold no device allocator, or that must
 * not pay an allocation's device synchronisation (or its failure under memory
 * pressure) inside a steady-state loop.  The paper has no counterpart: it is a
 * host-interface convenience that computes the same results as lcp_fused_ws,
 * with the same arguments except the workspace.
 * Set-up: every call looks up the array's device address on the current
 * device (after cudaDeviceReset the module may load at another address); the
 * first call on a device loads the library's module there, so make that first
 * call before any stream capture.
 * The per-band counters that must start at zero are cleared on `stream` by
 * every call.  The one array is shared by all calls on a device: calls that
 * overlap in time (other streams, other host threads) race and give undefined
 * results.  The row bands shrink to fit the 64 MiB (wide grids run in more,
 * smaller bands than with lcp_fused_workspace_bytes of workspace: an
 * 8192-wide grid in 248-row bands instead of 376).  Errors:
 * LCP_ERR_ARG when even the smallest band (8 cell rows plus the halo) needs more
 * than 64 MiB (grids wider than about 190,000 vertices) or on any argument
 * lcp_fused_ws rejects; LCP_ERR_CUDA when the address lookup fails.
 */
lcp_status lcp_fused_static_ws(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                               int64_t member_stride, int ddof, double dx, double dy, const float* iso, int K,
                               void* lcp_out, lcp_dtype out_dtype, uint32_t* mask, lcp_stream_t stream);

/*
 * lcp_fused_host - the closed-form LCP map of lcp_fused_ws (statistics of
 * Sec. 3.1, the divergence Gaussian of Eqs. 2/3, the LCP of every cell of the
 * last paragraph of Sec. 3.1, and the mean-field mask) for callers whose
 * ensembles and results live in host memory, end to end in one call.
 * u, v: device memory, or pinned host memory the device can address
 * (cudaHostAlloc, cudaHostRegister), read in place, each member byte once over
 * the CPU-GPU link; pageable memory is rejected with LCP_ERR_ARG (copy it into
 * pinned or device memory first).  Layout, dtypes, stride and ddof as
 * lcp_fused_ws.  lcp_out ([K][H-1][W-1], out_dtype F32 or F16) and mask (as
 * lcp_fused_ws, or NULL) may be host or device memory: the map and mask are
 * computed into device staging at the head of `workspace` and copied into
 * them on `stream` (asynchronously when they are pinned or device memory).
 * workspace: device, 256-byte aligned, lcp_fused_host_workspace_bytes(M, H,
 * W, K, out_dtype, mask != NULL) bytes for the largest bands (a smaller one
 * gives smaller bands, as lcp_fused_ws; it must exceed the staging).  The
 * members must stay unchanged, and the outputs must not be read, until the
 * work on `stream` is complete.  Calls sharing one workspace must not overlap.
 */
size_t lcp_fused_host_workspace_bytes(int M, int H, int W, int K, lcp_dtype out_dtype, int with_mask);
lcp_status lcp_fused_host(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                          int64_t member_stride, int ddof, double dx, double dy, const float* iso, int K,
                          void* lcp_out, lcp_dtype out_dtype, uint32_t* mask, void* workspace,
                          size_t workspace_bytes, lcp_stream_t stream);

/*
 * Batched closed form: many fields of uneven size (each its own H, W, M,
 * spacing and isovalue list) evaluated by ONE persistent kernel launch.  The
 * computation per field is exactly lcp_fused's (Eqs. 1-3 per vertex, the LCP of
 * Sec. 3.1's last paragraph per cell and isovalue, the mean-field mask); the paper evaluates one
 * field at a time, and batching is this library's addition.
 *
 * lcp_field_desc - one field of a batch (all pointers are device pointers owned
 * by the caller; they must stay valid for every lcp_batch call of the plan):
 *   u, v            [M][H][W] members of the two components, row-major planes
 *   member_stride   elements between consecutive members (>= H*W when M > 1)
 *   M, H, W, ddof   members, vertex rows, vertex columns, variance ddof
 *   dx, dy          grid spacing (finite, > 0)
 *   iso_begin, K    the field's isovalues are iso[iso_begin .. iso_begin+K) of
 *                   the batch's isovalue table
 *   lcp_out         [K][H-1][W-1] of the plan's out_dtype
 *   mask            [K][H-1][ceil((W-1)/32)] uint32 mean-field mask, or NULL
 */
typedef struct {
    const void* u;
    const void* v;
    int64_t member_stride;
    int M, H, W, ddof;
    double dx, dy;
    int iso_begin, K;
    void* lcp_out;
    uint32_t* mask;
} lcp_field_desc;

/*
 * lcp_tune - launch shape of the batch kernel: a tile of tile_rows cell rows by
 * tile_cols cell columns, one of (64, 64), (32, 128), (32, 64), (16, 128);
 * ctas_per_sm = 0 takes as many CTAs per SM as fit.
 */
typedef struct {
    int tile_rows, tile_cols;
    int ctas_per_sm;
} lcp_tune;

/*
 * lcp_batch_plan - filled by lcp_batch_prepare; read by lcp_batch and
 * lcp_batch_autotune.  Plain data: copy it freely, do not edit it.
 */
typedef struct {
    void* workspace;
    size_t workspace_bytes;
    int n_fields, n_iso;
    lcp_dtype in_dtype, out_dtype;
    int64_t cells;            /* sum over fields of (H-1)(W-1) */
    int64_t cell_isovalues;   /* sum over fields of K (H-1)(W-1) */
    int64_t member_bytes;     /* bytes of u and v read once */
    int64_t out_bytes;        /* bytes of LCP maps and masks written once */
} lcp_batch_plan;

/* Device workspace a batch of n_fields fields and n_iso isovalues needs. */
size_t lcp_batch_workspace_bytes(int n_fields, int n_iso);

/*
 * lcp_batch_prepare - validate every descriptor on the host (the checks of
 * lcp_fused, per field, with 1 <= K <= LCP_MAX_ISOVALUES and iso_begin + K <=
 * n_iso) and write the batch's work
 * table (field records ordered by cost, tile prefix sums for every tile shape,
 * the isovalue table) into `workspace` (device, 256-byte aligned, at least
 * lcp_batch_workspace_bytes).  fields and iso are HOST arrays and may be freed
 * on return: the call copies them on `stream` and synchronises with it, so it
 * must not be called during stream capture.  in_dtype LCP_F32 or LCP_BF16;
 * out_dtype LCP_F32 or LCP_F16.  Errors: LCP_ERR_ARG naming the first bad
 * field; LCP_ERR_CUDA.
 */
lcp_status lcp_batch_prepare(const lcp_field_desc* fields, int n_fields, const float* iso, int n_iso,
                             lcp_dtype in_dtype, lcp_dtype out_dtype, void* workspace, size_t workspace_bytes,
                             lcp_stream_t stream, lcp_batch_plan* plan);

/*
 * lcp_batch - evaluate every field of a prepared plan: a memset node (the tile
 * counter) and one persistent kernel launch on `stream`, nothing else, so the
 * call can be captured into a CUDA graph once it has run outside capture on the
 * device (the first call sets the kernel's shared-memory limit).  tune == NULL
 * takes (64, 64).  Each CTA takes tiles from the batch's work list in turn and
 * computes a tile's statistics and its one-vertex halo itself, so no CTA waits
 * on another.  Calls sharing one workspace must not overlap in time.  Errors:
 * LCP_ERR_ARG for an unknown tile shape or an unprepared plan; LCP_ERR_CUDA.
 */
lcp_status lcp_batch(const lcp_batch_plan* plan, const lcp_tune* tune, lcp_stream_t stream);

/*
 * lcp_batch_autotune - time every tile shape of lcp_tune (reps runs each, CUDA
 * events on `stream`, after one warm-up run) on the plan itself and return the
 * fastest in *best; ms (optional, HOST, 4 floats) receives each shape's mean
 * time in the order listed under lcp_tune.  Writes the plan's outputs (with the
 * correct results).  Synchronises; not for use during stream capture.
 */
lcp_status lcp_batch_autotune(const lcp_batch_plan* plan, int reps, lcp_tune* best, float* ms,
                              lcp_stream_t stream);

/*
 * Autotuner cache (this library's addition; the paper has no counterpart): the
 * tile lcp_batch_autotune picked, kept in a JSON file keyed by the batch's shape
 * and the device, so that a later call or process takes it without timing every
 * shape again.  The file holds {"lcp_tune_cache": 1, "entries": [{"key": ...,
 * "tile": [rows, cols], "ms": [4 times]}, ...]}; it is rewritten whole on each
 * store (a temporary file renamed over it).  A missing, empty or malformed file
 * reads as empty.  All strings and pointers are HOST.
 *
 * lcp_tune_cache_lookup - the entry of `key` in the file at `path`: returns 1 and
 *   fills *best (ctas_per_sm = 0) and ms (optional, 4 floats) on a hit, 0 on a
 *   miss or an entry whose tile is not one of lcp_tune's shapes, LCP_ERR_ARG for
 *   a NULL or empty path, a NULL key or best.  No device work.
 * lcp_tune_cache_store - add or replace the entry of `key` (ms optional, else
 *   zeros).  LCP_ERR_ARG for NULL arguments, a tile that is not one of the
 *   shapes, or a file that cannot be written.  No device work.
 * lcp_batch_tune_key - the key of a plan on the current device ("<device
 *   name>|sm<SMs>|in<dtype>|out<dtype>|fields<n>|iso<n>|cells<n>|ciso<n>|
 *   mbytes<n>") into buf (len bytes); returns its length, LCP_ERR_ARG when buf is
 *   too small, LCP_ERR_CUDA without a device.
 * lcp_batch_autotune_cached - the tile from the cache at cache_path (NULL: the
 *   LCP_TUNE_CACHE environment variable; neither: no cache) when it holds the
 *   plan's key (*from_cache = 1; no device work, so the plan's outputs are not
 *   written), else lcp_batch_autotune (which writes them) and a store of the
 *   result; ms (optional, 4 floats) as lcp_batch_autotune's.  A store that fails
 *   returns LCP_ERR_ARG with *best already valid.
 */
int lcp_tune_cache_lookup(const char* path, const char* key, lcp_tune* best, float* ms);
lcp_status lcp_tune_cache_store(const char* path, const char* key, const lcp_tune* best, const float* ms);
int lcp_batch_tune_key(const lcp_batch_plan* plan, char* buf, size_t len);
lcp_status lcp_batch_autotune_cached(const lcp_batch_plan* plan, int reps, const char* cache_path,
                                     lcp_tune* best, float* ms, int* from_cache, lcp_stream_t stream);

/*
 * Learned surrogate for ensembles that are not Gaussian.  The paper mentions
 * neural surrogates only among related work (Sec. 2); the network, its
 * features and its training are this library's addition.  Under the empirical
 * model (every vertex component an independent uniform draw from its own
 * members), the divergence D of a vertex is the Eq. 1 stencil sum of four
 * independent values, so its cumulants are sums of the terms' cumulants scaled
 * by the stencil weights (1/(2dx), or 1/dx at the grid's edges).  A
 * 17 -> 64 -> 64 -> 1 network (tanh, tanh, sigmoid; BF16 operands, FP32
 * accumulation on the tensor cores) maps per-cell features of those cumulants
 * to the LCP.  Features of cell (i, j) and isovalue c, vertices (i, j),
 * (i+1, j), (i, j+1), (i+1, j+1), sigma = sqrt(k2):
 *   4v+0 (c - k1)/sigma clipped to [-8, 8] (sigma = 0: -8, 0 or 8 by sign)
 *   4v+1 sigma / mean of the cell's four sigmas (1 if all are 0)
 *   4v+2 k3/sigma^3 clipped to [-5, 5];  4v+3 k4/sigma^4 clipped to [-2, 10]
 *        (both 0 when sigma = 0)
 *   16   the independent-Gaussian closed-form LCP with means k1, variances k2
 * A feature row is 32 bf16 values (features 17..31 are zero).  Each row also
 * has a prior, the logit of feature 16 clamped to [1e-6, 1 - 1e-6], in fp32:
 * the network's output is y = sigmoid(h2 . w3 + b3 + prior), so that it learns
 * the correction to the Gaussian closed form in logit space.
 *
 * Parameters: one fp32 buffer of LCP_MLP_NPARAMS floats:
 *   W1 [64][32] at 0     (hidden unit n, feature k; columns 17..31 stay zero)
 *   b1 [64]     at 2048
 *   W2 [64][64] at 2112  (output unit n, input unit k)
 *   b2 [64]     at 6208
 *   w3 [64]     at 6272
 *   b3          at 6336  (3 floats of padding follow)
 */
#define LCP_MLP_FEAT_STRIDE 32
#define LCP_MLP_NPARAMS 6340

/*
 * lcp_moments - plug-in central moments of every vertex component over the
 * members: mom[comp][j][i] = (mean, m2, m3, m4) as float4 (divisor M), comp 0 =
 * u, 1 = v; shifted power sums about member 0 in FP32.  mom: device
 * [2][H][W][4] fp32 (16-byte aligned).  Member arguments as lcp_stats.
 */
lcp_status lcp_moments(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                       int64_t member_stride, float* mom, lcp_stream_t stream);

/*
 * lcp_surrogate_features - the network's input rows for every cell and
 * isovalue: feat[(k (H-1) + j)(W-1) + i][32] bf16 (device, 16-byte aligned)
 * and their priors prior[same row] fp32 (device, or NULL), from mom
 * (lcp_moments' layout).  iso: HOST array of K <= 64 fp32 values.
 */
lcp_status lcp_surrogate_features(const float* mom, int H, int W, double dx, double dy, const float* iso,
                                  int K, void* feat, float* prior, lcp_stream_t stream);

/*
 * lcp_mlp_forward - y[r] = network(feat[r], prior[r]) for r < n (feat bf16
 * [n][32], prior fp32 [n] or NULL for 0, y fp32 [n], params fp32 as above; all
 * device).
 */
lcp_status lcp_mlp_forward(const float* params, const void* feat, const float* prior, int64_t n, float* y,
                           lcp_stream_t stream);

/*
 * lcp_mlp_backward - gradient of the mean squared error
 * (1/n) sum_r (network(feat[r], prior[r]) - target[r])^2 with respect to every
 * parameter, written to grad (fp32 [LCP_MLP_NPARAMS], device; overwritten,
 * padding and the zero columns of W1 get 0).  loss (device fp32 scalar, or
 * NULL) receives the loss itself.  Forward and backward products and the
 * weight gradients (contractions over the rows) run as tcgen05.mma on the
 * tensor cores, BF16 operands, FP32-accumulated in tensor memory.
 */
lcp_status lcp_mlp_backward(const float* params, const void* feat, const float* prior, const float* target,
                            int64_t n, float* grad, float* loss, lcp_stream_t stream);

/*
 * lcp_mlp_backward_ws - lcp_mlp_backward with a result that is the same, bit
 * for bit, on every run on a device: each CTA sums its rows in a fixed order
 * (its warps' partial vectors added in warp order) and writes its partial
 * gradient to its own row of the workspace, and a second kernel adds the rows
 * in CTA order.  Training with it (and the element-wise Adam step) is
 * reproducible, so a run resumed from a checkpoint continues exactly as the
 * uninterrupted run.  workspace: device, 16-byte aligned, at least
 * lcp_mlp_backward_workspace_bytes(n) bytes (about 25 KB per CTA, one CTA per
 * SM at most); grad and loss are overwritten.  The paper has no
 * counterpart (the surrogate is this library's addition).
 */
size_t lcp_mlp_backward_workspace_bytes(int64_t n);
lcp_status lcp_mlp_backward_ws(const float* params, const void* feat, const float* prior, const float* target,
                               int64_t n, float* grad, float* loss, void* workspace, size_t workspace_bytes,
                               lcp_stream_t stream);

/*
 * lcp_adam_step - one Adam update (Kingma and Ba, ICLR 2015, Algorithm 1) of n
 * fp32 parameters in place: m, v (device, n floats each, zero before step 1)
 * are the moving averages of grad and grad^2, bias-corrected with step count
 * t >= 1.
 */
lcp_status lcp_adam_step(float* params, const float* grad, float* m, float* v, int64_t n, int t, float lr,
                         float beta1, float beta2, float eps, lcp_stream_t stream);

/*
 * lcp_mlp_infer - the learned LCP map from moments: per cell and isovalue the
 * features above and the network, fused in one kernel (no feature rows in
 * HBM).  lcp_out [K][H-1][W-1] of out_dtype (LCP_F32 or LCP_F16); iso HOST,
 * K <= 64.
 */
lcp_status lcp_mlp_infer(const float* mom, int H, int W, double dx, double dy, const float* iso, int K,
                         const float* params, void* lcp_out, lcp_dtype out_dtype, lcp_stream_t stream);

/*
 * lcp_exact_empirical - the exact LCP under the empirical model (every vertex
 * component an independent uniform draw from its own members): the value the
 * Monte Carlo estimator of Sec. 3.2 converges to, computed by counting.  At an
 * interior vertex the Eq. 1 divergence is X + Y with X over the M^2 pairs of
 * u members at i+1, i-1 and Y over the M^2 pairs of v members at j+1, j-1, so
 * P(D < c) = #{x + y < c} / M^4 (both lists sorted, counted with two
 * pointers).  Interior vertex stencils share no value, so for cells whose four
 * vertices are interior LCP = 1 - prod p - prod (1 - p) exactly.
 *   u, v       device members [M][H][W] (LCP_F32 or LCP_BF16), M <= 64, H, W >= 4
 *   iso        HOST, 1 <= K <= 64
 *   below      device fp32 [K][H][W] scratch: P(D < c) of the interior vertices
 *   lcp_out    device fp32 [K][H-1][W-1]: the LCP of cells (i, j) with
 *              1 <= i <= W-3 and 1 <= j <= H-3; NaN elsewhere (the one-sided
 *              stencils of the outer ring share members)
 * Arithmetic in FP32 (a pair within rounding of c may count on either side);
 * counts are exact integers.  Not for NaN members.
 */
lcp_status lcp_exact_empirical(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                               int64_t member_stride, double dx, double dy, const float* iso, int K, float* below,
                               float* lcp_out, lcp_stream_t stream);

/*
 * lcp_mc - classical Monte Carlo estimate of the LCP map (Sec. 3.2 and Sec. 4):
 * every sample is one realisation of the whole field; its divergence (Eq. 1,
 * same boundary rule) is tested per cell and isovalue, "crossing" meaning
 * min < c <= max over the 4 vertices; counts[k][j][i] is the number of
 * crossing samples.  The estimate is counts / n_samples.
 *
 * mode LCP_MC_GAUSS      U ~ N(mu_u, var_u), V ~ N(mu_v, var_v) per vertex
 *                        (fp32 [H][W] inputs; u, v ignored, may be NULL)
 * mode LCP_MC_EMPIRICAL  U, V drawn uniformly and independently from the M
 *                        members of their own vertex (u, v, in_dtype, M,
 *                        member_stride used; statistics ignored, may be NULL)
 * Random numbers: Philox-4x32-10 (Salmon et al., SC'11) with counter
 * (j*W + i, t, offset lo, offset hi) and key (seed lo, seed hi) gives 4 words
 * per vertex and sample pair t; sample 2t uses words 0, 1 and sample 2t+1 words
 * 2, 3.  GAUSS: Box-Muller on the word pair with U1 = (word >> 8 + 1/2) 2^-24,
 * z_u = sqrt(-2 ln U1) cos(2 pi U2), z_v = sqrt(-2 ln U1) sin(2 pi U2).
 * EMPIRICAL: member index = (word * M) >> 32 for u and v respectively.
 * iso           HOST array of K fp32 isovalues
 * n_samples     1 <= S <= 2^32 - 1
 * counts        uint32 [K][H-1][W-1] (required)
 * lcp_out       optional fp32 [K][H-1][W-1] estimate counts / S, or NULL
 * Errors: LCP_ERR_ARG also when H*W > 2^32.
 */
lcp_status lcp_mc(lcp_mc_mode mode, const float* mu_u, const float* var_u, const float* mu_v,
                  const float* var_v, const void* u, const void* v, lcp_dtype in_dtype, int M,
                  int64_t member_stride, int H, int W, double dx, double dy, const float* iso, int K,
                  int64_t n_samples, uint64_t seed, uint64_t offset, uint32_t* counts,
                  float* lcp_out, lcp_stream_t stream);

/*
 * lcp_device_status - read (and optionally clear) the library's device status
 * word on the current device.  Bit 0 is set when a bounded device-side wait
 * (the TMA pipeline's mbarrier waits, the workspace path's waits for
 * statistics rows) gave up; the affected outputs are then undefined (an LCP
 * block of the workspace path whose wait gave up writes NaN into its cells and
 * clears its mask bits instead of reading incomplete statistics).  This call
 * synchronises with the device.
 * Bit 1: a wait of the learned-surrogate inference (tcgen05 mbarrier) gave up.
 * Bit 2: a contour look-back wait gave up.
 * Returns LCP_ERR_TIMEOUT if any bit is set, LCP_OK otherwise; `flags` (host,
 * may be NULL) receives the word; `reset` != 0 clears it.
 */
lcp_status lcp_device_status(uint32_t* flags, int reset);

/*
 * lcp_set_wait_budget - the clock-cycle budget after which a bounded device
 * wait gives up: the workspace path's LCP blocks waiting for their statistics
 * rows (lcp_fused_ws, lcp_fused_static_ws, lcp_speed_gradient_ws) and the
 * contour look-back (lcp_contours, lcp_member_contours).  The budget is read
 * on the host at every launch and passed to the kernel.  `cycles` <= 0
 * restores the default, 4e9 cycles (about 2 s at 2 GHz).  Returns the budget in
 * force before the call.  Process-wide; not a property of the paper's method
 * (these waits exist because this library overlaps its kernels).  The TMA
 * pipeline's and the learned inference's mbarrier waits keep a fixed budget of
 * the same size.
 */
long long lcp_set_wait_budget(long long cycles);

/*
 * Failure-path probes.  Each launches one of the library's waiting kernels
 * against a flag that nothing in the launch will ever set, so that its bounded
 * wait must run out (use a small lcp_set_wait_budget first); the kernel then
 * sets its bit of lcp_device_status and finishes.  They exist to test the
 * timeout path without a faulty producer; the paper has no counterpart.
 *
 * lcp_test_stalled_lcp_wait - the LCP kernels of lcp_fused_ws for the cells of
 * the workspace layout's first row band, waiting on that band's statistics
 * counters, which it clears and no statistics kernel releases.  Arguments as
 * lcp_fused_ws's (no members).  Every cell of the band receives NaN and its
 * mask bits 0; lcp_device_status then reports bit 0.
 *
 * lcp_test_stalled_lookback - lcp_contours with the first tile's ticket never
 * handed out: the tile that takes ticket 1 waits for tile 0's look-back flag,
 * which no tile writes.  Needs at least two tiles (more than 992 cells).  The
 * segments of tile 0's cells are missing and the others placed as if tile 0
 * had none; lcp_device_status then reports bit 2.
 */
lcp_status lcp_test_stalled_lcp_wait(int H, int W, const float* iso, int K, void* lcp_out, lcp_dtype out_dtype,
                                     uint32_t* mask, void* workspace, size_t workspace_bytes, lcp_stream_t stream);
lcp_status lcp_test_stalled_lookback(const float* field, int H, int W, const float* iso, int K, float* seg,
                                     long long* key, int64_t capacity, unsigned long long* count, void* workspace,
                                     size_t workspace_bytes, lcp_stream_t stream);

/*
 * lcp_speed_gradient - the preprocessing of the Red Sea study (Sec. 4.2,
 * Fig. 3): per member the velocity magnitude s = sqrt(u^2 + v^2) and its
 * gradient with the stencil of Eq. 1 and the boundary rule above:
 *   gx = (s[i+] - s[i-]) / ((i+ - i-) dx),  gy = (s[j+] - s[j-]) / ((j+ - j-) dy).
 * u, v    device members [M][H][W] (LCP_F32 or LCP_BF16), member_stride as above
 * gx, gy  device fp32 outputs [M][H][W], contiguous (member stride H*W)
 * FP32 arithmetic.  Errors: as lcp_stats (ddof is not used), NULL outputs, or
 * dx, dy <= 0.
 */
lcp_status lcp_speed_gradient(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                              int64_t member_stride, double dx, double dy, float* gx, float* gy,
                              lcp_stream_t stream);

/*
 * lcp_speed_gradient_ws - the closed-form LCP map of the divergence of the
 * speed gradient (Sec. 4.2, Fig. 3d) with the preprocessing fused into the
 * statistics pass: every member value is read once, no gradient member is
 * stored, and the result equals lcp_fused_ws on the members of
 * lcp_speed_gradient up to FP32 rounding.  Arguments as lcp_fused_ws (the
 * workspace is sized by lcp_fused_workspace_bytes and must be non-NULL);
 * H * W < 2^31.
 */
lcp_status lcp_speed_gradient_ws(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                                 int64_t member_stride, int ddof, double dx, double dy, const float* iso, int K,
                                 void* lcp_out, lcp_dtype out_dtype, uint32_t* mask, void* workspace,
                                 size_t workspace_bytes, lcp_stream_t stream);

/*
 * 3D vector fields.  Sec. 5 names 3D fields as the next step; the closed form
 * carries over term by term.  A volume has D planes (z, index k) of H rows (y,
 * j) of W columns (x, i); element (m, k, j, i) of u lives at
 * u[m * member_stride + (k * H + j) * W + i], member_stride >= D*H*W; u is the
 * x, v the y and w the z component.  Eq. 1 gains (w[k+] - w[k-]) / ((k+ - k-) dz)
 * with the same one-sided rule on every face; Eqs. 2/3 gain the matching terms.
 * Cell (i, j, k) has the 8 vertices (i..i+1, j..j+1, k..k+1) and
 *   LCP = 1 - prod_8 P(D < c) - prod_8 P(D >= c).
 * Maps are [K][D-1][H-1][W-1]; masks [K][D-1][H-1][ceil((W-1)/32)] words with
 * bit (i % 32) of word i / 32 set iff the mean-field cell crosses.
 */

/* Workspace bytes of lcp3d_fused_ws: a ring of z-planes of statistics records
 * (48 bytes per vertex) sized to stay in L2 where the planes allow it. */
size_t lcp3d_workspace_bytes(int M, int D, int H, int W, lcp_dtype in_dtype);

/*
 * lcp3d_fused_ws - members of (u, v, w) -> the 3D LCP map (and mask): FP32
 * shifted-sum statistics per vertex (read once), the 3D divergence Gaussian and
 * the LCP of every hexahedral cell and isovalue.
 *   u, v, w    device members (LCP_F32 or LCP_BF16), layout above
 *   M, D, H, W, member_stride, ddof, dx, dy, dz   as for the 2D calls
 *   iso        HOST, 1 <= K <= LCP_MAX_ISOVALUES (passes of up to 8)
 *   lcp_out    device [K][D-1][H-1][W-1] of out_dtype (LCP_F32 or LCP_F16)
 *   mask       optional device words (layout above, cleared by the call) or NULL
 *   workspace  device, 256-byte aligned, >= lcp3d_workspace_bytes
 * Errors: LCP_ERR_ARG for NULL pointers, D, H or W < 2, M - ddof < 1, a small
 * member_stride or workspace, dx, dy or dz <= 0, a bad dtype or K.
 */
lcp_status lcp3d_fused_ws(const void* u, const void* v, const void* w, lcp_dtype in_dtype, int M, int D, int H,
                          int W, int64_t member_stride, int ddof, double dx, double dy, double dz, const float* iso,
                          int K, void* lcp_out, lcp_dtype out_dtype, uint32_t* mask, void* workspace,
                          size_t workspace_bytes, lcp_stream_t stream);

/*
 * lcp3d_divergence - the 3D divergence Gaussian at every vertex from per-vertex
 * statistics (device fp32 [D][H][W] each, e.g. from lcp_stats on (u, v) and on
 * (w, w)); outputs mu_d, var_d device fp32 [D][H][W].
 */
lcp_status lcp3d_divergence(const float* mu_u, const float* var_u, const float* mu_v, const float* var_v,
                            const float* mu_w, const float* var_w, int D, int H, int W, double dx, double dy,
                            double dz, float* mu_d, float* var_d, lcp_stream_t stream);

/*
 * lcp3d_map - the LCP of every hexahedral cell from the divergence Gaussians
 * (device fp32 [D][H][W]); iso HOST, 1 <= K <= 64; lcp_out and mask as above
 * (the mask is written, not accumulated).
 */
lcp_status lcp3d_map(const float* mu_d, const float* var_d, int D, int H, int W, const float* iso, int K,
                     void* lcp_out, lcp_dtype out_dtype, uint32_t* mask, lcp_stream_t stream);

/*
 * Isocontour segments (marching squares).  The paper draws the mean-field
 * divergence isocontour (Fig. 1a, Fig. 3c) and the spaghetti plot of every
 * member's isocontour (Fig. 1b).  Cell (i, j) has corners v0 = (i, j),
 * v1 = (i+1, j), v2 = (i+1, j+1), v3 = (i, j+1); a corner is below when
 * f < c; edges E0 = v0v1, E1 = v1v2, E2 = v3v2, E3 = v0v3 cross where their
 * corners differ.  A crossing point is interpolated from the edge's
 * lower-coordinate vertex in fp32 (x = i + (c - f(i,j)) / (f(i+1,j) - f(i,j))
 * on a horizontal edge, y likewise on a vertical one), so neighbouring cells
 * produce the same shared point.  Two crossing edges give one segment (lower
 * edge first); the saddles (v0, v2 on one side of c, v1, v3 on the other) give
 * two: if the centre value ((f0 + f1) + (f2 + f3)) * 0.25, each operation an
 * fp32 operation rounded to nearest, lies on v0's side, (E0, E1) and (E2, E3),
 * else (E0, E3) and (E1, E2).  Cells with a NaN corner give none.
 *
 * Output: seg device fp32 [capacity][4] = (x0, y0, x1, y1) in grid units
 * (x = column, y = row), 16-byte aligned; key device int64 [capacity] or NULL,
 * ((j (W-1) + i) K + k) 2 + s (s = 0, 1 within the cell; member m adds
 * m (H-1)(W-1) K 2).  Segments are written in increasing key order, the same
 * on every run; count (device uint64) receives the total, of which the first
 * min(total, capacity) are stored.  The workspace (device, 256-byte aligned,
 * lcp_contours_workspace_bytes) is cleared by the call; H, W < 2^24.  A look-back wait
 * that gives up (it should not) sets bit 2 of lcp_device_status.
 */
size_t lcp_contours_workspace_bytes(int M, int H, int W);

/* Segments of a scalar field f (device fp32 [H][W], e.g. mu_d of
 * lcp_divergence) for K <= 64 isovalues (HOST array). */
lcp_status lcp_contours(const float* field, int H, int W, const float* iso, int K, float* seg, long long* key,
                        int64_t capacity, unsigned long long* count, void* workspace, size_t workspace_bytes,
                        lcp_stream_t stream);

/* Segments of every member's Eq. 1 divergence (the spaghetti plot), formed in
 * fp32 as (u[i+] - u[i-]) * sx + (v[j+] - v[j-]) * sy with sx = fp32(1 / ((i+ - i-) dx))
 * (likewise sy), each operation rounded to nearest.  Members as for
 * lcp_stats; K <= 64. */
lcp_status lcp_member_contours(const void* u, const void* v, lcp_dtype in_dtype, int M, int H, int W,
                               int64_t member_stride, double dx, double dy, const float* iso, int K, float* seg,
                               long long* key, int64_t capacity, unsigned long long* count, void* workspace,
                               size_t workspace_bytes, lcp_stream_t stream);

/*
 * lcp_colormap - colour mapping of a scalar map into a headless RGBA8 buffer.
 * Sec. 3.1 (last paragraph) shows the LCP map by colour mapping, and Sec. 4.2
 * clamps the mean-field divergence to a display range before mapping it
 * (Fig. 3c).  No graphics API is involved: the result is plain bytes in device
 * memory.
 *
 * values  device fp32 [planes][rows][cols] (contiguous), e.g. an LCP map
 *         [K][H-1][W-1]
 * vmin, vmax   display range, finite, vmin < vmax, with vmax - vmin finite
 *         in fp32 (below about 3.4e38)
 * stops   HOST array of n_stops x 5 floats (t, r, g, b, a), every entry in
 *         [0, 1], t strictly increasing from exactly 0 to exactly 1;
 *         2 <= n_stops <= LCP_MAX_COLOR_STOPS
 * nan_rgba   packed colour (r | g << 8 | b << 16 | a << 24) of NaN values
 * mask    optional device crossing bits for rows x cols cells in the library's
 *         mask layout ([planes][rows][ceil(cols/32)] uint32), or NULL; a set
 *         bit paints mask_rgba (the mean-field contour cells, Fig. 1a)
 * rgba    device uint8 [planes][rows][cols][4], bytes r, g, b, a per value
 *
 * The map (the mathematics): per value x, NaN -> nan_rgba; else if the mask
 * bit is set -> mask_rgba; else t = clamp((x - vmin) / (vmax - vmin), 0, 1)
 * (+inf -> 1, -inf -> 0), s = the largest stop index <= n_stops - 2 with
 * t_s <= t, ch = c_s + (t - t_s) / (t_{s+1} - t_s) (c_{s+1} - c_s) for each of
 * r, g, b, a, byte = floor(255 ch + 1/2).
 * The kernel evaluates it in fp32: R = 1 / (vmax - vmin), r_s = 1 / (t_{s+1} -
 * t_s) and d_s = c_{s+1} - c_s once per call, then t = clamp((x - vmin) R),
 * f = (t - t_s) r_s, ch = c_s + f d_s, each one operation rounded to nearest.
 * A byte therefore equals the exact one except where 255 ch + 1/2 lies within
 * about 2^-24 (255 (4 |d_s| r_s + 6 |d_s| + 2) + 512) of an integer, where it
 * can differ by one.
 * Alignment: values, mask and rgba 4-byte aligned (16 bytes gives vector
 * access).  Errors: LCP_ERR_ARG for a negative size, NULL pointers (n > 0),
 * a bad range or stop table, or misalignment.  planes * rows * cols == 0 is a
 * no-op.
 */
#define LCP_MAX_COLOR_STOPS 16
lcp_status lcp_colormap(const float* values, int planes, int rows, int cols, float vmin, float vmax,
                        const float* stops, int n_stops, uint32_t nan_rgba, const uint32_t* mask,
                        uint32_t mask_rgba, uint8_t* rgba, lcp_stream_t stream);

/*
 * lcp_philox_fill - the Monte Carlo generator's raw words, for testing and
 * for reproducible inputs: out[4 n + r] = word r of Philox-4x32-10 with counter
 * (n, c1, offset lo, offset hi) and key (seed lo, seed hi), n in [0, count).
 * out: uint32 [4 * count] device array; 0 <= count <= 2^32.
 */
lcp_status lcp_philox_fill(uint64_t seed, uint32_t c1, uint64_t offset, int64_t count,
                           uint32_t* out, lcp_stream_t stream);

/*
 * Multi-GPU partition (host arithmetic; no device work, no allocation).
 *
 * The LCP of a cell depends only on its four vertices' statistics and their
 * stencil neighbours (Eqs. 2/3; the paper's per-pixel data parallelism,
 * Sec. 3.3), so one field splits over ranks into strips of cell rows that need
 * no exchange: each rank re-reads a halo of member rows.
 *
 * lcp_strip_plan - rank `rank` of `nranks` (0 <= rank < nranks) takes the cell
 * rows [cell_begin, cell_end) = [floor(rank (H-1) / nranks), floor((rank+1)
 * (H-1) / nranks)); to compute them it reads the vertex rows [vrow_begin,
 * vrow_end) = [max(cell_begin - 1, 0), min(cell_end + 2, H)) of every member
 * and evaluates them as a grid of their own (same W, member_stride and
 * spacing, u and v advanced by vrow_begin * W elements).  Of that sub-grid's
 * cell rows it keeps [cell_begin - vrow_begin, cell_end - vrow_begin): the
 * others sit next to a halo row whose one-sided difference is not the full
 * grid's.  The kept rows equal the whole-grid result exactly.  More ranks
 * than cell rows leave some strips empty (vrow_begin == vrow_end).  Errors:
 * LCP_ERR_ARG for H < 2, a rank outside [0, nranks) or NULL outputs.
 */
lcp_status lcp_strip_plan(int H, int nranks, int rank, int* vrow_begin, int* vrow_end, int* cell_begin,
                          int* cell_end);

/*
 * lcp_lpt_assign - whole fields of a batch to ranks by the
 * longest-processing-time rule: fields in decreasing cost (ties in index
 * order), each to the currently least-loaded rank (ties to the lowest rank),
 * so that every rank computes the same plan.  cost: n host int64 >= 0 (e.g.
 * member bytes); owner: n host ints receive the rank of each field; load
 * (nranks host int64, may be NULL) receives each rank's total.  The largest
 * load is at most (4/3 - 1/(3 nranks)) of the best possible (Graham, 1969).
 */
lcp_status lcp_lpt_assign(const int64_t* cost, int n, int nranks, int* owner, int64_t* load);

#ifdef __cplusplus
}
#endif

#endif /* LCP_GB300_H */
