/*
 * gpr_lcp.h -- C ABI of the GB300 library for Gaussian-process reconstruction
 * and level-crossing probability (LCP) fields.
 *
 * Method: Li, Michaud, Biswas, Shen, "Efficient Level-Crossing Probability
 * Calculation for Gaussian Process Modeled Data".  Paper passages are cited as
 * Sec./Eq./Algorithm numbers.
 *
 * Conventions shared by every entry point
 *   - All calls return gpr_status.  Argument errors are detected on the host
 *     and returned before any work is queued.  Errors raised on the device
 *     (non positive-definite K, a bounded wait that ran out) are written to the
 *     model's device status word and returned by gpr_sync() or by the next
 *     call that synchronises.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is queued asynchronously on it unless stated otherwise.
 *   - Pointers marked "device" must be device (or managed) memory of the
 *     current CUDA device; pointers marked "host" must be host memory.
 *     Caller-owned buffers are never freed by the library.
 *   - Grids: n[d] >= 2 points per axis, coordinates x_i = lo + i (hi-lo)/(n-1),
 *     linear point index i + n0 (j + n1 k) (x fastest).  Cells are indexed by
 *     their minimum corner, linear index i + (n0-1)(j + (n1-1) k); a cell's
 *     corner c = bx + 2 by + 4 bz sits at (i+bx, j+by, k+bz).
 *   - Per-point statistics ("stats15"): slot 0 = posterior mean, 1 = variance,
 *     2+e = covariance with the forward neighbour p + OFF[e], where OFF is
 *     (1,-1,-1) (1,-1,0) (1,-1,1) (1,0,-1) (1,0,0) (1,0,1) (1,1,-1) (1,1,0)
 *     (1,1,1) (0,1,-1) (0,1,0) (0,1,1) (0,0,1); NaN where the neighbour is off
 *     the grid.  These 15 numbers per point determine every cell's 8x8 corner
 *     covariance (Sec. 4).
 */
#ifndef GPR_LCP_H
#define GPR_LCP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gpr_model gpr_model; /* opaque; owns its device buffers */

typedef enum {
    GPR_OK = 0,
    GPR_ERR_ARG = 1,         /* invalid argument (host check) */
    GPR_ERR_NOT_PD = 2,      /* K(X,X) + noise I not positive definite */
    GPR_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    GPR_ERR_OOM = 4,         /* device allocation failed */
    GPR_ERR_TIMEOUT = 5,     /* a bounded device wait ran out */
    GPR_ERR_UNSUPPORTED = 6  /* valid request this library does not serve */
} gpr_status;

typedef enum { GPR_K_SE = 0, GPR_K_MATERN52 = 1 } gpr_kernel;

/* Arithmetic of the O(m^2 n) contraction (the Cholesky, the inverse and the
 * solves are FP64 in every mode).  GPR_P_FP64 is the only mode whose
 * covariances are accurate enough for the cell LCP; the others serve the
 * posterior mean/variance, the octree bounds and the LCP pre-classification. */
typedef enum {
    GPR_P_FP64 = 0,   /* FP64 CUDA cores */
    GPR_P_FP32 = 1,   /* FP32 CUDA cores */
    GPR_P_TF32 = 2,   /* tcgen05 kind::tf32, FP32 accumulate in TMEM */
    GPR_P_TF32X3 = 3, /* three TF32 products (hi*hi + hi*lo + lo*hi) */
    GPR_P_BF16 = 4,   /* tcgen05 kind::f16 with bf16 operands */
    GPR_P_BF16X3 = 5  /* three bf16 slices, six products */
} gpr_precision;

/* Cell estimators (Sec. 4 and the alternatives the paper reviews, Sec. 2.2 and Sec. 9):
 *   GPR_EST_SOV_QMC   the orthant probabilities by sequential conditioning on a lattice
 *   GPR_EST_MC        the paper's Monte Carlo estimator
 *   GPR_EST_INDEP     closed form with the corners taken as independent (correlation ignored):
 *                     1 - prod_c P(Y_c < theta) - prod_c P(Y_c > theta)
 *   GPR_EST_EDGE_MAX  Pothkow et al.'s approximation: the largest edge-crossing probability
 *                     1 - P(Y_i < theta, Y_j < theta) - P(Y_i > theta, Y_j > theta) over the 12
 *                     cell edges, bivariate normal probabilities by Owen's T function
 *   GPR_EST_SOV_ORDERED  GPR_EST_SOV_QMC with each orthant's corners taken in ascending order
 *                     of their standardised thresholds s (theta - mu_c) / sigma_c (s = +1 for
 *                     all-below, -1 for all-above; ties by corner index; the order is decided
 *                     in FP64), so each orthant has its own Cholesky factor.  Same lattice and
 *                     no more work per sample; on strongly correlated corners far more accurate
 *                     at the same sample count.  Forward only: the backward calls, and the
 *                     allocation-free entry point, return GPR_ERR_UNSUPPORTED for it. */
typedef enum {
    GPR_EST_SOV_QMC = 0,
    GPR_EST_MC = 1,
    GPR_EST_INDEP = 2,
    GPR_EST_EDGE_MAX = 3,
    GPR_EST_SOV_ORDERED = 4
} gpr_estimator;

/* Arithmetic of the FP64-class reconstruction of the LCP cells' corners.
 * GPR_EXACT_AUTO: BF16 tensor cores with an error-free split of both operands into
 * seven 6-bit digit slices (28 products, exact FP32 accumulation for m <= 1024, SE
 * kernels) and float-float statistics; FP64 CUDA cores otherwise.
 * GPR_EXACT_FP64: always FP64 CUDA cores. */
typedef enum { GPR_EXACT_AUTO = 0, GPR_EXACT_FP64 = 1 } gpr_exact_mode;

typedef struct {
    double lo[3], hi[3];
    int32_t n[3]; /* points per axis */
} gpr_grid;

/* Subdivision of the adaptive query: the paper's octree (Algorithm 1), or the K-D tree it
 * proposes as future work (Sec. 9), which halves one axis per level (x, y, z in turn), so a
 * region can be dropped after one halving instead of three; max_depth D keeps its meaning
 * (cell cube 2^D per axis) and the K-D tree has 3D + 1 levels. */
typedef enum { GPR_TREE_OCTREE = 0, GPR_TREE_KD = 1 } gpr_tree;

/* Options of the LCP calls.  Defaults come from gpr_lcp_options_default(). */
typedef struct {
    double alpha;          /* octree threshold (Algorithm 1), default 1e-3 (Sec. 7.3) */
    double beta;           /* local model of the octree bound (Sec. 5.2): beta >= 0 minimises each node's bound on
                              the model restricted to the observations inside the node box enlarged by
                              beta * l_d per axis (the paper uses 6, Sec. 7.3); beta < 0 or +inf uses the full
                              model (default -1: on this GPU the full model's bound is the cheaper one) */
    gpr_estimator est;     /* cell estimator, default SOV-QMC */
    int32_t n_samples;     /* samples per cell, default 1600 (Sec. 6.4) */
    uint64_t seed;         /* lattice shifts / Philox key */
    double jitter;         /* tau: Sigma_8 += tau * max diag * I, default 1e-10 (the LCP then agrees with
                              the unregularised Sigma_8 of Sec. 4 to 1e-6) */
    double skip_eps;       /* Boole pre-skip threshold, default 1e-9 */
    gpr_precision prec;    /* precision of the pre-classification / octree pass, default GPR_P_FP32 */
    int32_t max_iters_min; /* projected steps T of the box minimiser, default 4 */
    gpr_exact_mode exact;  /* FP64-class corner statistics: tensor-core digit split or FP64, default AUTO */
    gpr_tree tree;         /* subdivision of the adaptive query, default GPR_TREE_OCTREE */
} gpr_lcp_options;

typedef struct {
    int64_t nodes_per_level[24];   /* nodes evaluated at each level of Algorithm 1 (the first 24) */
    int64_t subdiv_per_level[24];  /* nodes subdivided at each level */
    int64_t leaf_cells;            /* |S|: cells kept at the deepest level */
    int64_t recon_points;          /* grid points whose FP64-class rows this call reconstructed (points
                                      cached by earlier calls on the same model and grid are not
                                      counted again) */
    int64_t cells_estimated;       /* cells that ran the estimator (not pre-skipped) */
} gpr_adaptive_stats;

/* Fills the defaults listed above. */
void gpr_lcp_options_default(gpr_lcp_options *opts);

/* Human-readable name of a status code (static storage). */
const char *gpr_status_string(gpr_status s);

/*
 * gpr_model_create -- builds the stored GP model (Sec. 3, Eq. 1 with the
 * observations as inducing set):  Kt = K(X,X) + noise_var I = L L^T (FP64
 * blocked Cholesky on the device), L^-1, v = L^-1 y, alpha = Kt^-1 y, and the
 * latent posterior at the observations (mean y - noise_var alpha, variance
 * noise_var - noise_var^2 [Kt^-1]_ii) used by Algorithm 1's p1/p2 test.
 *   obs_xyz  host, m x 3 row-major FP64 observation sites
 *   y        host, m FP64 observation values
 *   m        1 <= m <= 8192
 *   kernel   GPR_K_SE: k = s exp(-sum_d (dx_d/l_d)^2 / 2)  (the paper's RBF,
 *            Sec. 3, with one length per axis); GPR_K_MATERN52: the
 *            Matern-5/2 function of r = |dx / l|
 *   length_scales host[3] > 0;  signal_var > 0;  noise_var >= 0
 *   stream   queue for the set-up kernels
 *   out      receives the model; the call synchronises `stream` and returns
 *            GPR_ERR_NOT_PD if a Cholesky pivot is not positive.
 * The model owns its device memory until gpr_model_destroy().
 */
gpr_status gpr_model_create(const double *obs_xyz, const double *y, int64_t m, gpr_kernel kernel,
                            const double length_scales[3], double signal_var, double noise_var,
                            void *stream, gpr_model **out);

/*
 * gpr_model_create_sgpr -- the general stored model of Sec. 3: a sparse GP given by
 * m inducing sites and the distribution N(mu_M, A_M) of the field values there
 * (as a fitted SGPR model stores it), whose posterior is Eq. 1:
 *   mu(x)      = k_xM K_MM^-1 mu_M
 *   Sigma(a,b) = k(a,b) - k_aM K_MM^-1 k_Mb + k_aM K_MM^-1 A_M K_MM^-1 k_Mb,
 * with K_MM = K(M, M) + kmm_jitter I.  Built on the device in FP64: the
 * Cholesky factor of K_MM, alpha = K_MM^-1 mu_M, and the lower-triangular G
 * with G^T G = K_MM^-1 - K_MM^-1 A_M K_MM^-1 (a Cholesky factorisation in
 * reversed index order), so that Sigma(a,b) = k(a,b) - (G k_a).(G k_b) and every
 * other entry point computes Eq. 1 with the same kernels as for plain GPR.
 * Algorithm 1's p-test (Sec. 5.3) reads mu_M and diag(A_M) directly.
 *   inducing_xyz  host, m x 3 row-major FP64 sites
 *   mu_M          host, m FP64;   A_M  host, m x m row-major FP64, symmetric
 *   kmm_jitter    >= 0 added to the diagonal of K_MM (fitting libraries add one)
 *   other arguments as gpr_model_create (no noise term: Eq. 1 has none)
 * Returns GPR_ERR_NOT_PD if K_MM + kmm_jitter I is not positive definite, or if
 * A_M is not strictly below K_MM (K_MM - A_M must be positive definite, as it is
 * for any inducing distribution conditioned on data).  gpr_lcp_backward does
 * not serve these models (GPR_ERR_UNSUPPORTED).  Synchronises `stream`.
 */
gpr_status gpr_model_create_sgpr(const double *inducing_xyz, const double *mu_M, const double *A_M, int64_t m,
                                 gpr_kernel kernel, const double length_scales[3], double signal_var,
                                 double kmm_jitter, void *stream, gpr_model **out);

/* Frees the model and its workspace (synchronises the device first). */
gpr_status gpr_model_destroy(gpr_model *model);

/* Observation count of a model. */
int64_t gpr_model_m(const gpr_model *model);

/*
 * gpr_reconstruct_dense -- posterior statistics at every grid point (Eq. 1):
 * mean mu(x) = k_x^T Kt^-1 y and variance k(x,x) - k_x^T Kt^-1 k_x, computed in
 * the whitened form w = L^-1 k_x (mu = w . L^-1 y, var = k(x,x) - |w|^2), with
 * kernel rows generated on the fly (never stored).
 *   prec == GPR_P_FP64: mean/var/cov13 are double* (device, n, n, n x 13).
 *   other precisions:   mean/var/cov13 are float*; the O(m^2) part runs in that
 *   precision, while the mean k_x . Kt^-1 y (O(m) per point, but a sum of terms
 *   ~1e3 times larger than the result) is summed in float-float arithmetic.
 *   cov13 may be NULL; if given, slot e holds cov(p, p + OFF[e]) (see top); for the
 *   tensor-core precisions the whitened rows of that precision are then written to HBM
 *   in z-slabs and reduced by the FP32 statistics kernel (for precision studies).
 *   The call may grow the model's workspace (cudaMalloc) on first use of a
 *   larger grid.
 */
gpr_status gpr_reconstruct_dense(gpr_model *model, const gpr_grid *grid, gpr_precision prec,
                                 void *mean, void *var, void *cov13, void *stream);

/*
 * gpr_stats_points -- stats15 (FP64) for an arbitrary list of grid points.
 *   point_idx  device, count int64 linear grid indices
 *   stats      device, count x 15 double (layout above); covariances whose
 *              neighbour is not in the list are NaN
 */
gpr_status gpr_stats_points(gpr_model *model, const gpr_grid *grid, const int64_t *point_idx, int64_t count,
                            double *stats, void *stream);

/*
 * gpr_cell_lcp_from_stats -- cell LCP (Sec. 4): LCP = 1 - P(all 8 corners <
 * theta) - P(all 8 corners > theta) for the listed cells, from FP64 stats15 of
 * a full grid (device, n x 15 double).  Sigma_8 gets jitter*max(diag) on its
 * diagonal; if sum_c P(Y_c > theta) or sum_c P(Y_c < theta) is below skip_eps
 * the LCP is 0 (Boole's inequality); a cell with a corner variance that is not
 * positive after the jitter describes no Gaussian and gets NaN; otherwise the
 * Cholesky pivots of Sigma_8 are floored at 1e-3 * jitter * max variance (harmless
 * for rounding-level indefiniteness; statistics far from any covariance, such as
 * single-pass TF32/BF16 ones, may still give NaN) and the estimator of opts->est
 * runs:
 *   SOV-QMC: Genz's sequential conditioning over corners 0..7 in index order,
 *            n_samples points of the rank-1 lattice with generators frac(sqrt p)
 *            (p = 2,3,5,...,17) as 32-bit fractions, shifted per cell by the
 *            SplitMix64 outputs 8 cell + i + 1 (top 32 bits), tent-periodised.
 *   MC:      the paper's estimator: n_samples draws of the 8-variate Gaussian
 *            (Philox-4x32-10, key = seed, counter = (sample, cell, 0|1), Box-
 *            Muller), LCP = fraction of draws whose corners straddle theta.
 *   cell_idx  device, count int64 linear cell indices (NULL = every cell, in order)
 *   lcp       device float, count values (or every cell when cell_idx is NULL)
 */
gpr_status gpr_cell_lcp_from_stats(const gpr_grid *grid, const double *stats15, double isovalue,
                                   const gpr_lcp_options *opts, const int64_t *cell_idx, int64_t count,
                                   float *lcp, void *stream);

/*
 * gpr_lcp_dense -- the dense baseline LCP field (Sec. 4, Sec. 6.4): every cell's
 * LCP.  A pre-pass in opts->prec computes mean/variance at all points and drops
 * cells whose Boole bound, widened by a margin that covers that precision's
 * error, is below skip_eps; the remaining cells' corners are reconstructed in
 * FP64 and estimated.  Result equals the all-FP64 computation.
 *   lcp  device float, (n0-1)(n1-1)(n2-1) values
 */
gpr_status gpr_lcp_dense(gpr_model *model, const gpr_grid *grid, double isovalue, const gpr_lcp_options *opts,
                         float *lcp, gpr_adaptive_stats *stats, void *stream);

/*
 * gpr_lcp_adaptive -- Algorithm 1 (Sec. 5.3) then leaf reconstruction: the
 * octree over the cell grid (root = cells [0, 2^D)^3) is refined level by level
 * on the device.  A node is subdivided when the observations inside it have
 * p1 > alpha and p2 > alpha, or when the regional upper bound 1 - B_l^d - B_u^d
 * (Eq. upper_bound; one-sided when the p-test says so) exceeds alpha; B is the
 * minimum of Phi(+-(theta - mu)/sigma) over the node (exact over grid points
 * when the node has <= 3 points per axis, else a 3x3x3 lattice start plus
 * opts->max_iters_min projected gradient steps).  Cells kept at depth D form S;
 * their LCP is computed exactly as gpr_lcp_dense does and all other cells are 0.
 *   max_depth  D with 2^D >= n_d - 1 for every axis, D <= 20
 *   lcp        device float, one value per cell
 *   stats      host, nullable: per-level counts and |S|
 */
gpr_status gpr_lcp_adaptive(gpr_model *model, const gpr_grid *grid, double isovalue, int32_t max_depth,
                            const gpr_lcp_options *opts, float *lcp, gpr_adaptive_stats *stats, void *stream);

/*
 * gpr_lcp_adaptive_batched -- many fields at once (no counterpart in the paper,
 * which treats one field per run): field i is gpr_lcp_adaptive(models[i],
 * &grids[i], isovalues[i], max_depths[i], opts, lcps[i]) and its result is the
 * same, value for value.  Fields are grouped by model (entries that share a
 * model run one after another and share its grid cache), the groups are ordered
 * by estimated cost (m^2 times the grid's face area, largest first) and taken by
 * a pool of host worker threads, each with its own CUDA stream and a pooled
 * device workspace, so small and large fields overlap on the GPU.  The cells
 * that need the estimator, from every field, are collected in one record
 * buffer and estimated by ONE persistent launch at the end.
 *   models, grids, isovalues, max_depths, lcps   host arrays of `count` entries;
 *                lcps[i] is a device float array of field i's cells
 *   stats        host, nullable: `count` entries, as gpr_lcp_adaptive fills them
 *   stream       the work is ordered after earlier work on `stream`, and later
 *                work on `stream` sees the results; the call returns when the
 *                host-side scheduling is done (results may still be in flight)
 * Argument errors (any entry) return GPR_ERR_ARG before any work; otherwise
 * the status of the first failing field (in index order) is returned.  The
 * environment variable GPR_BATCH_WORKERS (1..64, default 8) sets the pool size.
 */
gpr_status gpr_lcp_adaptive_batched(gpr_model *const *models, const gpr_grid *grids, const double *isovalues,
                                    const int32_t *max_depths, int32_t count, const gpr_lcp_options *opts,
                                    float *const *lcps, gpr_adaptive_stats *stats, void *stream);

/* Frees the library's pooled device scratch that is kept between calls: the batch workers'
 * workspaces and record buffer, and the digit buffers of the tensor-core FP64-class products
 * (those no call is using; up to a few GB).  Synchronises the device. */
gpr_status gpr_batch_release(void);

/*
 * gpr_cell_lcp_from_stats_noalloc -- no counterpart in the paper.  The same cell
 * LCP as gpr_cell_lcp_from_stats (same arguments, same results), for callers that
 * may not allocate device memory when they call: a plug-in inside an application
 * or framework that owns the device memory through its own pool allocator, or a
 * latency-critical loop (cudaFree synchronises the whole device).
 *   - Allocates nothing: the estimator's scratch is a static device array of the
 *     library holding GPR_NOALLOC_MAX_CELLS cell records (~3 MB), kept by every
 *     GPU that loads the library until the process exits.
 *   - count (or, with cell_idx == NULL, the grid's cell count) must be at most
 *     GPR_NOALLOC_MAX_CELLS, else GPR_ERR_ARG; split larger requests.
 *   - The first call on a device resolves the array's device address on that
 *     device (cudaGetSymbolAddress, with the device current); make that first call
 *     before any stream capture on the device.
 *   - All calls share the array and it keeps the last call's contents; calls that
 *     overlap on the GPU race on it, so order them (one stream, or events).
 *   - Cell indices off the grid are skipped (their output is left unchanged) and
 *     reported as GPR_ERR_ARG by the next gpr_sync(), as for gpr_cell_lcp_from_stats.
 */
#define GPR_NOALLOC_MAX_CELLS 16384
gpr_status gpr_cell_lcp_from_stats_noalloc(const gpr_grid *grid, const double *stats15, double isovalue,
                                           const gpr_lcp_options *opts, const int64_t *cell_idx, int64_t count,
                                           float *lcp, void *stream);

/*
 * gpr_lcp_backward -- hand-written adjoint (no counterpart in the paper) of
 * loss = sum_c dL_dlcp[c] * LCP_c, the SOV-QMC cell LCP of gpr_lcp_dense, with
 * respect to the observation values y and the log length scales.  The forward
 * quantities are recomputed (kernel rows regenerated, never stored): FP64-class
 * whitened rows of the kept cells' corners (the tensor-core digit split widened
 * to FP64 under GPR_EXACT_AUTO where it applies, FP64 cores under
 * GPR_EXACT_FP64 or for Matern kernels), the reverse sweep of the estimator
 * per cell (FP32 samples, FP64 8x8 Cholesky adjoint), then through Eq. 1 in
 * FP64.  Cells with dL_dlcp[c] == 0 or dropped by the Boole test contribute 0.
 *   dL_dlcp     device float, one weight per cell
 *   dL_dy       host double[m];  dL_dloglen host double[3]
 * Synchronises `stream`.  opts->est must be GPR_EST_SOV_QMC (the indicator
 * MC estimator is piecewise constant), else GPR_ERR_UNSUPPORTED.
 */
gpr_status gpr_lcp_backward(gpr_model *model, const gpr_grid *grid, double isovalue, const gpr_lcp_options *opts,
                            const float *dL_dlcp, double *dL_dy, double *dL_dloglen, void *stream);

/*
 * gpr_lcp_backward_adaptive -- as gpr_lcp_backward, for the adaptive field of
 * gpr_lcp_adaptive (same model, grid, isovalue, max_depth and opts): Algorithm 1
 * (Sec. 5.3) is run again on the device to find the leaf cells S, and cells outside
 * S (whose adaptive LCP is the constant 0) contribute 0 whatever their weight.
 * The set S itself is piecewise constant in y and the length scales, so this is
 * the gradient of the adaptive field wherever it is differentiable.
 *   max_depth  D as for gpr_lcp_adaptive
 *   other arguments, errors and synchronisation as gpr_lcp_backward; the call
 *   allocates one byte per cell for S (stream-ordered) and frees it before it
 *   returns.
 */
gpr_status gpr_lcp_backward_adaptive(gpr_model *model, const gpr_grid *grid, double isovalue, int32_t max_depth,
                                     const gpr_lcp_options *opts, const float *dL_dlcp, double *dL_dy,
                                     double *dL_dloglen, void *stream);

/* ---- Autotuner (no counterpart in the paper).  Launches with interchangeable shapes (the
 * tensor-core pre-pass tile width per precision, the estimator's CTAs per SM) are timed on
 * first use per (kernel, size bucket) and the fastest is kept for the process; the choice never
 * changes results.  GPR_AUTOTUNE=0 disables timing (first alternative always);
 * GPR_TUNE_FILE=<path> loads the table at first use and rewrites it on every new entry.
 * gpr_autotune_table writes the table as "kernel bucket choice" lines into buf (host, len
 * bytes, NUL-terminated, truncated if short) and returns the full length. */
int64_t gpr_autotune_table(char *buf, int64_t len);
/* Forgets every tuned choice. */
void gpr_autotune_clear(void);

/* Waits for `stream` and returns the first device-side error recorded on the
 * current device since the last call (GPR_OK if none); the status word is one
 * per device, held by the library (no allocation). */
gpr_status gpr_sync(void *stream);

/* ---- Tracing (no counterpart in the paper; the paper reports per-phase wall time,
 * Sec. 6.2).  When enabled, the library records CUDA events on the launching stream
 * around its main kernels, grouped by name ("w64", "meanvar32", "stats_from_w64",
 * "cell_prep", "sov", "mc", "classify", ...).  Independently of this switch, every call
 * below that computes opens an NVTX range named after itself, with nested ranges for its
 * phases ("algorithm1_levels", "leaf_lcp", "batched_estimator" and the group names above),
 * for a profiler attached through NVTX (a no-op otherwise). */
void gpr_profile_enable(int on);
/* Clears the accumulated times and the launch counter. */
void gpr_profile_reset(void);
/* Synchronises the recorded events; total milliseconds and launches of `name`.
 * Returns 1 if the name was seen, else 0 (outputs zeroed).  Pointers are host. */
int gpr_profile_read(const char *name, double *total_ms, int64_t *count);
/* Work units behind the time of `name` while profiling was on (host): rows for "oz_w",
 * "oz_adig" and "stats_ff", points for "tc_sumsq"; "sov_orthants" is counted on the device:
 * the orthants (P(all < theta), P(all > theta)) that the cell estimator integrated, one or two per
 * estimated cell.  Returns 1 if the name has units, else 0 (*units = 0).  Synchronises the device
 * for "sov_orthants". */
int gpr_profile_units(const char *name, double *units);
/* Number of the library's own kernel launches since the last reset. */
int64_t gpr_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* GPR_LCP_H */
