// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <functional>
#include <mutex>
#include <vector>

#include "../../include/gpr_lcp.h"

#define GPR_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) {                             \
            gpr_internal_note_cuda_error(_e, #expr, __LINE__); \
            return (_e == cudaErrorMemoryAllocation) ? GPR_ERR_OOM : GPR_ERR_CUDA; \
        }                                                    \
    } while (0)

#define GPR_TRY(expr)                   \
    do {                                \
        gpr_status _s = (expr);         \
        if (_s != GPR_OK) return _s;    \
    } while (0)

void gpr_internal_note_cuda_error(cudaError_t e, const char *what, int line);

// Process-wide device status word (one int in device memory): 0 = OK, otherwise the
// first gpr_status a kernel recorded.  Read and cleared by gpr_sync().
int *gpr_status_word();

// Forward neighbour offsets of the stats15 layout (see gpr_lcp.h).
static constexpr int kOff13[13][3] = {
    {1, -1, -1}, {1, -1, 0}, {1, -1, 1}, {1, 0, -1}, {1, 0, 0}, {1, 0, 1}, {1, 1, -1},
    {1, 1, 0},   {1, 1, 1},  {0, 1, -1}, {0, 1, 0},  {0, 1, 1}, {0, 0, 1}};

// Grid description on the device side.
struct GridDev {
    double lo[3], h[3];
    int32_t n[3];
    int64_t npts() const { return (int64_t)n[0] * n[1] * n[2]; }
    int64_t ncells() const { return (int64_t)(n[0] - 1) * (n[1] - 1) * (n[2] - 1); }
};

GridDev make_grid(const gpr_grid *g);
bool grid_valid(const gpr_grid *g);

// Kernel parameters passed by value to device code.
struct KernParams {
    int kind;          // gpr_kernel
    double ell[3];
    double sf2;
};

// Tensor-core B operands (rows of L^-1, K-major, mpt x mpt with mpt = mp rounded up to 256).
struct TcOperands {
    int64_t mpt = 0;
    float *thi = nullptr, *tlo = nullptr;        // TF32 hi/lo (FP32 storage)
    void *b0 = nullptr, *b1 = nullptr, *b2 = nullptr;  // BF16 slices
};

struct OzOperands;  // tensor-core FP64-class operands (ozaki.cu)

// Two independent device workspaces (grow, never shrink): slot 0 for a call's first phase,
// slot 1 for buffers sized after a device->host count read-back.
struct Workspace {
    void *ptr[2] = {nullptr, nullptr};
    size_t bytes[2] = {0, 0};
};
struct GridCache;   // isovalue-independent per-grid results (cache.cu)

struct gpr_model {
    int64_t m = 0;
    int64_t mp = 0;  // m rounded up to a multiple of 64 (GEMM column padding)
    KernParams kp;
    double sn2 = 0.0;
    int device = 0;
    // device buffers (FP64 unless noted)
    double *X = nullptr;       // m x 3
    double *y = nullptr;       // m
    double *L = nullptr;       // m x m lower Cholesky factor
    double *Linv = nullptr;    // m x m lower inverse
    double *vy = nullptr;      // mp: L^-1 y (zero padded)
    double *alpha = nullptr;   // m: Kt^-1 y
    double *mu_obs = nullptr;  // m
    double *var_obs = nullptr; // m
    double *BT64 = nullptr;    // mp x mp: BT[i][j] = Linv[j][i] (upper triangular), zero padded
    float *BT32 = nullptr;     // mp x mp FP32 copy
    float *vy32 = nullptr;     // mp
    float2 *alpha_ff = nullptr; // mp: alpha as float-float (hi, lo)
    float *X32 = nullptr;      // m x 3 FP32 observation sites (float-float: hi, then lo at + 3 mp), zero-padded to mp x 3
    float *alpha32 = nullptr;  // mp FP32 alpha
    TcOperands *tc = nullptr;  // built on first tensor-core use
    OzOperands *oz = nullptr;  // built on first FP64-class tensor-core use
    GridCache *cache = nullptr;
    // host copies used by the octree p-test
    std::vector<double> hX, hy;
    // the model's own workspaces (see Workspace); batch workers use theirs instead
    Workspace own_ws;
    // serialises the lazy creation of tc / oz operands when fields of one model run concurrently
    std::mutex init_mu;
    // serialises the leaf phases of concurrent fields of one model, so that each finds the rows
    // and statistics the previous one cached instead of recomputing them alongside it
    std::mutex leaf_mu;
    // orders the fills of the per-point (mean, var) table by concurrent fields of one model: a
    // fill waits (on the device) for the previous one, so no point is computed twice
    std::mutex mv_mu;
    cudaEvent_t mv_ev = nullptr;
    // SGPR model (gpr_model_create_sgpr): Linv holds G, the lower-triangular factor of
    // Q = K_MM^-1 - K_MM^-1 A_M K_MM^-1 = G^T G, so every whitened kernel computes Eq. 1 unchanged;
    // vy = G^-T alpha, alpha = K_MM^-1 mu_M, y = mu_M, L = chol(K_MM + jitter I), sn2 = 0
    bool sgpr = false;
    double kmm_jitter = 0.0;  // SGPR: jitter on the diagonal of K_MM
    double *A_M = nullptr;    // SGPR: m x m A_M (FP64), read by the local model of the bound
};

// Scope of one fill of the per-point (mean, var) table: holds the model's mv lock, orders the
// caller's stream after the previous fill, and marks the end of this fill on exit.
struct MvFillScope {
    gpr_model *M;
    cudaStream_t st;
    std::lock_guard<std::mutex> lock;
    MvFillScope(gpr_model *m, cudaStream_t s) : M(m), st(s), lock(m->mv_mu)
    {
        if (M->mv_ev) cudaStreamWaitEvent(st, M->mv_ev, 0);
        else cudaEventCreateWithFlags(&M->mv_ev, cudaEventDisableTiming);
    }
    ~MvFillScope()
    {
        if (M->mv_ev) cudaEventRecord(M->mv_ev, st);
    }
};

// Makes workspace slot `which` at least `bytes` long (cudaMalloc only when it grows).  The
// workspace is the model's own, or the calling thread's if one is set (batch workers).
gpr_status ws_reserve(gpr_model *M, int which, size_t bytes, cudaStream_t st);
void *ws_ptr(gpr_model *M, int which);
size_t ws_size(gpr_model *M, int which);
void set_thread_workspace(Workspace *w);  // nullptr: back to the models' own

// Bump allocator over a workspace block (256-byte aligned pieces).
struct Carver {
    char *base;
    size_t off = 0;
    template <typename T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return p;
    }
    static size_t round(size_t b) { return (b + 255) & ~size_t(255); }
};

// ---- plain FP64 products (adjoint.cu): C = A B, C = A^T B (row-major, one launch each)
void gemm64_nn(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
               int64_t ldc, cudaStream_t st);
void gemm64_tn(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
               int64_t ldc, cudaStream_t st);

// ---- stats (stats.cu)
// Per-axis SE factor tables E_d[g][j] (or squared scaled distance for Matern), FP64 and FP32.
gpr_status build_tables(const gpr_model *M, const GridDev &g, double *T64, float *T32, cudaStream_t st,
                        float2 *Tff = nullptr);
size_t table_elems(const gpr_model *M, const GridDev &g);  // per precision, all 3 axes

// Point lists: `pts` (device int64 grid indices) or, when pts == nullptr, the consecutive
// grid points pt_base, pt_base+1, ...  Row r of W belongs to list position r.
// Slot maps: grid index -> row of W (`slot`, int32, -1 = absent) or, when slot == nullptr,
// row = grid index - slot_base.
void launch_w64(const gpr_model *M, const GridDev &g, const double *T64, const int64_t *pts, int64_t pt_base,
                int64_t count, double *W, cudaStream_t st);
void launch_w32(const gpr_model *M, const GridDev &g, const float *T32, const int64_t *pts, int64_t pt_base,
                int64_t count, float *W, cudaStream_t st);
// stats from W rows: either out15 (count x 15) or separate mean/var/cov13 (cov13 nullable).
void launch_stats_from_w64(const gpr_model *M, const GridDev &g, const int64_t *pts, int64_t pt_base, int64_t count,
                           const int32_t *slot, int64_t slot_base, const double *W, double *out15, double *mean,
                           double *var, double *cov13, cudaStream_t st);
void launch_stats_from_w32(const gpr_model *M, const GridDev &g, const int64_t *pts, int64_t pt_base, int64_t count,
                           const int32_t *slot, int64_t slot_base, const float *W, float *mean, float *var,
                           float *cov13, cudaStream_t st);
// Posterior mean k . alpha in float-float (SE) or FP64 (Matern); Tff / T64 tables as built.
void launch_mean_compensated(const gpr_model *M, const GridDev &g, const float2 *Tff, const double *T64,
                             const int64_t *pts, int64_t pt_base, int64_t count, float *mean, cudaStream_t st);
// Fused FP32 mean/variance (W never stored).
void launch_meanvar32(const gpr_model *M, const GridDev &g, const float *T32, const int64_t *pts, int64_t pt_base,
                      int64_t count, float *mean, float *var, cudaStream_t st);

// ---- launch-shape autotuner (tune.cu)
// Smallest power of two >= v (at least 64): the size bucket of a tuned launch.
int64_t tune_bucket(int64_t v);
// Runs alternative `choice` of a launch with equal results; on the first use of (name, bucket)
// all `ncand` alternatives are timed on `st` and the fastest is kept (and queued last).
gpr_status tune_run(const char *name, int64_t bucket, int ncand, const std::function<gpr_status(int)> &run,
                    cudaStream_t st);

// ---- tensor cores (tc.cu)
bool tc_precision(gpr_precision p);
gpr_status tc_prepare(gpr_model *M, cudaStream_t st);
void tc_release(gpr_model *M);
size_t tc_partial_elems(gpr_precision p, const gpr_model *M, int64_t count);
// TF32x3 whitened rows at arbitrary points (count x 3 FP64 coordinates), reduced to partial sums
// of |w|^2 and, with grad, of w . L^-1 d_k k per coordinate: partial[(point * T + type) * nN + g],
// T = 4 with grad (else 1), nN = (mp rounded up to 256) / 64 groups of 64 columns; after the
// count * 4 * nN partial sums, 8 floats per point: mu and (grad) grad mu as float-float pairs.
size_t tc_eval_partial_elems(const gpr_model *M, int64_t count);
gpr_status launch_tc_eval(gpr_model *M, const double *xyz, int64_t count, bool grad, float *partial,
                          size_t partial_elems, cudaStream_t st);
// W (nullable, count x mp): also write the whitened rows of this precision (plain kernel).
gpr_status launch_tc_var(const gpr_model *M, const GridDev &g, gpr_precision prec, const float *T32,
                         const int64_t *pts, int64_t pt_base, int64_t count, float *partial, float *var, cudaStream_t st,
                         float *W = nullptr);
// FP32-class mean/variance of a point list in any non-FP64 precision (SIMT FP32 or tensor cores);
// the mean is always the compensated k . alpha.  `partial` needs tc_partial_elems floats (TC only).
gpr_status fast_meanvar(gpr_model *M, const GridDev &g, gpr_precision prec, const float *T32, const float2 *Tff,
                        const double *T64, const int64_t *pts, int64_t pt_base, int64_t count, float *mean, float *var,
                        float *partial, cudaStream_t st);

// ---- FP64-class whitened rows on the tensor cores (ozaki.cu)
bool oz_supported(const gpr_model *M);
gpr_status oz_prepare(gpr_model *M, cudaStream_t st);
void oz_release(gpr_model *M);
gpr_status oz_unit_tables(const gpr_model *M, const GridDev &g, float2 *Tu, cudaStream_t st);
// out_by_point: row (or stats) of listed point p goes to position p of a full-grid array (rows
// at p % row_mod, a ring of grid planes, when row_mod > 0); without a slot map the statistics
// read the row of point q at q % row_mod.
gpr_status launch_oz_w(const gpr_model *M, const GridDev &g, const float2 *Tu, const int64_t *pts, int64_t pt_base,
                       int64_t count, float2 *W, cudaStream_t st, bool out_by_point = false,
                       int64_t row_mod = 0);
gpr_status launch_stats_ff(const gpr_model *M, const GridDev &g, const int64_t *pts, int64_t count, const int32_t *slot,
                           const float2 *W, double *out15, cudaStream_t st, bool out_by_point = false,
                           int64_t row_mod = 0);
// Frees the digit-split GEMMs' pooled digit buffers that no call is using.
void adig_free_idle();
// FP64-class products of FP64 matrices by the same digit split (42-bit fixed-point digits per
// row / column exponent): C = X L^-1 (X rows x m, ld ldx; C ld ldc), and C = A^T B for
// A, B: K x nc (ld) as nsplit partials of (nc rounded up to 64)^2 whose sum is C.
gpr_status oz_mul_linv(gpr_model *M, const double *X, int64_t rows, int64_t ldx, double *C, int64_t ldc,
                       cudaStream_t st);
gpr_status oz_mul_tn(const double *A, const double *B, int64_t K, int64_t nc, int64_t ld, double *part, int nsplit,
                     cudaStream_t st, int64_t kchunk = 0);

// ---- per-model, per-grid cache of isovalue-independent results (cache.cu)
struct GridCache {
    gpr_grid key;
    int64_t n = 0;
    size_t bytes = 0;
    size_t wbytes = 0;           // bytes of W counted against the budget of all models
    float *T32 = nullptr;
    double *T64 = nullptr;
    float2 *Tff = nullptr, *Tu = nullptr;
    float2 *mv = nullptr;        // per-point (mean, var) of the FP32-class pass
    uint8_t *have_mv = nullptr;
    gpr_precision mv_prec = GPR_P_FP32;
    float2 *W = nullptr;         // float-float whitened rows, full grid (nullptr when over budget)
    uint8_t *have_W = nullptr;
    double *S15 = nullptr;       // complete stats15 (all forward neighbours), full grid
    uint8_t *have_S = nullptr;
};
// Returns the model's cache for `g` (allocating / resetting it on a new grid or precision).
gpr_status grid_cache(gpr_model *M, const gpr_grid *grid, const GridDev &g, gpr_precision mv_prec, GridCache **out,
                      cudaStream_t st);
void cache_release(gpr_model *M);
struct OctTrace;
gpr_status octree_lcp(gpr_model *M, const gpr_grid *grid, double theta, int D, const gpr_lcp_options *opts,
                      float *lcp, gpr_adaptive_stats *stats, cudaStream_t st, OctTrace *trace);
// Algorithm 1's leaf cells S for one isovalue (leaf: device, one byte per cell), without the
// leaf reconstruction.
gpr_status octree_leaf_mask(gpr_model *M, const gpr_grid *grid, double theta, int D, const gpr_lcp_options *opts,
                            uint8_t *leaf, cudaStream_t st);
// Fills the per-point table for flagged points that lack it (flags: uint8 per point).
gpr_status cache_fill_mv(gpr_model *M, GridCache *C, const GridDev &g, const uint8_t *flag, int64_t *list, float *tmp_mean,
                         float *tmp_var, float *part, void *cscr, size_t csb, cudaStream_t st);
// Complete FP64-class stats15 in C->S15 for every flagged point (digit-split W rows cached).
// tmpflag: 2n bytes of scratch; list: 2n int64.
gpr_status cache_fill_stats(gpr_model *M, GridCache *C, const GridDev &g, const uint8_t *flag, uint8_t *tmpflag,
                            int64_t *list, void *cscr, size_t csb, int64_t *n_new_rows, cudaStream_t st);

// ---- LCP (lcp.cu)
struct LcpOpts {
    double theta, tau, skip_eps;
    int est, n_samples;
    uint64_t seed;
    int exact_mode;  // gpr_lcp_options.exact
};
// For cells in `cells` (nullptr = all), build Sigma_8 from stats (indexed via slot map, nullptr = identity),
// write 0/1 for skipped/deterministic cells into lcp[cell-or-position], and queue the rest.
// out_by_position: lcp indexed by position in `cells` (true) or by linear cell index (false).
// Records of several fields collected for one estimator launch (the batched entry point): a
// worker thread sets its sink; run_cell_lcp then appends its records there while `reserved`
// (host counter of records promised) stays within `capacity`, else estimates on its own.
struct RecordSink {
    void *recs;
    unsigned long long *nrec;  // device counter of appended records (and the estimator's ticket after it)
    int64_t capacity;
    std::atomic<int64_t> *reserved;
    void *recs2;  // GPR_EST_SOV_ORDERED: the all-above orthants' records, parallel to recs (else null)
};
void set_record_sink(RecordSink *sink);  // for the calling thread; nullptr to clear
size_t record_bytes();
// nrec[0]: the device record count; nrec[1]: scratch for the estimator's work ticket.  recs2:
// the all-above orthants' records of GPR_EST_SOV_ORDERED, index for index with recs (else null).
void launch_estimator(const void *recs, const void *recs2, unsigned long long *nrec, int64_t max_records,
                      const LcpOpts &o, cudaStream_t st);
gpr_status run_cell_lcp(const GridDev &g, const double *stats, const int32_t *slot, const int64_t *cells,
                        int64_t count, const LcpOpts &o, float *lcp, bool out_by_position, void *scratch,
                        size_t scratch_bytes, int64_t *n_estimated, cudaStream_t st);
size_t cell_lcp_scratch_bytes(int64_t count, int est);  // est: gpr_estimator
size_t cell_rec_bytes();
gpr_status run_cell_lcp_on_scratch(const GridDev &g, const double *stats, const int64_t *cells, int64_t count,
                                   const LcpOpts &o, float *lcp, bool by_pos, void *scratch, int64_t max_records,
                                   int *status, cudaStream_t st);

// Pre-classification: keep[cell] = 1 unless the widened Boole bound is below skip_eps.
void launch_classify_cells(const GridDev &g, const float *mean, const float *var, double theta, double skip_eps,
                           double tau, double margin_var, double margin_mu, uint8_t *keep, cudaStream_t st);

void launch_classify_cells_mv(const GridDev &g, const float2 *mvt, double theta, double skip_eps, double tau,
                              double margin_var, double margin_mu, uint8_t *keep, cudaStream_t st);

// Compaction helpers
// Marks corners of kept cells in point_flag (uint8 per grid point).
void launch_mark_corners(const GridDev &g, const uint8_t *keep_cell, uint8_t *point_flag, cudaStream_t st);
// Stream compaction of flagged indices: out_idx gets indices i with flag[i] != 0 in increasing order,
// *count_dev the number; slot (optional) gets the position of each flagged index (-1 otherwise).
gpr_status compact_flags(const uint8_t *flag, int64_t n, int64_t *out_idx, int32_t *slot, int64_t *count_host,
                         void *scratch, size_t scratch_bytes, cudaStream_t st);
// As compact_flags over the n grid points, the list in bricked order (8^3 bricks) so that
// neighbouring points are processed together; bflag: n bytes of scratch; slot (nullable) maps
// point -> position (-1 elsewhere).
gpr_status compact_flags_bricked(const GridDev &g, const uint8_t *flag, uint8_t *bflag, int64_t *out_idx,
                                 int32_t *slot, int64_t *count_host, void *scratch, size_t scratch_bytes,
                                 cudaStream_t st);
size_t compact_scratch_bytes(int64_t n);

int num_sms();

// ---- shared by the LCP entry points (capi.cu)
void launch_flag_zrange(const uint8_t *flag, int64_t n, int64_t nxy, int64_t za, int64_t zb, uint8_t *out,
                        cudaStream_t st);
bool opts_valid(const gpr_lcp_options *o);
bool est_opts_valid(const gpr_lcp_options *o);  // the fields the cell estimator reads
LcpOpts lcp_opts(const gpr_lcp_options *o, double theta);
void prepass_margins(const gpr_model *M, double &mv, double &mm);
// keep[cell] != 0 cells: FP64 stats of their corners, estimator, field (zeroed elsewhere).
gpr_status lcp_from_kept_cells(gpr_model *M, const GridDev &g, const double *T64, const uint8_t *keep, uint8_t *pflag,
                               int64_t *plist, int32_t *slot, int64_t *clist, void *cscr, size_t csb, const LcpOpts &lo,
                               float *lcp, gpr_adaptive_stats *stats, cudaStream_t st);

// ---- tracing (profile.cu)
void note_launch(int n = 1);
// RAII host range on the NVTX timeline (a no-op unless a tool such as ncu or nsys is attached):
// one per C-ABI call and per phase, so a capture can be filtered by phase.  end() closes it early.
struct TraceRange {
    bool open;
    explicit TraceRange(const char *name);
    ~TraceRange() { end(); }
    void end();
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
// RAII scope: records CUDA events around the enclosed launches when profiling is on, and adds
// `units` (rows, points: the work the launches process) to the scope's total.  It also opens an
// NVTX range of the same name.
struct ProfScope {
    const char *name;
    cudaStream_t st;
    bool active;
    double units;
    void *a = nullptr, *b = nullptr;
    ProfScope(const char *name, cudaStream_t st, double units = 0.0);
    ~ProfScope();
};
// Device-side work counters of the tracer (a module global per device, no allocation): nullptr
// unless profiling is on.  Counter 0: orthants queued for the estimator (1 or 2 per cell record).
enum { PROF_CTR_ORTHANTS = 0, PROF_NCTR = 4 };
unsigned long long *prof_counter(int which);
