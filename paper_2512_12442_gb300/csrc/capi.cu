// C-ABI entry points: argument checks, workspace carving and the launch sequences.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "internal.h"

extern "C" void gpr_lcp_options_default(gpr_lcp_options *o)
{
    if (!o) return;
    o->alpha = 1e-3;
    o->beta = -1.0;
    o->est = GPR_EST_SOV_QMC;
    o->n_samples = 1600;
    o->seed = 0;
    o->jitter = 1e-10;
    o->skip_eps = 1e-9;
    o->prec = GPR_P_FP32;
    o->max_iters_min = 4;
    o->exact = GPR_EXACT_AUTO;
    o->tree = GPR_TREE_OCTREE;
}

extern "C" const char *gpr_status_string(gpr_status s)
{
    switch (s) {
    case GPR_OK: return "ok";
    case GPR_ERR_ARG: return "invalid argument";
    case GPR_ERR_NOT_PD: return "kernel matrix not positive definite";
    case GPR_ERR_CUDA: return "CUDA error";
    case GPR_ERR_OOM: return "out of device memory";
    case GPR_ERR_TIMEOUT: return "bounded device wait ran out";
    case GPR_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

extern "C" gpr_status gpr_sync(void *stream)
{
    GPR_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int *sw = gpr_status_word();
    if (!sw) return GPR_ERR_CUDA;
    int h = 0;
    GPR_CUDA_TRY(cudaMemcpy(&h, sw, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) GPR_CUDA_TRY(cudaMemset(sw, 0, sizeof(int)));
    return (gpr_status)h;
}

bool est_opts_valid(const gpr_lcp_options *o)
{
    if (!o) return false;
    if (o->est != GPR_EST_SOV_QMC && o->est != GPR_EST_MC && o->est != GPR_EST_INDEP && o->est != GPR_EST_EDGE_MAX &&
        o->est != GPR_EST_SOV_ORDERED)
        return false;
    if (o->n_samples < 1 || o->n_samples > (1 << 24)) return false;
    if (!(o->jitter >= 0.0) || !(o->skip_eps >= 0.0) || !isfinite(o->jitter) || !isfinite(o->skip_eps)) return false;
    return true;
}

bool opts_valid(const gpr_lcp_options *o)
{
    if (!est_opts_valid(o)) return false;
    if (!(o->alpha >= 0.0) || !isfinite(o->alpha)) return false;
    if (isnan(o->beta)) return false;
    if (o->tree != GPR_TREE_OCTREE && o->tree != GPR_TREE_KD) return false;
    if (o->prec < GPR_P_FP64 || o->prec > GPR_P_BF16X3) return false;
    if (o->max_iters_min < 0 || o->max_iters_min > 64) return false;
    if (o->exact != GPR_EXACT_AUTO && o->exact != GPR_EXACT_FP64) return false;
    return true;
}

// FP64 stats of every grid point, in z-slabs whose W rows fit `w_budget` bytes.
static gpr_status dense_stats64(gpr_model *M, const GridDev &g, const double *T64, double *W, size_t w_rows,
                                double *out15, double *mean, double *var, double *cov13, cudaStream_t st)
{
    int64_t nxy = (int64_t)g.n[0] * g.n[1], nz = g.n[2];
    int64_t zs = (int64_t)(w_rows / nxy) - 2;
    if (zs < 1) return GPR_ERR_OOM;
    for (int64_t z0 = 0; z0 < nz; z0 += zs) {
        int64_t z1 = z0 + zs < nz ? z0 + zs : nz;
        int64_t za = z0 > 0 ? z0 - 1 : 0, zb = z1 < nz ? z1 + 1 : nz;
        int64_t base = za * nxy;
        launch_w64(M, g, T64, nullptr, base, (zb - za) * nxy, W, st);
        int64_t o = z0 * nxy;
        launch_stats_from_w64(M, g, nullptr, o, (z1 - z0) * nxy, nullptr, base, W, out15 ? out15 + o * 15 : nullptr,
                              mean ? mean + o : nullptr, var ? var + o : nullptr, cov13 ? cov13 + o * 13 : nullptr, st);
    }
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

static gpr_status dense_stats32(gpr_model *M, const GridDev &g, const float *T32, float *W, size_t w_rows, float *mean,
                                float *var, float *cov13, cudaStream_t st)
{
    int64_t nxy = (int64_t)g.n[0] * g.n[1], nz = g.n[2];
    int64_t zs = (int64_t)(w_rows / nxy) - 2;
    if (zs < 1) return GPR_ERR_OOM;
    for (int64_t z0 = 0; z0 < nz; z0 += zs) {
        int64_t z1 = z0 + zs < nz ? z0 + zs : nz;
        int64_t za = z0 > 0 ? z0 - 1 : 0, zb = z1 < nz ? z1 + 1 : nz;
        int64_t base = za * nxy;
        launch_w32(M, g, T32, nullptr, base, (zb - za) * nxy, W, st);
        int64_t o = z0 * nxy;
        launch_stats_from_w32(M, g, nullptr, o, (z1 - z0) * nxy, nullptr, base, W, mean + o, var + o,
                              cov13 ? cov13 + o * 13 : nullptr, st);
    }
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

static size_t slab_rows(const GridDev &g, int64_t mp, size_t elem, size_t budget)
{
    int64_t nxy = (int64_t)g.n[0] * g.n[1];
    size_t rows = budget / ((size_t)mp * elem);
    size_t need = (size_t)g.npts();
    size_t min_rows = (size_t)nxy * 3;
    if (rows > need + 2 * (size_t)nxy) rows = need + 2 * (size_t)nxy;
    if (rows < min_rows) rows = min_rows;
    return rows;
}

static const size_t kWBudget = (size_t)4 << 30;  // bytes of W rows held at once

extern "C" gpr_status gpr_reconstruct_dense(gpr_model *M, const gpr_grid *grid, gpr_precision prec, void *mean,
                                            void *var, void *cov13, void *stream)
{
    TraceRange trace_("gpr_reconstruct_dense");
    if (!M || !grid_valid(grid) || !mean || !var) return GPR_ERR_ARG;
    if (prec < GPR_P_FP64 || prec > GPR_P_BF16X3) return GPR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    GridDev g = make_grid(grid);
    size_t te = table_elems(M, g);
    if (tc_precision(prec) && cov13) {
        // covariances of this precision: the tensor-core rows themselves (written by the plain
        // kernel) and the FP32 statistics kernel over them, in z-slabs with one halo plane
        GPR_TRY(tc_prepare(M, st));
        size_t rows = slab_rows(g, M->mp, sizeof(float), kWBudget);
        size_t np = tc_partial_elems(prec, M, (int64_t)rows);
        size_t bytes = Carver::round(te * sizeof(float)) + Carver::round(te * sizeof(float2)) +
                       Carver::round(te * sizeof(double)) + Carver::round(np * sizeof(float)) +
                       Carver::round(rows * M->mp * sizeof(float)) + 1024;
        GPR_TRY(ws_reserve(M, 0, bytes, st));
        Carver cv{(char *)ws_ptr(M, 0)};
        float *T32 = cv.take<float>(te);
        float2 *Tff = cv.take<float2>(te);
        double *T64 = cv.take<double>(te);
        float *part = cv.take<float>(np);
        float *W = cv.take<float>(rows * M->mp);
        GPR_TRY(build_tables(M, g, T64, T32, st, Tff));
        int64_t nxy = (int64_t)g.n[0] * g.n[1], nz = g.n[2];
        int64_t zs = (int64_t)(rows / nxy) - 2;
        if (zs < 1) return GPR_ERR_OOM;
        for (int64_t z0 = 0; z0 < nz; z0 += zs) {
            int64_t z1 = z0 + zs < nz ? z0 + zs : nz;
            int64_t za = z0 > 0 ? z0 - 1 : 0, zb = z1 < nz ? z1 + 1 : nz;
            int64_t base = za * nxy, o = z0 * nxy;
            GPR_TRY(launch_tc_var(M, g, prec, T32, nullptr, base, (zb - za) * nxy, part, (float *)var + base, st, W));
            launch_stats_from_w32(M, g, nullptr, o, (z1 - z0) * nxy, nullptr, base, W, (float *)mean + o,
                                  (float *)var + o, (float *)cov13 + o * 13, st);
        }
        launch_mean_compensated(M, g, Tff, T64, nullptr, 0, g.npts(), (float *)mean, st);
        GPR_CUDA_TRY(cudaGetLastError());
        return GPR_OK;
    }
    if (tc_precision(prec)) {
        size_t np = tc_partial_elems(prec, M, g.npts());
        size_t bytes = Carver::round(te * sizeof(float)) + Carver::round(te * sizeof(float2)) +
                       Carver::round(te * sizeof(double)) + Carver::round(np * sizeof(float)) + 1024;
        GPR_TRY(ws_reserve(M, 0, bytes, st));
        Carver cv{(char *)ws_ptr(M, 0)};
        float *T32 = cv.take<float>(te);
        float2 *Tff = cv.take<float2>(te);
        double *T64 = cv.take<double>(te);
        float *part = cv.take<float>(np);
        GPR_TRY(build_tables(M, g, T64, T32, st, Tff));
        return fast_meanvar(M, g, prec, T32, Tff, T64, nullptr, 0, g.npts(), (float *)mean, (float *)var, part, st);
    }
    if (prec == GPR_P_FP64) {
        size_t rows = slab_rows(g, M->mp, sizeof(double), kWBudget);
        size_t bytes = Carver::round(te * sizeof(double)) + Carver::round(rows * M->mp * sizeof(double)) + 1024;
        GPR_TRY(ws_reserve(M, 0, bytes, st));
        Carver cv{(char *)ws_ptr(M, 0)};
        double *T64 = cv.take<double>(te);
        double *W = cv.take<double>(rows * M->mp);
        GPR_TRY(build_tables(M, g, T64, nullptr, st));
        return dense_stats64(M, g, T64, W, rows, nullptr, (double *)mean, (double *)var, (double *)cov13, st);
    }
    float *T32;
    float2 *Tff;
    if (!cov13) {
        size_t bytes = Carver::round(te * sizeof(float)) + Carver::round(te * sizeof(float2)) +
                       Carver::round(te * sizeof(double)) + 1024;
        GPR_TRY(ws_reserve(M, 0, bytes, st));
        Carver cv{(char *)ws_ptr(M, 0)};
        T32 = cv.take<float>(te);
        Tff = cv.take<float2>(te);
        double *T64 = cv.take<double>(te);
        GPR_TRY(build_tables(M, g, T64, T32, st, Tff));
        launch_meanvar32(M, g, T32, nullptr, 0, g.npts(), (float *)mean, (float *)var, st);
        launch_mean_compensated(M, g, Tff, T64, nullptr, 0, g.npts(), (float *)mean, st);
        GPR_CUDA_TRY(cudaGetLastError());
        return GPR_OK;
    }
    size_t rows = slab_rows(g, M->mp, sizeof(float), kWBudget);
    size_t bytes = Carver::round(te * sizeof(float)) + Carver::round(te * sizeof(float2)) +
                   Carver::round(te * sizeof(double)) + Carver::round(rows * M->mp * sizeof(float)) + 1024;
    GPR_TRY(ws_reserve(M, 0, bytes, st));
    Carver cv{(char *)ws_ptr(M, 0)};
    T32 = cv.take<float>(te);
    Tff = cv.take<float2>(te);
    double *T64 = cv.take<double>(te);
    float *W = cv.take<float>(rows * M->mp);
    GPR_TRY(build_tables(M, g, T64, T32, st, Tff));
    GPR_TRY(dense_stats32(M, g, T32, W, rows, (float *)mean, (float *)var, (float *)cov13, st));
    launch_mean_compensated(M, g, Tff, T64, nullptr, 0, g.npts(), (float *)mean, st);
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

__global__ void k_flag_zrange(const uint8_t *flag, int64_t n, int64_t nxy, int64_t za, int64_t zb, uint8_t *out)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t z = p / nxy;
    out[p] = (flag[p] && z >= za && z < zb) ? 1 : 0;
}

void launch_flag_zrange(const uint8_t *flag, int64_t n, int64_t nxy, int64_t za, int64_t zb, uint8_t *out,
                        cudaStream_t st)
{
    k_flag_zrange<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(flag, n, nxy, za, zb, out);
    note_launch();
}

__global__ void k_fill_slot(const int64_t *idx, int64_t count, int64_t npts, int32_t *slot, int *status)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    int64_t p = idx[i];
    if (p < 0 || p >= npts) {
        atomicCAS(status, 0, (int)GPR_ERR_ARG);
        return;
    }
    slot[p] = (int32_t)i;
}

extern "C" gpr_status gpr_stats_points(gpr_model *M, const gpr_grid *grid, const int64_t *point_idx, int64_t count,
                                       double *stats, void *stream)
{
    TraceRange trace_("gpr_stats_points");
    if (!M || !grid_valid(grid) || count < 0 || (count > 0 && (!point_idx || !stats))) return GPR_ERR_ARG;
    if (count == 0) return GPR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    GridDev g = make_grid(grid);
    if (count > g.npts()) return GPR_ERR_ARG;
    size_t te = table_elems(M, g);
    size_t bytes = Carver::round(te * sizeof(double)) + Carver::round((size_t)g.npts() * sizeof(int32_t)) +
                   Carver::round((size_t)count * M->mp * sizeof(double)) + 1024;
    GPR_TRY(ws_reserve(M, 0, bytes, st));
    Carver cv{(char *)ws_ptr(M, 0)};
    double *T64 = cv.take<double>(te);
    int32_t *slot = cv.take<int32_t>((size_t)g.npts());
    double *W = cv.take<double>((size_t)count * M->mp);
    GPR_TRY(build_tables(M, g, T64, nullptr, st));
    GPR_CUDA_TRY(cudaMemsetAsync(slot, 0xff, sizeof(int32_t) * (size_t)g.npts(), st));
    int *status = gpr_status_word();
    if (!status) return GPR_ERR_CUDA;
    k_fill_slot<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(point_idx, count, g.npts(), slot, status);
    note_launch();
    launch_w64(M, g, T64, point_idx, 0, count, W, st);
    launch_stats_from_w64(M, g, point_idx, 0, count, slot, 0, W, stats, nullptr, nullptr, nullptr, st);
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

// Process-level scratch for the model-less entry point.
static void *g_scratch = nullptr;
static size_t g_scratch_bytes = 0;
static gpr_status scratch_reserve(size_t bytes, cudaStream_t st)
{
    if (bytes <= g_scratch_bytes) return GPR_OK;
    if (g_scratch) {
        cudaStreamSynchronize(st);
        cudaFree(g_scratch);
        g_scratch = nullptr;
        g_scratch_bytes = 0;
    }
    GPR_CUDA_TRY(cudaMalloc(&g_scratch, bytes));
    g_scratch_bytes = bytes;
    return GPR_OK;
}

LcpOpts lcp_opts(const gpr_lcp_options *o, double theta)
{
    LcpOpts l;
    l.theta = theta;
    l.tau = o->jitter;
    l.skip_eps = o->skip_eps;
    l.est = o->est;
    l.n_samples = o->n_samples;
    l.seed = o->seed;
    l.exact_mode = o->exact;
    return l;
}

extern "C" gpr_status gpr_cell_lcp_from_stats(const gpr_grid *grid, const double *stats15, double isovalue,
                                              const gpr_lcp_options *opts, const int64_t *cell_idx, int64_t count,
                                              float *lcp, void *stream)
{
    TraceRange trace_("gpr_cell_lcp_from_stats");
    if (!grid_valid(grid) || !stats15 || !lcp || !opts_valid(opts) || !isfinite(isovalue)) return GPR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    GridDev g = make_grid(grid);
    if (!cell_idx) count = g.ncells();
    if (count < 0 || count > g.ncells()) return GPR_ERR_ARG;
    if (count == 0) return GPR_OK;
    size_t bytes = cell_lcp_scratch_bytes(count, opts->est);
    GPR_TRY(scratch_reserve(bytes, st));
    return run_cell_lcp(g, stats15, nullptr, cell_idx, count, lcp_opts(opts, isovalue), lcp, cell_idx != nullptr,
                        g_scratch, g_scratch_bytes, nullptr, st);
}

// Widening of the pre-pass Boole test so that it never drops a cell the FP64 test keeps:
// the FP32 whitened mean/variance errors measured on the configurations are below 1e-5 of
// the field scale; the margins are 100x that.
void prepass_margins(const gpr_model *M, double &mv, double &mm)
{
    double ymax = 0.0;
    for (double v : M->hy) ymax = fmax(ymax, fabs(v));
    mv = 1e-3 * M->kp.sf2;
    mm = 1e-3 * (ymax > 0.0 ? ymax : 1.0);
}

extern "C" gpr_status gpr_lcp_dense(gpr_model *M, const gpr_grid *grid, double isovalue, const gpr_lcp_options *opts,
                                    float *lcp, gpr_adaptive_stats *stats, void *stream)
{
    TraceRange trace_("gpr_lcp_dense");
    if (!M || !grid_valid(grid) || !lcp || !opts_valid(opts) || !isfinite(isovalue)) return GPR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    GridDev g = make_grid(grid);
    int64_t n = g.npts(), nc = g.ncells();
    size_t te = table_elems(M, g);
    LcpOpts lo = lcp_opts(opts, isovalue);
    if (stats) memset(stats, 0, sizeof *stats);
    if (opts->prec == GPR_P_FP64) {
        // every point in FP64, every cell estimated (no pre-pass)
        size_t rows = slab_rows(g, M->mp, sizeof(double), kWBudget);
        size_t bytes = Carver::round(te * sizeof(double)) + Carver::round(rows * M->mp * sizeof(double)) +
                       Carver::round((size_t)n * 15 * sizeof(double)) + cell_lcp_scratch_bytes(nc, lo.est) + 2048;
        GPR_TRY(ws_reserve(M, 0, bytes, st));
        Carver cv{(char *)ws_ptr(M, 0)};
        double *T64 = cv.take<double>(te);
        double *W = cv.take<double>(rows * M->mp);
        double *S15 = cv.take<double>((size_t)n * 15);
        void *scr = cv.take<char>(cell_lcp_scratch_bytes(nc, lo.est));
        GPR_TRY(build_tables(M, g, T64, nullptr, st));
        GPR_TRY(dense_stats64(M, g, T64, W, rows, S15, nullptr, nullptr, nullptr, st));
        int64_t nest = 0;
        GPR_TRY(run_cell_lcp(g, S15, nullptr, nullptr, nc, lo, lcp, false, scr, cell_lcp_scratch_bytes(nc, lo.est),
                             stats ? &nest : nullptr, st));
        if (stats) {
            stats->recon_points = n;
            stats->leaf_cells = nc;
            stats->cells_estimated = nest;
        }
        return GPR_OK;
    }
    // Phase 1: FP32-class mean/variance everywhere (cached per grid), widened Boole test per cell.
    gpr_precision pp = opts->prec;
    GridCache *C = nullptr;
    GPR_TRY(grid_cache(M, grid, g, pp, &C, st));
    size_t b1 = 2 * Carver::round((size_t)n * sizeof(float)) + Carver::round((size_t)nc) + Carver::round((size_t)n) +
                Carver::round((size_t)n * 2 * sizeof(int64_t)) + Carver::round((size_t)n * sizeof(int32_t)) +
                Carver::round((size_t)nc * sizeof(int64_t)) + compact_scratch_bytes(nc > n ? nc : n) +
                Carver::round(tc_partial_elems(GPR_P_BF16X3, M, n) * 4) + 4096;
    GPR_TRY(ws_reserve(M, 0, b1, st));
    Carver cv{(char *)ws_ptr(M, 0)};
    float *mean = cv.take<float>((size_t)n);
    float *var = cv.take<float>((size_t)n);
    uint8_t *keep = cv.take<uint8_t>((size_t)nc);
    uint8_t *pflag = cv.take<uint8_t>((size_t)n);
    int64_t *plist = cv.take<int64_t>((size_t)n * 2);
    int32_t *slot = cv.take<int32_t>((size_t)n);
    int64_t *clist = cv.take<int64_t>((size_t)nc);
    size_t csb = compact_scratch_bytes(nc > n ? nc : n);
    void *cscr = cv.take<char>(csb);
    float *part = cv.take<float>(tc_partial_elems(GPR_P_BF16X3, M, n));
    double *T64 = C->T64;
    GPR_CUDA_TRY(cudaMemsetAsync(pflag, 1, (size_t)n, st));
    GPR_TRY(cache_fill_mv(M, C, g, pflag, plist, mean, var, part, cscr, csb, st));
    double mv, mm;
    prepass_margins(M, mv, mm);
    if (opts->prec == GPR_P_TF32 || opts->prec == GPR_P_BF16) mv = M->kp.sf2;  // single-pass: ~1e-1 var error
    launch_classify_cells_mv(g, C->mv, isovalue, opts->skip_eps, opts->jitter, mv, mm, keep, st);
    return lcp_from_kept_cells(M, g, T64, keep, pflag, plist, slot, clist, cscr, csb, lo, lcp, stats, st);
}

gpr_status lcp_from_kept_cells(gpr_model *M, const GridDev &g, const double *T64, const uint8_t *keep, uint8_t *pflag,
                               int64_t *plist, int32_t *slot, int64_t *clist, void *cscr, size_t csb, const LcpOpts &lo,
                               float *lcp, gpr_adaptive_stats *stats, cudaStream_t st)
{
    std::lock_guard<std::mutex> leaf_lock(M->leaf_mu);
    int64_t n = g.npts(), nc = g.ncells();
    GPR_CUDA_TRY(cudaMemsetAsync(pflag, 0, (size_t)n, st));
    launch_mark_corners(g, keep, pflag, st);
    GPR_CUDA_TRY(cudaGetLastError());
    const bool cached = lo.exact_mode == GPR_EXACT_AUTO && M->cache && M->cache->W && M->cache->n == n;
    int64_t npts = 0, ncell = 0;
    if (!cached) GPR_TRY(compact_flags(pflag, n, plist, slot, &npts, cscr, csb, st));
    GPR_TRY(compact_flags(keep, nc, clist, nullptr, &ncell, cscr, csb, st));
    GPR_CUDA_TRY(cudaMemsetAsync(lcp, 0, sizeof(float) * (size_t)nc, st));
    if (stats) {
        stats->recon_points = npts;
        stats->leaf_cells = ncell;
    }
    if (ncell == 0) return GPR_OK;
    // Cached path: complete stats15 of every corner in the model's grid cache (rows reconstructed
    // only for points no earlier call of this model and grid touched), then the estimator.
    if (cached) {
        GridCache *C = M->cache;
        int64_t nrows = 0;
        GPR_TRY(cache_fill_stats(M, C, g, pflag, (uint8_t *)slot, plist, cscr, csb, &nrows, st));
        GPR_TRY(ws_reserve(M, 1, cell_lcp_scratch_bytes(ncell, lo.est) + 1024, st));
        if (stats) stats->recon_points = nrows;
        int64_t nest = 0;
        GPR_TRY(run_cell_lcp(g, C->S15, nullptr, clist, ncell, lo, lcp, false, ws_ptr(M, 1), ws_size(M, 1),
                             stats ? &nest : nullptr, st));
        if (stats) stats->cells_estimated = nest;
        return GPR_OK;
    }
    // FP64-class W rows and stats15 for the kept cells' corners, then the estimator.  Default:
    // the tensor-core digit-split GEMM with float-float statistics; FP64 CUDA cores on request
    // or for kernels the split does not serve (Matern).
    const bool use_oz = lo.exact_mode == GPR_EXACT_AUTO && oz_supported(M);
    size_t te = table_elems(M, g);
    // bound on the float-float row buffer (GPR_ROW_BUDGET_MB overrides it, for tests of the slab path)
    size_t kRowBudget = (size_t)4 << 30;
    if (const char *e = getenv("GPR_ROW_BUDGET_MB")) kRowBudget = (size_t)atoll(e) << 20;
    if (use_oz && (size_t)npts * M->mp * 8 > kRowBudget) {
        // Planes of rows in a ring of R grid planes (row of point p at p % (R nx ny)): slab
        // [z0, z1) of R - 2 planes reconstructs the rows of its new planes up to z1 and then the
        // statistics of planes z0..z1-1, whose neighbours lie in planes z0-1..z1, all resident.
        const int64_t nxy = (int64_t)g.n[0] * g.n[1], nz = g.n[2];
        const int64_t R = (int64_t)(kRowBudget / ((size_t)nxy * M->mp * 8));
        if (R < 3) return GPR_ERR_OOM;
        const int64_t zs = R - 2, ring = R * nxy;
        size_t b2 = Carver::round((size_t)ring * M->mp * 8) + Carver::round((size_t)n * 15 * 8) +
                    cell_lcp_scratch_bytes(ncell, lo.est) + Carver::round(te * sizeof(float2)) + 2 * Carver::round((size_t)n) +
                    2048;
        GPR_TRY(ws_reserve(M, 1, b2, st));
        Carver cv2{(char *)ws_ptr(M, 1)};
        float2 *W = cv2.take<float2>((size_t)ring * M->mp);
        double *S15 = cv2.take<double>((size_t)n * 15);
        void *scr = cv2.take<char>(cell_lcp_scratch_bytes(ncell, lo.est));
        float2 *Tu = cv2.take<float2>(te);
        uint8_t *zflag = cv2.take<uint8_t>((size_t)n);
        uint8_t *bflag = cv2.take<uint8_t>((size_t)n);
        GPR_TRY(oz_prepare(M, st));
        GPR_TRY(oz_unit_tables(M, g, Tu, st));
        int64_t rows_to = 0;  // rows of planes < rows_to are in the ring
        for (int64_t z0 = 0; z0 < nz; z0 += zs) {
            const int64_t z1 = z0 + zs < nz ? z0 + zs : nz, hi = z1 + 1 < nz ? z1 + 1 : nz;
            int64_t cnt = 0;
            if (hi > rows_to) {
                launch_flag_zrange(pflag, n, nxy, rows_to, hi, zflag, st);
                GPR_TRY(compact_flags(zflag, n, plist, nullptr, &cnt, cscr, csb, st));
                if (cnt > 0) GPR_TRY(launch_oz_w(M, g, Tu, plist, 0, cnt, W, st, true, ring));
                rows_to = hi;
            }
            launch_flag_zrange(pflag, n, nxy, z0, z1, zflag, st);
            GPR_TRY(compact_flags_bricked(g, zflag, bflag, plist, nullptr, &cnt, cscr, csb, st));
            if (cnt > 0) GPR_TRY(launch_stats_ff(M, g, plist, cnt, nullptr, W, S15, st, true, ring));
        }
        int64_t nest = 0;
        GPR_TRY(run_cell_lcp(g, S15, nullptr, clist, ncell, lo, lcp, false, scr, cell_lcp_scratch_bytes(ncell, lo.est),
                             stats ? &nest : nullptr, st));
        if (stats) stats->cells_estimated = nest;
        return GPR_OK;
    }
    size_t b2 = Carver::round((size_t)npts * M->mp * sizeof(double)) + Carver::round((size_t)npts * 15 * sizeof(double)) +
                cell_lcp_scratch_bytes(ncell, lo.est) + Carver::round(te * sizeof(float2)) + 2048;
    GPR_TRY(ws_reserve(M, 1, b2, st));
    Carver cv2{(char *)ws_ptr(M, 1)};
    double *W = cv2.take<double>((size_t)npts * M->mp);
    double *S15 = cv2.take<double>((size_t)npts * 15);
    void *scr = cv2.take<char>(cell_lcp_scratch_bytes(ncell, lo.est));
    float2 *Tu = cv2.take<float2>(te);
    if (use_oz) {
        GPR_TRY(oz_prepare(M, st));
        GPR_TRY(oz_unit_tables(M, g, Tu, st));
        GPR_TRY(launch_oz_w(M, g, Tu, plist, 0, npts, (float2 *)W, st));
        GPR_TRY(launch_stats_ff(M, g, plist, npts, slot, (const float2 *)W, S15, st));
    } else {
        launch_w64(M, g, T64, plist, 0, npts, W, st);
        launch_stats_from_w64(M, g, plist, 0, npts, slot, 0, W, S15, nullptr, nullptr, nullptr, st);
    }
    GPR_CUDA_TRY(cudaGetLastError());
    int64_t nest = 0;
    GPR_TRY(run_cell_lcp(g, S15, slot, clist, ncell, lo, lcp, false, scr, cell_lcp_scratch_bytes(ncell, lo.est),
                         stats ? &nest : nullptr, st));
    if (stats) stats->cells_estimated = nest;
    return GPR_OK;
}

