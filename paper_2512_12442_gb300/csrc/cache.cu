// Isovalue-independent results kept on the device between calls for one model and grid:
// the separable tables, the per-point (mean, var) table of the FP32-class pass, the
// float-float whitened rows W of every point reconstructed so far and complete stats15.
// The LCP of a new isovalue then reconstructs only points no earlier call touched.
// W rows are cached only while they fit a fixed budget of device memory.
#include <stdlib.h>
#include <string.h>

#include <atomic>

#include "internal.h"

namespace {
constexpr size_t kWCacheBudget = (size_t)24 << 30;       // rows of one model and grid
constexpr size_t kWCacheTotal = (size_t)64 << 30;        // rows of all models together
std::atomic<size_t> g_wcache_total{0};

bool reserve_rows(size_t b)
{
    size_t cur = g_wcache_total.load();
    while (cur + b <= kWCacheTotal)
        if (g_wcache_total.compare_exchange_weak(cur, cur + b)) return true;
    return false;
}

bool same_grid(const gpr_grid &a, const gpr_grid &b) { return memcmp(&a, &b, sizeof a) == 0; }

__global__ void k_need(const uint8_t *flag, const uint8_t *have, int64_t n, uint8_t *need)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) need[i] = (flag[i] && !have[i]) ? 1 : 0;
}

__global__ void k_scatter_mv2(const int64_t *pts, int64_t count, const float *mean, const float *var, float2 *mv,
                              uint8_t *have)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    int64_t p = pts[i];
    mv[p] = make_float2(mean[i], var[i]);
    __threadfence();  // the value before its flag, for readers on other streams
    have[p] = 1;
}

__constant__ int c_off[13][3] = {{1, -1, -1}, {1, -1, 0}, {1, -1, 1}, {1, 0, -1}, {1, 0, 0}, {1, 0, 1}, {1, 1, -1},
                                 {1, 1, 0},   {1, 1, 1},  {0, 1, -1}, {0, 1, 0},  {0, 1, 1}, {0, 0, 1}};

// Points whose stats are needed, plus their forward neighbours, that have no cached W row.
__global__ void k_need_rows(GridDev g, const int64_t *pts, int64_t count, const uint8_t *haveW, uint8_t *need)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    int64_t p = pts[i];
    int64_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
    int ix = (int)(p % nx), iy = (int)((p / nx) % ny), iz = (int)(p / (nx * ny));
    if (!haveW[p]) need[p] = 1;
    for (int e = 0; e < 13; ++e) {
        int a = ix + c_off[e][0], b = iy + c_off[e][1], c = iz + c_off[e][2];
        if (a >= 0 && b >= 0 && c >= 0 && a < nx && b < ny && c < nz) {
            int64_t q = a + nx * (b + ny * (int64_t)c);
            if (!haveW[q]) need[q] = 1;
        }
    }
}

__global__ void k_set_flags(const int64_t *pts, int64_t count, uint8_t *have)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) have[pts[i]] = 1;
}

unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
}  // namespace

void cache_release(gpr_model *M)
{
    GridCache *C = M->cache;
    if (!C) return;
    cudaFree(C->T32); cudaFree(C->T64); cudaFree(C->Tff); cudaFree(C->Tu);
    cudaFree(C->mv); cudaFree(C->have_mv); cudaFree(C->W); cudaFree(C->have_W); cudaFree(C->S15); cudaFree(C->have_S);
    g_wcache_total -= C->wbytes;
    delete C;
    M->cache = nullptr;
}

static gpr_status grid_cache_locked(gpr_model *M, const gpr_grid *grid, const GridDev &g, gpr_precision mv_prec,
                                    GridCache **out, cudaStream_t st);

// Under the model's lock; a new or reset cache is finished on the stream before it is shared
// (fields of one model on one grid can run concurrently in the batched path).
gpr_status grid_cache(gpr_model *M, const gpr_grid *grid, const GridDev &g, gpr_precision mv_prec, GridCache **out,
                      cudaStream_t st)
{
    std::lock_guard<std::mutex> lock(M->init_mu);
    GridCache *before = M->cache;
    gpr_precision pbefore = before ? before->mv_prec : mv_prec;
    GPR_TRY(grid_cache_locked(M, grid, g, mv_prec, out, st));
    if (M->cache != before || pbefore != mv_prec) GPR_CUDA_TRY(cudaStreamSynchronize(st));
    return GPR_OK;
}

static gpr_status grid_cache_locked(gpr_model *M, const gpr_grid *grid, const GridDev &g, gpr_precision mv_prec,
                                    GridCache **out, cudaStream_t st)
{
    if (M->cache && same_grid(M->cache->key, *grid)) {
        GridCache *C = M->cache;
        if (C->mv_prec != mv_prec) {  // the table holds another precision's values: start it again
            GPR_CUDA_TRY(cudaMemsetAsync(C->have_mv, 0, (size_t)C->n, st));
            C->mv_prec = mv_prec;
        }
        *out = C;
        return GPR_OK;
    }
    cudaStreamSynchronize(st);
    cache_release(M);
    GridCache *C = new GridCache();
    C->key = *grid;
    C->n = g.npts();
    C->mv_prec = mv_prec;
    size_t te = table_elems(M, g), n = (size_t)C->n;
    cudaError_t e = cudaSuccess;
#define CA(ptr, nbytes)                                        \
    if (e == cudaSuccess) {                                    \
        e = cudaMalloc((void **)&(ptr), (nbytes));             \
        C->bytes += (nbytes);                                  \
    }
    CA(C->T32, te * 4);
    CA(C->T64, te * 8);
    CA(C->Tff, te * 8);
    CA(C->Tu, te * 8);
    CA(C->mv, n * 8);
    CA(C->have_mv, n);
    size_t wbudget = kWCacheBudget;  // GPR_WCACHE_BUDGET_MB overrides it (tests of the uncached paths)
    if (const char *ev = getenv("GPR_WCACHE_BUDGET_MB")) wbudget = (size_t)atoll(ev) << 20;
    const size_t wb = n * (size_t)M->mp * 8;
    if (e == cudaSuccess && oz_supported(M) && wb <= wbudget && reserve_rows(wb)) {
        C->wbytes = wb;
        CA(C->W, wb);
        CA(C->have_W, n);
        CA(C->S15, n * 15 * 8);  // complete statistics: kept only beside the rows
        CA(C->have_S, n);
        if (e != cudaSuccess) {  // no room for the rows: run without them
            cudaGetLastError();
            cudaFree(C->W); cudaFree(C->have_W); cudaFree(C->S15); cudaFree(C->have_S);
            C->W = nullptr; C->have_W = nullptr; C->S15 = nullptr; C->have_S = nullptr;
            g_wcache_total -= wb;
            C->wbytes = 0;
            e = cudaSuccess;
        }
    }
#undef CA
    if (e != cudaSuccess) {
        M->cache = C;
        cache_release(M);
        return e == cudaErrorMemoryAllocation ? GPR_ERR_OOM : GPR_ERR_CUDA;
    }
    GPR_CUDA_TRY(cudaMemsetAsync(C->have_mv, 0, n, st));
    if (C->have_S) GPR_CUDA_TRY(cudaMemsetAsync(C->have_S, 0, n, st));
    if (C->have_W) GPR_CUDA_TRY(cudaMemsetAsync(C->have_W, 0, n, st));
    GPR_TRY(build_tables(M, g, C->T64, C->T32, st, C->Tff));
    if (oz_supported(M)) GPR_TRY(oz_unit_tables(M, g, C->Tu, st));
    M->cache = C;
    *out = C;
    return GPR_OK;
}

gpr_status cache_fill_mv(gpr_model *M, GridCache *C, const GridDev &g, const uint8_t *flag, int64_t *list, float *tmp_mean,
                         float *tmp_var, float *part, void *cscr, size_t csb, cudaStream_t st)
{
    // `list` doubles as the need-flag buffer (n bytes) before holding the compacted indices
    MvFillScope fill(M, st);
    int64_t n = C->n;
    uint8_t *need = (uint8_t *)tmp_var;  // n floats >= n bytes
    k_need<<<nb(n, 256), 256, 0, st>>>(flag, C->have_mv, n, need);
    note_launch();
    int64_t cnt = 0;
    GPR_TRY(compact_flags(need, n, list, nullptr, &cnt, cscr, csb, st));
    if (cnt == 0) return GPR_OK;
    GPR_TRY(fast_meanvar(M, g, C->mv_prec, C->T32, C->Tff, C->T64, list, 0, cnt, tmp_mean, tmp_var, part, st));
    k_scatter_mv2<<<nb(cnt, 256), 256, 0, st>>>(list, cnt, tmp_mean, tmp_var, C->mv, C->have_mv);
    note_launch();
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}

gpr_status cache_fill_stats(gpr_model *M, GridCache *C, const GridDev &g, const uint8_t *flag, uint8_t *tmpflag,
                            int64_t *list, void *cscr, size_t csb, int64_t *n_new_rows, cudaStream_t st)
{
    int64_t n = C->n;
    if (!C->W) return GPR_ERR_UNSUPPORTED;
    GPR_TRY(oz_prepare(M, st));
    // stats needed and not yet cached
    k_need<<<nb(n, 256), 256, 0, st>>>(flag, C->have_S, n, tmpflag);
    note_launch();
    int64_t ns = 0;
    // bricked order: the 13 forward neighbours' rows of a warp's point are mostly the rows of
    // points that nearby warps read at the same time (L2 reuse); tmpflag holds 2n bytes
    GPR_TRY(compact_flags_bricked(g, tmpflag, tmpflag + n, list, nullptr, &ns, cscr, csb, st));
    if (n_new_rows) *n_new_rows = 0;
    if (ns == 0) return GPR_OK;
    // W rows of those points and of their forward neighbours that the cache lacks
    int64_t *wlist = list + ns;
    GPR_CUDA_TRY(cudaMemsetAsync(tmpflag, 0, (size_t)n, st));
    k_need_rows<<<nb(ns, 256), 256, 0, st>>>(g, list, ns, C->have_W, tmpflag);
    note_launch();
    int64_t nw = 0;
    // the stats list occupies list[0, ns); the row list goes after it (list holds 2n entries)
    GPR_TRY(compact_flags(tmpflag, n, wlist, nullptr, &nw, cscr, csb, st));
    if (nw > 0) {
        GPR_TRY(launch_oz_w(M, g, C->Tu, wlist, 0, nw, C->W, st, true));
        k_set_flags<<<nb(nw, 256), 256, 0, st>>>(wlist, nw, C->have_W);
        note_launch();
    }
    GPR_TRY(launch_stats_ff(M, g, list, ns, nullptr, C->W, C->S15, st, true));
    k_set_flags<<<nb(ns, 256), 256, 0, st>>>(list, ns, C->have_S);
    note_launch();
    if (n_new_rows) *n_new_rows = nw;
    GPR_CUDA_TRY(cudaGetLastError());
    return GPR_OK;
}
