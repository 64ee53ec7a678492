// Cell-LCP estimator entry point that allocates no device memory.
//
// Who needs it: callers that may not call cudaMalloc/cudaFree at the time they run --
// a plug-in living inside a host application or framework that has reserved the
// device memory for its own pool allocator (a cudaMalloc of ours would fail or
// fragment that pool), and latency-critical loops, where cudaFree synchronises the
// whole device.  The other entry points grow a workspace with cudaMalloc on first use.
//
// The estimator's scratch (record counter, per-cell records) lives in one file-scope
// __device__ array below.  Every GPU that loads the library holds it until
// the process exits.  All calls share it and it keeps the last call's contents, so
// calls that overlap on the GPU (different streams, or different host threads) race
// on it; callers must order them (one stream, or events).
#include <mutex>

#include "internal.h"

namespace {

constexpr int64_t kMaxCells = GPR_NOALLOC_MAX_CELLS;
constexpr size_t kRecBytes = 192;  // sizeof(CellRec) in lcp.cu, checked at set-up
constexpr size_t kScratchBytes = 256 /* counter */ + kRecBytes * (size_t)kMaxCells;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device addresses of g_noalloc_scratch, resolved once per device with that device current.
// In host code the symbol name is only a host-side stand-in and must never be passed to a kernel.
std::mutex g_mu;
void *g_addr[128] = {nullptr};

gpr_status scratch_address(void **out)
{
    int dev = 0;
    GPR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return GPR_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        if (cell_rec_bytes() != kRecBytes) return GPR_ERR_UNSUPPORTED;
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            gpr_internal_note_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __LINE__);
            return GPR_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return GPR_OK;
}

}  // namespace

extern "C" gpr_status gpr_cell_lcp_from_stats_noalloc(const gpr_grid *grid, const double *stats15, double isovalue,
                                                      const gpr_lcp_options *opts, const int64_t *cell_idx,
                                                      int64_t count, float *lcp, void *stream)
{
    if (!grid_valid(grid) || !stats15 || !lcp || !est_opts_valid(opts) || !isfinite(isovalue)) return GPR_ERR_ARG;
    GridDev g = make_grid(grid);
    if (!cell_idx) count = g.ncells();
    if (count < 0 || count > g.ncells()) return GPR_ERR_ARG;
    if (count > kMaxCells) return GPR_ERR_ARG;  // beyond the static scratch: split the call
    if (count == 0) return GPR_OK;
    void *base = nullptr;
    GPR_TRY(scratch_address(&base));
    // Listed cells off the grid are reported through the library's status word (gpr_sync), as
    // the allocating entry point reports them; the word is a module global, not an allocation.
    int *status = gpr_status_word();
    if (!status) return GPR_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    LcpOpts o;
    o.theta = isovalue;
    o.tau = opts->jitter;
    o.skip_eps = opts->skip_eps;
    o.est = opts->est;
    o.n_samples = opts->n_samples;
    o.seed = opts->seed;
    return run_cell_lcp_on_scratch(g, stats15, cell_idx, count, o, lcp, cell_idx != nullptr, base, kMaxCells, status,
                                   st);
}
