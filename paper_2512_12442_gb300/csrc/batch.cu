// Many adaptive LCP fields in one call (no counterpart in the paper, which computes one field
// per run).  A native scheduler spreads the fields over host worker threads, each with its own
// CUDA stream and a pooled device workspace, so the latency-bound octree levels of small fields
// overlap with the tensor-core and estimator work of large ones.  The cells that need the
// estimator, from every field, are appended to one record buffer and estimated by a single
// persistent launch after all fields' octrees and corner statistics are done.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

struct Pool {
    std::mutex mu;  // held for the whole batched call: one batch at a time per process
    std::vector<Workspace> arenas;  // one per worker thread
    void *recs = nullptr;
    size_t rec_bytes = 0;
    unsigned long long *nrec = nullptr;
    cudaEvent_t done = nullptr;  // the last estimator launch over the buffer
};

Pool &pool()
{
    static Pool p;
    return p;
}

constexpr size_t kRecordBudget = (size_t)8 << 30;  // shared estimator records (192 B each)

struct Job {
    gpr_model *M;
    std::vector<int> items;
    double cost = 0.0;
};

int worker_count(int jobs)
{
    int w = 8;
    if (const char *e = getenv("GPR_BATCH_WORKERS")) {
        int v = atoi(e);
        if (v >= 1 && v <= 64) w = v;
    }
    return jobs < w ? jobs : w;
}

}  // namespace

extern "C" gpr_status gpr_lcp_adaptive_batched(gpr_model *const *models, const gpr_grid *grids,
                                               const double *isovalues, const int32_t *max_depths, int32_t count,
                                               const gpr_lcp_options *opts, float *const *lcps,
                                               gpr_adaptive_stats *stats, void *stream)
{
    TraceRange trace_("gpr_lcp_adaptive_batched");
    if (count < 0 || !opts_valid(opts)) return GPR_ERR_ARG;
    if (count == 0) return GPR_OK;
    if (!models || !grids || !isovalues || !max_depths || !lcps) return GPR_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        const int D = max_depths[i];
        if (!models[i] || !grid_valid(&grids[i]) || !lcps[i] || !isfinite(isovalues[i])) return GPR_ERR_ARG;
        if (D < 0 || D > 20) return GPR_ERR_ARG;
        for (int d = 0; d < 3; ++d)
            if (((int64_t)1 << D) < (int64_t)grids[i].n[d] - 1) return GPR_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    GPR_CUDA_TRY(cudaGetDevice(&dev));

    // Jobs: a model whose fields all use one grid gives one job per field (they may run
    // concurrently: its grid cache and operands are created under the model's lock and its cache
    // fills are idempotent); a model with fields on several grids gives one job that runs them in
    // order (the cache holds one grid).  Largest estimated cost first.
    std::vector<Job> jobs;
    std::unordered_map<gpr_model *, int> first_of, one_grid;
    int64_t total_cells = 0;
    for (int i = 0; i < count; ++i) {
        auto it = first_of.find(models[i]);
        if (it == first_of.end()) {
            first_of[models[i]] = i;
            one_grid[models[i]] = 1;
        } else if (memcmp(&grids[it->second], &grids[i], sizeof(gpr_grid)) != 0) {
            one_grid[models[i]] = 0;
        }
    }
    std::unordered_map<gpr_model *, int> job_of;
    for (int i = 0; i < count; ++i) {
        int jix;
        if (one_grid[models[i]]) {
            jix = (int)jobs.size();
            jobs.push_back(Job{models[i], {}, 0.0});
        } else {
            auto it = job_of.find(models[i]);
            if (it == job_of.end()) {
                job_of[models[i]] = (int)jobs.size();
                jobs.push_back(Job{models[i], {}, 0.0});
                it = job_of.find(models[i]);
            }
            jix = it->second;
        }
        Job &J = jobs[jix];
        J.items.push_back(i);
        const double n0 = grids[i].n[0], n1 = grids[i].n[1], n2 = grids[i].n[2];
        const double mp = (double)J.M->mp;
        J.cost += mp * mp * (n0 * n1 + n1 * n2 + n0 * n2) + 64.0 * n0 * n1 * n2;
        total_cells += (int64_t)(n0 - 1) * (int64_t)(n1 - 1) * (int64_t)(n2 - 1);
    }
    std::stable_sort(jobs.begin(), jobs.end(), [](const Job &a, const Job &b) { return a.cost > b.cost; });

    Pool &P = pool();
    std::lock_guard<std::mutex> lock(P.mu);
    const int W = worker_count((int)jobs.size());
    if ((int)P.arenas.size() < W) P.arenas.resize(W);

    // the shared record buffer (records of fields that do not fit estimate on their own stream);
    // the ordered estimator keeps a second factor per cell, in a parallel array after the first
    const bool two = opts->est == GPR_EST_SOV_ORDERED;
    const size_t rb = record_bytes() * (two ? 2 : 1);
    int64_t cap = total_cells;
    if ((size_t)cap * rb > kRecordBudget) cap = (int64_t)(kRecordBudget / rb);
    if (const char *e = getenv("GPR_BATCH_RECORD_CAP")) {  // tests of the per-field fallback
        int64_t v = atoll(e);
        if (v >= 0 && v < cap) cap = v;
    }
    const size_t want = (size_t)cap * rb;
    // the previous call's estimator (maybe on another stream) still reads the buffer
    if (P.done) GPR_CUDA_TRY(cudaStreamWaitEvent(st, P.done, 0));
    if (P.rec_bytes < want) {
        GPR_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(P.recs);
        P.recs = nullptr;
        P.rec_bytes = 0;
        GPR_CUDA_TRY(cudaMalloc(&P.recs, want));
        P.rec_bytes = want;
    }
    if (!P.nrec) GPR_CUDA_TRY(cudaMalloc(&P.nrec, 2 * sizeof(unsigned long long)));  // count, estimator ticket
    std::atomic<int64_t> reserved{0};
    void *recs2 = two ? (void *)((char *)P.recs + (size_t)cap * record_bytes()) : nullptr;
    RecordSink sink{P.recs, P.nrec, cap, &reserved, recs2};

    GPR_CUDA_TRY(cudaMemsetAsync(P.nrec, 0, sizeof(unsigned long long), st));
    cudaEvent_t fork;
    GPR_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    GPR_CUDA_TRY(cudaEventRecord(fork, st));

    std::vector<gpr_status> status(count, GPR_OK);
    std::vector<cudaStream_t> streams(W, nullptr);
    std::vector<cudaEvent_t> joins(W, nullptr);
    std::atomic<int> ticket{0};
    gpr_status setup = GPR_OK;
    for (int w = 0; w < W && setup == GPR_OK; ++w) {
        if (cudaStreamCreateWithFlags(&streams[w], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&joins[w], cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamWaitEvent(streams[w], fork, 0) != cudaSuccess)
            setup = GPR_ERR_CUDA;
    }
    if (setup == GPR_OK) {
        auto work = [&](int w) {
            cudaSetDevice(dev);
            set_record_sink(&sink);
            set_thread_workspace(&P.arenas[w]);
            for (;;) {
                const int j = ticket.fetch_add(1);
                if (j >= (int)jobs.size()) break;
                Job &J = jobs[j];
                for (int i : J.items) {
                    gpr_adaptive_stats *si = stats ? &stats[i] : nullptr;
                    status[i] = octree_lcp(J.M, &grids[i], isovalues[i], max_depths[i], opts, lcps[i], si,
                                           streams[w], nullptr);
                }
            }
            set_record_sink(nullptr);
            set_thread_workspace(nullptr);
            cudaEventRecord(joins[w], streams[w]);
        };
        std::vector<std::thread> threads;
        for (int w = 1; w < W; ++w) threads.emplace_back(work, w);
        work(0);
        for (auto &t : threads) t.join();
        for (int w = 0; w < W; ++w)
            if (cudaStreamWaitEvent(st, joins[w], 0) != cudaSuccess) setup = GPR_ERR_CUDA;
    }
    for (int w = 0; w < W; ++w) {
        if (joins[w]) cudaEventDestroy(joins[w]);
        if (streams[w]) cudaStreamDestroy(streams[w]);
    }
    cudaEventDestroy(fork);
    GPR_TRY(setup);
    // one persistent estimator launch over every field's records
    int64_t nres = reserved.load();
    if (nres > cap) nres = cap;
    if (nres > 0) {
        TraceRange est("batched_estimator");
        launch_estimator(P.recs, recs2, P.nrec, nres, lcp_opts(opts, 0.0), st);
    }
    GPR_CUDA_TRY(cudaGetLastError());
    if (!P.done) GPR_CUDA_TRY(cudaEventCreateWithFlags(&P.done, cudaEventDisableTiming));
    GPR_CUDA_TRY(cudaEventRecord(P.done, st));
    for (int i = 0; i < count; ++i)
        if (status[i] != GPR_OK) return status[i];
    return GPR_OK;
}

extern "C" gpr_status gpr_batch_release(void)
{
    Pool &P = pool();
    std::lock_guard<std::mutex> lock(P.mu);
    cudaDeviceSynchronize();
    for (Workspace &A : P.arenas)
        for (int i = 0; i < 2; ++i) {
            cudaFree(A.ptr[i]);
            A.ptr[i] = nullptr;
            A.bytes[i] = 0;
        }
    cudaFree(P.recs);
    cudaFree(P.nrec);
    P.recs = nullptr;
    P.nrec = nullptr;
    P.rec_bytes = 0;
    adig_free_idle();
    return GPR_OK;
}
