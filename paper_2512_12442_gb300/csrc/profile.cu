// Phase timing and launch counting (tracing support): when enabled, CUDA events are
// recorded on the launching stream around each instrumented kernel, and launches of the
// library's own kernels are counted.  Every instrumented scope and every C-ABI call also opens
// an NVTX range (header-only NVTX v3: without an attached tool each call is a branch).
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace {
struct Rec {
    std::string name;
    cudaEvent_t a, b;
    double units;
};
struct Total {
    double ms = 0.0;
    int64_t count = 0;
    double units = 0.0;
};
std::mutex mu;
bool enabled = false;
std::vector<Rec> pending;
std::map<std::string, Total> totals;
long long launches = 0;
std::vector<cudaEvent_t> pool;

cudaEvent_t get_event()
{
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void drain()
{
    for (auto &r : pending) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto &t = totals[r.name];
        t.ms += ms;
        t.count += 1;
        t.units += r.units;
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    pending.clear();
}
constexpr int kMaxDev = 128;
__device__ unsigned long long g_prof_ctr[PROF_NCTR];
unsigned long long *g_ctr_addr[kMaxDev] = {nullptr};

unsigned long long *ctr_base(bool create)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return nullptr;
    if (!g_ctr_addr[dev] && create) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_prof_ctr) != cudaSuccess) return nullptr;
        g_ctr_addr[dev] = (unsigned long long *)p;
    }
    return g_ctr_addr[dev];
}
}  // namespace

unsigned long long *prof_counter(int which)
{
    std::lock_guard<std::mutex> g(mu);
    if (!enabled || which < 0 || which >= PROF_NCTR) return nullptr;
    unsigned long long *b = ctr_base(true);
    return b ? b + which : nullptr;
}

void note_launch(int n)
{
    std::lock_guard<std::mutex> g(mu);
    launches += n;
}

TraceRange::TraceRange(const char *name) : open(true) { nvtxRangePushA(name); }

void TraceRange::end()
{
    if (open) nvtxRangePop();
    open = false;
}

ProfScope::ProfScope(const char *name_, cudaStream_t st_, double units_)
    : name(name_), st(st_), active(false), units(units_)
{
    nvtxRangePushA(name_);
    std::lock_guard<std::mutex> g(mu);
    if (!enabled) return;
    active = true;
    a = get_event();
    b = get_event();
    cudaEventRecord((cudaEvent_t)a, st);
}

ProfScope::~ProfScope()
{
    nvtxRangePop();
    if (!active) return;
    std::lock_guard<std::mutex> g(mu);
    cudaEventRecord((cudaEvent_t)b, st);
    pending.push_back(Rec{name, (cudaEvent_t)a, (cudaEvent_t)b, units});
    if (pending.size() > 4096) drain();
}

extern "C" void gpr_profile_enable(int on)
{
    std::lock_guard<std::mutex> g(mu);
    enabled = on != 0;
}

extern "C" void gpr_profile_reset(void)
{
    std::lock_guard<std::mutex> g(mu);
    drain();
    totals.clear();
    launches = 0;
    unsigned long long *b = ctr_base(false);
    if (b) {
        cudaDeviceSynchronize();
        cudaMemset(b, 0, sizeof(unsigned long long) * PROF_NCTR);
        cudaDeviceSynchronize();
    }
}

extern "C" int gpr_profile_read(const char *name, double *total_ms, int64_t *count)
{
    std::lock_guard<std::mutex> g(mu);
    drain();
    auto it = totals.find(name ? name : "");
    if (it == totals.end()) {
        if (total_ms) *total_ms = 0.0;
        if (count) *count = 0;
        return 0;
    }
    if (total_ms) *total_ms = it->second.ms;
    if (count) *count = it->second.count;
    return 1;
}

extern "C" int gpr_profile_units(const char *name, double *units)
{
    if (units) *units = 0.0;
    if (!name) return 0;
    if (strcmp(name, "sov_orthants") == 0) {
        std::lock_guard<std::mutex> g(mu);
        unsigned long long *b = ctr_base(false);
        if (!b) return 0;
        unsigned long long h = 0;
        if (cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(&h, b + PROF_CTR_ORTHANTS, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
            return 0;
        if (units) *units = (double)h;
        return 1;
    }
    std::lock_guard<std::mutex> g(mu);
    drain();
    auto it = totals.find(name);
    if (it == totals.end()) return 0;
    if (units) *units = it->second.units;
    return 1;
}

extern "C" int64_t gpr_launch_count(void)
{
    std::lock_guard<std::mutex> g(mu);
    return launches;
}
