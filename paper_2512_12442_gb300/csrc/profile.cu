// Phase timing and launch counting (tracing support): when enabled, CUDA events are
// recorded on the launching stream around each instrumented kernel, and launches of the
// library's own kernels are counted.
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace {
struct Rec {
    std::string name;
    cudaEvent_t a, b;
};
std::mutex mu;
bool enabled = false;
std::vector<Rec> pending;
std::map<std::string, std::pair<double, int64_t>> totals;
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
        t.first += ms;
        t.second += 1;
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    pending.clear();
}
}  // namespace

void note_launch(int n)
{
    std::lock_guard<std::mutex> g(mu);
    launches += n;
}

ProfScope::ProfScope(const char *name_, cudaStream_t st_) : name(name_), st(st_), active(false)
{
    std::lock_guard<std::mutex> g(mu);
    if (!enabled) return;
    active = true;
    a = get_event();
    b = get_event();
    cudaEventRecord((cudaEvent_t)a, st);
}

ProfScope::~ProfScope()
{
    if (!active) return;
    std::lock_guard<std::mutex> g(mu);
    cudaEventRecord((cudaEvent_t)b, st);
    pending.push_back(Rec{name, (cudaEvent_t)a, (cudaEvent_t)b});
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
    if (total_ms) *total_ms = it->second.first;
    if (count) *count = it->second.second;
    return 1;
}

extern "C" int64_t gpr_launch_count(void)
{
    std::lock_guard<std::mutex> g(mu);
    return launches;
}
