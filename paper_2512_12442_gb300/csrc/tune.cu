// Launch-shape autotuner (no counterpart in the paper).  A tunable launch offers a few
// alternatives that give the same results (tile widths of the tensor-core pre-pass, persistent
// grid sizes of the estimator); on its first use for a (kernel, size bucket) key the tuner
// queues every alternative on the caller's stream, times each with CUDA events, keeps the
// fastest in a process-wide table and queues it once more, so the call's output is the
// winner's.  Later calls with the same key run the winner only.  The table can be saved to and
// loaded from a text file (GPR_TUNE_FILE), one "kernel bucket choice" line per entry.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "internal.h"

namespace {

struct Table {
    std::mutex mu;
    std::map<std::pair<std::string, int64_t>, int> best;
    std::map<std::string, int> forced;  // test hook: alternative per kernel name
    bool loaded = false;
    bool enabled = true;
};

Table &table()
{
    static Table t;
    return t;
}

void load_locked(Table &T)
{
    if (T.loaded) return;
    T.loaded = true;
    if (const char *e = getenv("GPR_AUTOTUNE")) T.enabled = atoi(e) != 0;
    const char *path = getenv("GPR_TUNE_FILE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char name[128];
    long long bucket;
    int choice;
    while (fscanf(f, "%127s %lld %d", name, &bucket, &choice) == 3) T.best[{name, (int64_t)bucket}] = choice;
    fclose(f);
}

void save_locked(Table &T)
{
    const char *path = getenv("GPR_TUNE_FILE");
    if (!path) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    for (auto &kv : T.best) fprintf(f, "%s %lld %d\n", kv.first.first.c_str(), (long long)kv.first.second, kv.second);
    fclose(f);
}

}  // namespace

int64_t tune_bucket(int64_t v)
{
    int64_t b = 64;
    while (b < v) b <<= 1;
    return b;
}

gpr_status tune_run(const char *name, int64_t bucket, int ncand, const std::function<gpr_status(int)> &run,
                    cudaStream_t st)
{
    Table &T = table();
    int choice = -1;
    {
        std::lock_guard<std::mutex> lock(T.mu);
        load_locked(T);
        auto f = T.forced.find(name);
        if (f != T.forced.end()) choice = f->second < ncand ? f->second : ncand - 1;
        else if (!T.enabled) choice = 0;
        else {
            auto it = T.best.find({name, bucket});
            if (it != T.best.end() && it->second < ncand) choice = it->second;
        }
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (choice < 0 && cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone)
        choice = 0;  // no timing inside a graph capture
    if (choice >= 0) return run(choice);
    // time every alternative once, keep the fastest, and run it again (its output stands)
    std::vector<float> ms(ncand, 0.f);
    cudaEvent_t ev[2];
    GPR_CUDA_TRY(cudaEventCreate(&ev[0]));
    GPR_CUDA_TRY(cudaEventCreate(&ev[1]));
    gpr_status s = GPR_OK;
    for (int c = 0; c < ncand && s == GPR_OK; ++c) {
        cudaEventRecord(ev[0], st);
        s = run(c);
        cudaEventRecord(ev[1], st);
        if (s == GPR_OK && cudaEventSynchronize(ev[1]) == cudaSuccess) cudaEventElapsedTime(&ms[c], ev[0], ev[1]);
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (s != GPR_OK) return s;
    int win = 0;
    for (int c = 1; c < ncand; ++c)
        if (ms[c] < ms[win]) win = c;
    {
        std::lock_guard<std::mutex> lock(T.mu);
        T.best[{name, bucket}] = win;
        save_locked(T);
    }
    return win == ncand - 1 ? GPR_OK : run(win);
}

extern "C" int64_t gpr_autotune_table(char *buf, int64_t len)
{
    Table &T = table();
    std::lock_guard<std::mutex> lock(T.mu);
    load_locked(T);
    std::string out;
    for (auto &kv : T.best)
        out += kv.first.first + " " + std::to_string((long long)kv.first.second) + " " + std::to_string(kv.second) + "\n";
    if (buf && len > 0) {
        int64_t n = (int64_t)out.size() < len - 1 ? (int64_t)out.size() : len - 1;
        memcpy(buf, out.data(), (size_t)n);
        buf[n] = 0;
    }
    return (int64_t)out.size();
}

extern "C" void gpr_autotune_clear(void)
{
    Table &T = table();
    std::lock_guard<std::mutex> lock(T.mu);
    load_locked(T);
    T.best.clear();
}

// Test hook (not in the public header): run alternative `choice` of kernel `name` (-1: tune).
extern "C" void gpr_autotune_force(const char *name, int choice)
{
    Table &T = table();
    std::lock_guard<std::mutex> lock(T.mu);
    if (choice < 0) T.forced.erase(name);
    else T.forced[name] = choice;
}
