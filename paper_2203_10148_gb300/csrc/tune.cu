// Autotuner: picks the fastest of a few launch variants of a kernel by
// timing each on the problem's own shapes with CUDA events, once per
// (kernel, shape, device) key.  Choices are cached for the process and,
// when the environment variable PIT_AUTOTUNE_CACHE names a file, persisted
// there as "key choice" lines.  PIT_AUTOTUNE=0, or a thread that set
// tl_tune_fallback (serving workers, whose requests rarely share a shape),
// takes the caller's fallback variant for shapes not yet tuned.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <functional>
#include <map>
#include <mutex>
#include <string>

#include "pit_internal.h"

namespace pit {
namespace {

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_file_loaded = false;

const char *cache_path() {
    const char *p = getenv("PIT_AUTOTUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

void load_file_locked() {
    if (g_file_loaded) return;
    g_file_loaded = true;
    const char *path = cache_path();
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char key[512];
    int choice;
    while (fscanf(f, "%511s %d", key, &choice) == 2) g_tune[key] = choice;
    fclose(f);
}

void append_file_locked(const std::string &key, int choice) {
    const char *path = cache_path();
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d\n", key.c_str(), choice);
    fclose(f);
}

}  // namespace

thread_local bool tl_tune_fallback = false;

pit_status autotune(const std::string &key_base, int ncand,
                    const std::function<pit_status(int)> &run, cudaStream_t s, int *choice,
                    int fallback) {
    int dev = 0, sms = 0;
    PIT_CUDA(cudaGetDevice(&dev));
    PIT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const std::string key = key_base + "|sm" + std::to_string(sms);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        load_file_locked();
        auto it = g_tune.find(key);
        if (it != g_tune.end() && it->second >= 0 && it->second < ncand) {
            *choice = it->second;
            return PIT_OK;
        }
    }
    const char *off = getenv("PIT_AUTOTUNE");
    if ((off && strcmp(off, "0") == 0) || tl_tune_fallback) {
        *choice = fallback;
        return PIT_OK;
    }
    cudaEvent_t e0, e1;
    PIT_CUDA(cudaEventCreate(&e0));
    PIT_CUDA(cudaEventCreate(&e1));
    int best = 0;
    float best_ms = 1e30f;
    pit_status st = PIT_OK;
    for (int c = 0; c < ncand && st == PIT_OK; ++c) {
        st = run(c);                      // warm-up
        float acc = 0.f;
        for (int rep = 0; rep < 3 && st == PIT_OK; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess) st = PIT_E_CUDA;
            if (st == PIT_OK) st = run(c);
            if (st == PIT_OK && cudaEventRecord(e1, s) != cudaSuccess) st = PIT_E_CUDA;
            if (st == PIT_OK && cudaEventSynchronize(e1) != cudaSuccess) st = PIT_E_CUDA;
            float ms = 0.f;
            if (st == PIT_OK) cudaEventElapsedTime(&ms, e0, e1);
            acc += ms;
        }
        if (st == PIT_OK && acc < best_ms) {
            best_ms = acc;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PIT_OK) return st;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[key] = best;
        append_file_locked(key, best);
    }
    *choice = best;
    return PIT_OK;
}

}  // namespace pit
