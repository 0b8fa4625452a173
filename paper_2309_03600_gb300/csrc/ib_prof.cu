// Launch counting and sampled kernel timing (CUDA events on the launching
// stream).  Used by benchmarks to measure per-kernel device time inside a
// timed region without bracketing every launch.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ib_common.cuh"

namespace {
struct Entry {
    std::string name;
    int64_t launches = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> samples;
};
std::mutex g_mu;
std::vector<Entry> g_entries;
int g_stride = 0;

Entry& entry(const char* name) {
    for (auto& e : g_entries)
        if (e.name == name) return e;
    g_entries.push_back(Entry());
    g_entries.back().name = name;
    return g_entries.back();
}

void clear() {
    for (auto& e : g_entries)
        for (auto& p : e.samples) {
            cudaEventDestroy(p.first);
            cudaEventDestroy(p.second);
        }
    g_entries.clear();
}
}  // namespace

void ib_count_launch(const char* name) {
    std::lock_guard<std::mutex> lk(g_mu);
    entry(name).launches++;
}

ProfToken ib_prof_begin(const char* name, cudaStream_t s) {
    ProfToken t;
    t.name = name;
    t.sampled = false;
    std::lock_guard<std::mutex> lk(g_mu);
    Entry& e = entry(name);
    if (g_stride > 0 && (e.launches % g_stride) == 0) {
        if (cudaEventCreate(&t.e0) == cudaSuccess && cudaEventCreate(&t.e1) == cudaSuccess) {
            cudaEventRecord(t.e0, s);
            t.sampled = true;
        }
    }
    e.launches++;
    return t;
}

void ib_prof_end(const ProfToken& t, cudaStream_t s) {
    if (!t.sampled) return;
    cudaEventRecord(t.e1, s);
    std::lock_guard<std::mutex> lk(g_mu);
    entry(t.name).samples.push_back({t.e0, t.e1});
}

extern "C" ib_status ib_profile_enable(int32_t stride) {
    std::lock_guard<std::mutex> lk(g_mu);
    clear();
    g_stride = stride > 0 ? stride : 0;
    return IB_OK;
}

extern "C" int32_t ib_profile_count(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    return (int32_t)g_entries.size();
}

extern "C" ib_status ib_profile_get(int32_t i, char* name, int32_t name_len, int64_t* launches, int64_t* sampled,
                                    double* sampled_ms) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (i < 0 || i >= (int32_t)g_entries.size()) {
        ib_set_error("profile index out of range");
        return IB_ERR_ARG;
    }
    Entry& e = g_entries[i];
    if (name && name_len > 0) {
        strncpy(name, e.name.c_str(), (size_t)name_len - 1);
        name[name_len - 1] = 0;
    }
    if (launches) *launches = e.launches;
    if (sampled) *sampled = (int64_t)e.samples.size();
    double ms = 0.0;
    for (auto& p : e.samples) {
        float f = 0.f;
        if (cudaEventSynchronize(p.second) != cudaSuccess) continue;
        if (cudaEventElapsedTime(&f, p.first, p.second) == cudaSuccess) ms += f;
    }
    if (sampled_ms) *sampled_ms = ms;
    return IB_OK;
}
