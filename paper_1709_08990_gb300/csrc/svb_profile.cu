// Opt-in per-kernel timing: while profiling is on, every kernel the library
// launches is bracketed by two CUDA events recorded on its own stream, and
// svb_profile_end() reports launches and total milliseconds per kernel.
// Off by default; then each launch site costs one relaxed atomic load.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "svb.h"
#include "svb_internal.h"

namespace {

struct Rec {
    const char *name;
    cudaEvent_t a, b;
};

std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Rec> g_done;
std::vector<cudaEvent_t> g_pool;
thread_local Rec t_open = {nullptr, nullptr, nullptr};

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

void svb::prof_begin(const char *name, cudaStream_t s)
{
    if (!g_on.load(std::memory_order_relaxed))
        return;
    std::lock_guard<std::mutex> lock(g_mu);
    t_open.name = name;
    t_open.a = take_event();
    t_open.b = take_event();
    cudaEventRecord(t_open.a, s);
}

void svb::prof_end(cudaStream_t s)
{
    if (!g_on.load(std::memory_order_relaxed) || !t_open.name)
        return;
    std::lock_guard<std::mutex> lock(g_mu);
    cudaEventRecord(t_open.b, s);
    g_done.push_back(t_open);
    t_open.name = nullptr;
}

extern "C" int svb_profile_begin(void)
{
    std::lock_guard<std::mutex> lock(g_mu);
    g_done.clear();
    g_on.store(true, std::memory_order_relaxed);
    return SVB_OK;
}

extern "C" size_t svb_profile_end(char *buf, size_t len)
{
    std::vector<Rec> recs;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        g_on.store(false, std::memory_order_relaxed);
        recs.swap(g_done);
    }
    std::map<std::string, std::pair<long, double>> agg;
    for (const Rec &r : recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess &&
            cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            auto &x = agg[r.name];
            x.first += 1;
            x.second += ms;
        }
    }
    {
        std::lock_guard<std::mutex> lock(g_mu);
        for (const Rec &r : recs) {
            g_pool.push_back(r.a);
            g_pool.push_back(r.b);
        }
    }
    std::vector<std::pair<std::string, std::pair<long, double>>> rows(agg.begin(), agg.end());
    std::sort(rows.begin(), rows.end(),
              [](const auto &x, const auto &y) { return x.second.second > y.second.second; });
    std::string out;
    char line[256];
    for (const auto &r : rows) {
        std::snprintf(line, sizeof line, "%s %ld %.6f\n", r.first.c_str(), r.second.first,
                      r.second.second);
        out += line;
    }
    if (buf && len) {
        size_t k = std::min(len - 1, out.size());
        std::copy(out.begin(), out.begin() + k, buf);
        buf[k] = '\0';
    }
    return out.size() + 1;
}
