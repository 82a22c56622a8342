// Launch accounting and optional per-kernel timing with CUDA events.
//
// Every kernel launch of the library goes through ST_LAUNCH_CHECK, which
// counts it.  When profiling is on, tagged launch sites also record an event
// pair on their stream plus the launch's algorithmic bytes and flops, so that
// a caller can compute achieved bandwidth or throughput per kernel over a
// region of its choosing.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "st_common.cuh"

namespace {
std::atomic<unsigned long long> g_launches{0};
thread_local int g_capture_depth = 0;
std::mutex g_mu;
bool g_on = false;
struct Rec {
    const char* tag;
    cudaEvent_t a, b;
    double bytes, flops;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
thread_local Rec g_open{};
thread_local bool g_has_open = false;

cudaEvent_t take_event() {
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

void st_count_launch() {
    if (g_capture_depth == 0) g_launches.fetch_add(1, std::memory_order_relaxed);
}

void st_count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void st_capture_enter() { ++g_capture_depth; }
void st_capture_leave() { --g_capture_depth; }

void st_prof_begin(cudaStream_t s, const char* tag, double bytes, double flops) {
    if (!g_on || g_capture_depth > 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    g_open = Rec{tag, take_event(), take_event(), bytes, flops};
    g_has_open = true;
    cudaEventRecord(g_open.a, s);
}

void st_prof_end(cudaStream_t s) {
    if (!g_has_open) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(g_open.b, s);
    g_recs.push_back(g_open);
    g_has_open = false;
}

extern "C" unsigned long long st_launch_count(void) { return g_launches.load(); }

extern "C" int st_profile_begin(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    g_on = true;
    return ST_OK;
}

extern "C" int st_profile_end(st_kernel_time* out, int max, int* count) {
    std::vector<Rec> recs;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_on = false;
        recs.swap(g_recs);
    }
    std::vector<st_kernel_time> agg;
    int st = ST_OK;
    for (auto& r : recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            st = ST_ECUDA;
            continue;
        }
        st_kernel_time* t = nullptr;
        for (auto& a : agg)
            if (std::strncmp(a.name, r.tag, sizeof(a.name)) == 0) t = &a;
        if (!t) {
            agg.push_back(st_kernel_time{});
            t = &agg.back();
            std::strncpy(t->name, r.tag, sizeof(t->name) - 1);
        }
        t->launches += 1;
        t->ms += ms;
        t->bytes += r.bytes;
        t->flops += r.flops;
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (auto& r : recs) {
            g_pool.push_back(r.a);
            g_pool.push_back(r.b);
        }
    }
    int n = (int)agg.size();
    if (count) *count = n;
    if (out)
        for (int i = 0; i < n && i < max; ++i) out[i] = agg[i];
    return st;
}
