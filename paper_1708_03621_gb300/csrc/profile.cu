// Tracing: a launch counter for every kernel the library starts, and optional
// per-kernel timing with CUDA events recorded on the launching stream around
// each launch.  Events come from a reusable pool; jdft_profile_read waits for
// them, reports count and total milliseconds per kernel name, and recycles
// the pool.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "profile.cuh"

namespace jdft {

static std::atomic<long long> g_launches{0};
static std::atomic<bool> g_prof_on{false};
static std::mutex g_mu;
struct Rec { const char* name; int ev; };
static std::vector<cudaEvent_t> g_pool;
static size_t g_used = 0;
static std::vector<Rec> g_recs;

static int take_events() {
    // two consecutive pool slots; grows the pool on demand
    if (g_used + 2 > g_pool.size()) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            g_pool.push_back(e);
        }
    }
    int idx = (int)g_used;
    g_used += 2;
    return idx;
}

Trace::Trace(const char* name, cudaStream_t st) : st_(st), slot_(-1) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    slot_ = take_events();
    if (slot_ < 0) return;
    g_recs.push_back({name, slot_});
    cudaEventRecord(g_pool[slot_], st_);
}

Trace::~Trace() {
    if (slot_ < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(g_pool[slot_ + 1], st_);
}

}  // namespace jdft

using namespace jdft;

extern "C" {

jdft_status jdft_profile_enable(int on) {
    clear_error();
    g_prof_on.store(on != 0);
    return JDFT_OK;
}

long long jdft_launch_count(void) { return g_launches.load(); }

jdft_status jdft_profile_read(char* buf, int buflen) {
    clear_error();
    JDFT_CHECK_ARG(buf && buflen > 0, "null or empty buffer");
    std::lock_guard<std::mutex> lk(g_mu);
    std::map<std::string, std::pair<long long, double>> agg;
    for (const Rec& r : g_recs) {
        JDFT_CUDA_TRY(cudaEventSynchronize(g_pool[r.ev + 1]));
        float ms = 0.f;
        JDFT_CUDA_TRY(cudaEventElapsedTime(&ms, g_pool[r.ev], g_pool[r.ev + 1]));
        auto& a = agg[r.name];
        a.first += 1;
        a.second += ms;
    }
    g_recs.clear();
    g_used = 0;
    std::string out;
    char line[256];
    for (auto& kv : agg) {
        snprintf(line, sizeof line, "%s %lld %.6f\n", kv.first.c_str(), kv.second.first, kv.second.second);
        out += line;
    }
    if ((int)out.size() + 1 > buflen) return set_error(JDFT_ERR_ARG, "buffer too small");
    memcpy(buf, out.c_str(), out.size() + 1);
    return JDFT_OK;
}

}  // extern "C"
