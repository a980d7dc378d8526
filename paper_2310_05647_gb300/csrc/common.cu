// Error reporting, launch accounting and the per-kernel event profiler of the
// C ABI.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.h"

namespace mrf {
static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

namespace {
struct Mark {
    const char* name;   // nullptr: boundary mark
    cudaStream_t stream;
    cudaEvent_t ev;
};
struct Profiler {
    std::mutex mu;
    bool on = false;
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
    std::map<std::string, std::pair<double, long long>> acc;
    std::vector<std::pair<std::string, std::pair<double, long long>>> table;

    cudaEvent_t event() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void record(const char* name, cudaStream_t s) {
        cudaEvent_t e = event();
        if (e && cudaEventRecord(e, s) == cudaSuccess) marks.push_back({name, s, e});
    }
};
Profiler& prof() {
    static Profiler* p = new Profiler();   // never destroyed: usable during process exit
    return *p;
}
std::atomic<long long> g_launches{0};
}  // namespace

long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
void note_replayed_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool profiling_enabled() {
    Profiler& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    return P.on;
}

void note_launch(const char* name, cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    Profiler& P = prof();
    if (!P.on) return;
    std::lock_guard<std::mutex> lk(P.mu);
    if (P.on) P.record(name, s);
}
}  // namespace mrf

using namespace mrf;

extern "C" const char* mrf_last_error(void) { return mrf::g_err; }
extern "C" int mrf_abi_version(void) { return 1; }

extern "C" long long mrf_launch_count(void) { return g_launches.load(); }

extern "C" mrf_status mrf_profile_enable(int on) {
    Profiler& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    for (auto& m : P.marks) P.pool.push_back(m.ev);
    P.marks.clear();
    P.acc.clear();
    P.table.clear();
    P.on = on != 0;
    return MRF_OK;
}

extern "C" mrf_status mrf_profile_mark(mrf_stream stream) {
    Profiler& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    if (P.on) P.record(nullptr, as_stream(stream));
    return MRF_OK;
}

extern "C" int mrf_profile_collect(void) {
    Profiler& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    std::map<cudaStream_t, cudaEvent_t> last;
    for (auto& m : P.marks) {
        if (cudaEventSynchronize(m.ev) != cudaSuccess) {
            set_error("mrf_profile_collect: event wait failed");
            return -1;
        }
        auto it = last.find(m.stream);
        if (m.name && it != last.end()) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, it->second, m.ev) == cudaSuccess) {
                auto& a = P.acc[m.name];
                a.first += ms;
                a.second += 1;
            }
        }
        last[m.stream] = m.ev;
    }
    for (auto& m : P.marks) P.pool.push_back(m.ev);
    P.marks.clear();
    P.table.assign(P.acc.begin(), P.acc.end());
    return (int)P.table.size();
}

extern "C" mrf_status mrf_profile_entry(int i, char* name, int name_len, double* ms, long long* launches) {
    Profiler& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    MRF_REQUIRE(i >= 0 && i < (int)P.table.size(), "mrf_profile_entry: index %d out of range", i);
    if (name && name_len > 0) {
        std::strncpy(name, P.table[i].first.c_str(), (size_t)name_len - 1);
        name[name_len - 1] = 0;
    }
    if (ms) *ms = P.table[i].second.first;
    if (launches) *launches = P.table[i].second.second;
    return MRF_OK;
}
