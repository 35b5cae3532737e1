// profile.cu -- launch accounting of libcsc.
//
// Every kernel launch of the library goes through CSC_KLAUNCH, which counts
// it and, while profiling is enabled, brackets it with a pair of CUDA events
// recorded on the launch's own stream and tags it with a kernel-class name
// and the launch's algorithmic bytes (the bytes the operation must move at
// minimum, as defined at each launch site).  csc_profile_query sums the
// event-measured durations per class.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace csc {

bool g_prof_enabled = false;
std::atomic<long long> g_launches{0};

namespace {
struct Mark {
    int cls;
    cudaEvent_t a, b;
};
struct Class {
    std::string name;
    long long launches = 0;
    double bytes = 0.0;
    double ms = 0.0;
};
std::mutex g_mu;
std::vector<Mark> g_marks;          // pending (unresolved) marks
std::vector<cudaEvent_t> g_pool;    // free events
std::vector<Class> g_classes;

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

int class_of(const char* name) {
    for (size_t i = 0; i < g_classes.size(); ++i)
        if (g_classes[i].name == name) return (int)i;
    g_classes.push_back(Class{name});
    return (int)g_classes.size() - 1;
}

// Resolve pending marks (requires their events to have completed).
void resolve_locked() {
    for (const Mark& m : g_marks) {
        float ms = 0.f;
        if (cudaEventSynchronize(m.b) == cudaSuccess && cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess)
            g_classes[m.cls].ms += ms;
        else
            cudaGetLastError();
        g_pool.push_back(m.a);
        g_pool.push_back(m.b);
    }
    g_marks.clear();
}
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

int prof_begin(const char* name, double bytes, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    const int c = class_of(name);
    g_classes[c].launches += 1;
    g_classes[c].bytes += bytes;
    Mark m{c, take_event(), take_event()};
    if (!m.a || !m.b) return -1;
    cudaEventRecord(m.a, s);
    g_marks.push_back(m);
    return (int)g_marks.size() - 1;
}

void prof_end(int slot, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (slot >= 0 && slot < (int)g_marks.size()) cudaEventRecord(g_marks[slot].b, s);
}

}  // namespace csc

using namespace csc;

extern "C" {

csc_status csc_profile_enable(int32_t on) {
    g_prof_enabled = on != 0;
    return CSC_OK;
}

csc_status csc_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    resolve_locked();
    g_classes.clear();
    g_launches.store(0);
    return CSC_OK;
}

csc_status csc_profile_launches(int64_t* n) {
    if (!n) return CSC_E_INVALID;
    *n = (int64_t)g_launches.load();
    return CSC_OK;
}

csc_status csc_profile_query(int32_t i, char* name, int32_t name_len, int64_t* launches, double* total_ms,
                             double* bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    resolve_locked();
    if (i < 0 || i >= (int32_t)g_classes.size()) return CSC_E_INVALID;
    const Class& c = g_classes[i];
    if (name && name_len > 0) {
        const size_t n = std::min((size_t)(name_len - 1), c.name.size());
        memcpy(name, c.name.data(), n);
        name[n] = 0;
    }
    if (launches) *launches = c.launches;
    if (total_ms) *total_ms = c.ms;
    if (bytes) *bytes = c.bytes;
    return CSC_OK;
}

}  // extern "C"
