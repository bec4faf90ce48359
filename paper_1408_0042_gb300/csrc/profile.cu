// Launch counter and CUDA-event phase timers exposed through the C ABI.
#include <atomic>
#include <mutex>
#include <vector>

#include "plhr_internal.h"

namespace plhr {
namespace {
std::atomic<long long> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_mu;
struct Pending {
    int phase;
    cudaEvent_t a, b;
};
std::vector<Pending> g_pending;
double g_ms[PH_COUNT] = {0};
long long g_calls[PH_COUNT] = {0};
double g_work[PH_COUNT] = {0};
double g_bytes[PH_COUNT] = {0};
}  // namespace

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

PhaseScope::PhaseScope(int ph, cudaStream_t st, double work, double bytes) : phase(ph), s(st) {
    if (!g_prof_on.load()) return;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_work[ph] += work;
        g_bytes[ph] += bytes;
    }
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) { a = b = nullptr; return; }
    cudaEventRecord(a, s);
}

PhaseScope::~PhaseScope() {
    if (!a) return;
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back({phase, a, b});
}

void profile_flush() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_ms[p.phase] += ms;
            g_calls[p.phase] += 1;
        }
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pending.clear();
}

}  // namespace plhr

extern "C" {

long long plhr_kernel_launches(void) { return plhr::g_launches.load(); }

void plhr_profile_enable(int on) {
    plhr::profile_flush();
    plhr::g_prof_on.store(on ? 1 : 0);
}

void plhr_profile_read(double* ms, long long* calls, int reset) {
    plhr::profile_flush();
    std::lock_guard<std::mutex> lk(plhr::g_mu);
    for (int i = 0; i < plhr::PH_COUNT; ++i) {
        if (ms) ms[i] = plhr::g_ms[i];
        if (calls) calls[i] = plhr::g_calls[i];
        if (reset) { plhr::g_ms[i] = 0.0; plhr::g_calls[i] = 0; plhr::g_work[i] = 0.0; plhr::g_bytes[i] = 0.0; }
    }
}

void plhr_profile_work(double* work) {
    plhr::profile_flush();
    std::lock_guard<std::mutex> lk(plhr::g_mu);
    for (int i = 0; i < plhr::PH_COUNT; ++i)
        if (work) work[i] = plhr::g_work[i];
}

void plhr_profile_bytes(double* bytes) {
    plhr::profile_flush();
    std::lock_guard<std::mutex> lk(plhr::g_mu);
    for (int i = 0; i < plhr::PH_COUNT; ++i)
        if (bytes) bytes[i] = plhr::g_bytes[i];
}

}  // extern "C"
