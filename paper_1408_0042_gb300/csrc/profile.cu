// Launch counter and CUDA-event phase timers exposed through the C ABI, and
// the CUDA-graph replay of V-cycles (whose launch counts it keeps).
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

namespace plhr {

namespace {
constexpr size_t kMaxGraphs = 64;   // distinct V-cycle argument sets kept per hierarchy (oldest dropped)
}

cudaError_t mg_graphed(const MGHierarchy& H, int kind, int nc, const void* r, int64_t ldr, const void* w,
                       int64_t ldw, const void* work, cudaStream_t s,
                       const std::function<cudaError_t(cudaStream_t)>& body, const void* r2, int64_t ldr2,
                       int nc2) {
    for (const MGHierarchy::Graph& g : H.graphs)
        if (g.kind == kind && g.nc == nc && g.r == r && g.ldr == ldr && g.w == w && g.ldw == ldw && g.work == work &&
            g.r2 == r2 && g.ldr2 == ldr2 && g.nc2 == nc2) {
            count_launches(g.launches);
            return cudaGraphLaunch(g.exec, s);
        }
    if (H.graphs.size() >= kMaxGraphs) {
        // a replay of the oldest may still be queued: the executable graph is
        // released once that work completes (cudaGraphExecDestroy defers it)
        cudaGraphExecDestroy(H.graphs.front().exec);
        H.graphs.erase(H.graphs.begin());
    }
    if (!H.capture && cudaStreamCreateWithFlags(&H.capture, cudaStreamNonBlocking) != cudaSuccess) {
        H.capture = nullptr;
        cudaGetLastError();
        return body(s);
    }
    // capture (nothing runs): the launches the body counts are taken back and
    // counted again for each replay
    const long long before = g_launches.load();
    if (cudaStreamBeginCapture(H.capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return body(s);
    }
    const cudaError_t eb = body(H.capture);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(H.capture, &graph);
    const int nl = (int)(g_launches.load() - before);
    g_launches.fetch_sub(nl);
    cudaGraphExec_t exec = nullptr;
    cudaError_t ei = cudaErrorUnknown;
    if (eb == cudaSuccess && ee == cudaSuccess && graph) ei = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        return body(s);
    }
    H.graphs.push_back({kind, nc, r, ldr, w, ldw, work, r2, ldr2, nc2, exec, nl});
    count_launches(nl);
    return cudaGraphLaunch(exec, s);
}

void mg_release_graphs(const MGHierarchy& H) {
    for (const MGHierarchy::Graph& g : H.graphs) cudaGraphExecDestroy(g.exec);
    H.graphs.clear();
}

}  // namespace plhr
