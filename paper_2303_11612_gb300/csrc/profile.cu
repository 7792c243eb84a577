// Launch counting and an optional per-kernel-class CUDA-event profiler.
//
// Every kernel launch made by the library bumps a process-wide counter. When
// profiling is on, the launches of the heavy kernels are bracketed by CUDA
// events on their own stream and carry the launch's algorithmic bytes and
// flops; the events are read back after the stream is synchronised.
#include <atomic>
#include <mutex>
#include <vector>

#include "internal.h"

namespace tk {
namespace {

struct Rec {
    int cls;
    double bytes, flops;
    cudaEvent_t a, b;
};
struct Accum {
    long long launches = 0;
    double ms = 0, bytes = 0, flops = 0;
};

std::atomic<long long> g_launches{0};
std::atomic<bool> g_enabled{false};
std::mutex g_mu;
std::vector<Rec> g_pending;
std::vector<cudaEvent_t> g_pool;
Accum g_acc[kKernelClasses];

cudaEvent_t get_event() {
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

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

ProfScope::ProfScope(int cls, double bytes, double flops, cudaStream_t s)
    : cls_(cls), bytes_(bytes), flops_(flops), s_(s) {
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> g(g_mu);
    a_ = get_event();
    b_ = get_event();
    if (a_) cudaEventRecord((cudaEvent_t)a_, s_);
}

ProfScope::~ProfScope() {
    if (!a_) return;
    cudaEventRecord((cudaEvent_t)b_, s_);
    std::lock_guard<std::mutex> g(g_mu);
    g_pending.push_back(Rec{cls_, bytes_, flops_, (cudaEvent_t)a_, (cudaEvent_t)b_});
}

void profile_drain() {
    std::lock_guard<std::mutex> g(g_mu);
    for (const Rec& r : g_pending) {
        float ms = 0.f;
        const bool ok = cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess;
        if (!ok) cudaGetLastError();     // leave no stale error for the next launch check
        if (ok) {
            Accum& a = g_acc[r.cls];
            a.launches += 1;
            a.ms += ms;
            a.bytes += r.bytes;
            a.flops += r.flops;
        }
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_pending.clear();
}

}  // namespace tk

extern "C" {

int64_t tucker_launch_count(void) { return tk::g_launches.load(); }

tucker_status tucker_profile_enable(int on) {
    tk::profile_drain();
    std::lock_guard<std::mutex> g(tk::g_mu);
    for (auto& a : tk::g_acc) a = tk::Accum{};
    tk::g_enabled.store(on != 0);
    return TUCKER_OK;
}

tucker_status tucker_profile_read(int kernel_class, int64_t* launches, double* total_ms, double* bytes,
                                  double* flops) {
    if (kernel_class < 0 || kernel_class >= tk::kKernelClasses) return TUCKER_ERR_INVALID_ARG;
    tk::profile_drain();
    std::lock_guard<std::mutex> g(tk::g_mu);
    const tk::Accum& a = tk::g_acc[kernel_class];
    if (launches) *launches = a.launches;
    if (total_ms) *total_ms = a.ms;
    if (bytes) *bytes = a.bytes;
    if (flops) *flops = a.flops;
    return TUCKER_OK;
}

}  // extern "C"
