// Autotuner: per shape class of a tunable kernel, the first eligible call times
// every candidate configuration on its own data and stream (one warm-up launch,
// one timed launch each, CUDA events) and keeps the fastest; later calls of the
// class, synchronous or not, launch the kept choice. Eligible means: tuning is
// enabled, the calling thread is inside a synchronous library call, and the
// stream is not being captured into a graph (timing needs a synchronisation).
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace tk {
namespace {

struct Entry {
    int choice;
    float ms;
    std::string text;
};

std::mutex g_mu;
std::map<TuneKey, Entry> g_table;
std::vector<std::string> g_lines;        // in order of tuning, for the report
bool g_enabled = false;
thread_local int tl_allowed = 0;

}  // namespace

bool operator<(const TuneKey& a, const TuneKey& b) {
    if (a.site != b.site) return a.site < b.site;
    for (int k = 0; k < 4; ++k)
        if (a.k[k] != b.k[k]) return a.k[k] < b.k[k];
    return false;
}

TuneAllow::TuneAllow(bool allow) : on_(allow) {
    if (on_) ++tl_allowed;
}
TuneAllow::~TuneAllow() {
    if (on_) --tl_allowed;
}

bool tune_active(cudaStream_t s) {
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (!g_enabled) return false;
    }
    if (tl_allowed <= 0) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusNone;
}

int tune_get(const TuneKey& k) {
    std::lock_guard<std::mutex> g(g_mu);
    auto it = g_table.find(k);
    return it == g_table.end() ? -1 : it->second.choice;
}

void tune_put(const TuneKey& k, int choice, float ms, const std::string& text) {
    std::lock_guard<std::mutex> g(g_mu);
    if (g_table.count(k)) return;
    g_table[k] = Entry{choice, ms, text};
    g_lines.push_back(text);
}

float tune_time(cudaStream_t s, const std::function<cudaError_t()>& launch) {
    if (launch() != cudaSuccess) return -1.f;          // warm-up (and shared-memory setup)
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        return -1.f;
    }
    float ms = -1.f;
    cudaEventRecord(a, s);
    const cudaError_t e = launch();
    cudaEventRecord(b, s);
    if (e == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

int tune_pick(cudaStream_t s, const TuneKey& key, const char* what, const std::vector<std::string>& names,
              const std::function<cudaError_t(int)>& launch_candidate, int fallback) {
    int best = -1;
    float best_ms = 0.f;
    std::string times;
    for (int c = 0; c < (int)names.size(); ++c) {
        const float ms = tune_time(s, [&] { return launch_candidate(c); });
        char buf[96];
        snprintf(buf, sizeof(buf), "%s%s %.4f ms", times.empty() ? "" : ", ", names[c].c_str(), ms);
        times += ms >= 0 ? buf : "";
        if (ms >= 0 && (best < 0 || ms < best_ms)) {
            best = c;
            best_ms = ms;
        }
    }
    if (best < 0) best = fallback;
    char head[160];
    snprintf(head, sizeof(head), "%s [%lld, %lld, %lld, %lld] -> %s (", what, (long long)key.k[0],
             (long long)key.k[1], (long long)key.k[2], (long long)key.k[3], names[best].c_str());
    tune_put(key, best, best_ms, std::string(head) + times + ")");
    return best;
}

}  // namespace tk

using namespace tk;

extern "C" {

tucker_status tucker_autotune_enable(int on) {
    std::lock_guard<std::mutex> g(g_mu);
    g_enabled = on != 0;
    return TUCKER_OK;
}

int64_t tucker_autotune_count(void) {
    std::lock_guard<std::mutex> g(g_mu);
    return (int64_t)g_lines.size();
}

const char* tucker_autotune_entry(int64_t k) {
    static thread_local std::string copy;
    std::lock_guard<std::mutex> g(g_mu);
    if (k < 0 || k >= (int64_t)g_lines.size()) return "";
    copy = g_lines[(size_t)k];
    return copy.c_str();
}

}  // extern "C"
