// Allocation-free variant of the power step (tucker_power_step_noalloc).
//
// Who needs it: callers that must not allocate device memory while they run.
// Examples are code that runs under a strict memory budget set up once at
// start (an embedded or real-time service that reserves everything in
// advance), code that is called while a caching allocator is locked or
// being torn down, and hosts that forbid cudaMalloc/cudaFree after set-up
// because those calls can synchronise the whole device and stall other work.
// tucker_power_step obtains its per-CTA partial sums from the stream-ordered
// allocator on every call; this entry point takes them instead from one fixed
// block of device memory that is part of the loaded library.
//
// The block is g_noalloc_scratch below (TUCKER_NOALLOC_SCRATCH_BYTES). Every
// GPU that loads this library holds it until the process exits. Host code
// cannot use the array's name as a device address, so the first call on each
// device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it; that first call should therefore come before any
// stream capture. All calls share the block: two calls whose work overlaps on
// the GPU (different host threads or streams, or TUCKER_FLAG_ASYNC calls that
// are still running) race on it, so calls must be ordered by the caller.
// The block keeps the previous call's contents; nothing in it needs clearing
// because every partial sum this call reads is written earlier in the call.
#include <mutex>

#include "internal.h"

namespace tk {
namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[TUCKER_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch block for the current device (set-up on first use).
cudaError_t noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

tucker_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return TUCKER_OK;
    if (e == cudaErrorMemoryAllocation) return TUCKER_ERR_OOM;
    return TUCKER_ERR_CUDA;
}

}  // namespace
}  // namespace tk

extern "C" tucker_status tucker_power_step_noalloc(const void* A, tucker_dtype dt, const int64_t* dims, int N,
                                                   int mode, const void* X_in, int64_t L, void* X_out,
                                                   const tucker_opts* opts) {
    using namespace tk;
    cudaStream_t s = nullptr;
    if (opts) {
        if (opts->struct_size < sizeof(tucker_opts)) return TUCKER_ERR_INVALID_ARG;
        s = reinterpret_cast<cudaStream_t>(opts->stream);
    }
    if (!A || !dims || N < 1 || N > 8 || mode < 0 || mode >= N || !X_in || !X_out || L < 1)
        return TUCKER_ERR_INVALID_ARG;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    ModeView v{1, 0, 1};
    for (int n = 0; n < N; ++n) {
        if (dims[n] < 1) return TUCKER_ERR_INVALID_ARG;
        if (n < mode) v.lf *= dims[n];
        if (n > mode) v.rt *= dims[n];
    }
    v.i = dims[mode];
    const int elem = dt == TUCKER_F64 ? 8 : 4;
    if (v.i > 1024 || L > 4096 || (elem == 8 && v.i > 512)) return TUCKER_ERR_UNSUPPORTED;
    // One partial block (I_n x L) must fit in the fixed scratch; more of them
    // only add parallelism, so the number of partials is capped to what fits.
    const size_t per_part = (size_t)v.i * (size_t)L * elem;
    if (per_part > (size_t)TUCKER_NOALLOC_SCRATCH_BYTES) return TUCKER_ERR_UNSUPPORTED;
    PowerPlan pp = power_plan(v, (int)L, elem, num_sms());
    const int64_t fit = (int64_t)(TUCKER_NOALLOC_SCRATCH_BYTES / per_part);
    if (pp.parts > fit) pp.parts = (int)fit;
    void* scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return status_of(e);
    e = elem == 4 ? launch_power<float>((const float*)A, v, (const float*)X_in, (int)L, (float*)X_out, scratch, pp,
                                        false, 0, 0, s)
                  : launch_power<double>((const double*)A, v, (const double*)X_in, (int)L, (double*)X_out,
                                         scratch, pp, false, 0, 0, s);
    if (e != cudaSuccess) return status_of(e);
    return status_of(cudaStreamSynchronize(s));
}
