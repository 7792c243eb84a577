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
// cannot use the array's name as a device address, so the address is looked
// up with cudaGetSymbolAddress, with the device current, once per device and
// context: the first call on a device does this set-up (and so does the first
// call after that device's context was destroyed and created again, e.g. by
// cudaDeviceReset, which gives the block a new address), so the first call on
// a device should come before any stream capture. All calls share the block:
// two calls whose work overlaps on the GPU (different host threads or
// streams) race on it, so calls must be ordered by the caller. The block
// keeps the previous call's contents; nothing in it needs clearing because
// every partial sum this call reads is written earlier in the call.
//
// Only the exact FFMA arithmetic is served (opts->prec TUCKER_SK_FP32): the
// tensor-core forms of tucker_power_step keep a status word beside their
// partials, which this block does not provide.
#include <mutex>

#include <cuda.h>

#include "internal.h"

namespace tk {
namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[TUCKER_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
struct Cached {
    unsigned long long ctx_id = 0;   // 0: not set up
    void* addr = nullptr;
};
Cached g_noalloc[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// The driver's context queries, looked up once through the runtime.
template <typename Fn>
Fn driver_fn(const char* name) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        return reinterpret_cast<Fn>(p);
    cudaGetLastError();
    return nullptr;
}

// Unique id of the calling thread's current context, or 0 when there is none
// yet or the driver cannot say.
unsigned long long current_context_id() {
    static const CtxGetCurrentFn get_ctx = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
    static const CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
    if (!get_ctx || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_ctx(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch block for the current device, set up on the
// first call on a device and again when the device's context has changed; when
// the context cannot be identified the address is looked up on every call.
cudaError_t noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    unsigned long long id = current_context_id();
    Cached& c = g_noalloc[dev];
    if (id == 0 || c.ctx_id != id) {
        void* p = nullptr;
        // makes the runtime's context current if none was (the first call on a device)
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (id == 0) id = current_context_id();
        c.addr = p;
        c.ctx_id = id;
    }
    *out = c.addr;
    return cudaSuccess;
}

}  // namespace
}  // namespace tk

extern "C" tucker_status tucker_power_step_noalloc(const void* A, tucker_dtype dt, const int64_t* dims, int N,
                                                   int mode, const void* X_in, int64_t L, void* X_out,
                                                   const tucker_opts* opts) {
    using namespace tk;
    cudaStream_t s = nullptr;
    if (opts) {
        // the same option checks as tucker_power_step
        if (opts->struct_size < sizeof(tucker_opts)) return TUCKER_ERR_INVALID_ARG;
        if (opts->form != TUCKER_FORM_PAPER && opts->form != TUCKER_FORM_RANGE && opts->form != TUCKER_FORM_RELATED)
            return TUCKER_ERR_INVALID_ARG;
        if (opts->prec < TUCKER_SK_FP32 || opts->prec > TUCKER_SK_BF16X1) return TUCKER_ERR_INVALID_ARG;
        if (!(opts->alpha >= 0.0) || opts->alpha > 1.0) return TUCKER_ERR_INVALID_ARG;
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
    if (opts && opts->prec != TUCKER_SK_FP32) return TUCKER_ERR_UNSUPPORTED;
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
    if (e != cudaSuccess) return status_from_cuda(e);
    e = elem == 4 ? launch_power<float>((const float*)A, v, (const float*)X_in, (int)L, (float*)X_out, scratch, pp,
                                        false, 0, 0, s)
                  : launch_power<double>((const double*)A, v, (const double*)X_in, (int)L, (double*)X_out,
                                         scratch, pp, false, 0, 0, s);
    if (e != cudaSuccess) return status_from_cuda(e);
    return status_from_cuda(cudaStreamSynchronize(s));
}
