// Serving loop: decompositions submitted from any host thread wait in a FIFO
// queue, are admitted against a device-memory budget when one of max_inflight
// streams is free, and run as asynchronous decompositions on their own stream,
// so admitted requests overlap on the device and a new arrival starts as soon
// as a stream and memory free up (continuous batching at request granularity).
//
// One worker thread owns every CUDA call of the server: it retires finished
// requests (event query, device status word read back into pinned memory,
// stream-ordered free), then admits from the head of the queue. Device memory
// comes from a pool private to the server (stream-ordered allocation, kept
// mapped for the server's lifetime). Head-of-line order is strict, so a large request
// is never overtaken indefinitely by small ones. Host inputs are staged by one
// copy stream shared by all requests, in admission order: concurrent
// host-to-device copies on many streams share the chip link badly (a third of
// one stream's rate in eight, measured), while one stream keeps it busy and
// each request's decomposition starts as soon as its own copy lands.
//
// With ticks, the consecutive requests at the head of the queue that the work
// list takes (and that are small enough) are admitted together into one block
// of memory and run as one work-list batch on the slot's stream (the work-list
// kernel's steps and grouped orthonormalisations, worklist.cu); each request
// keeps its workspace slice, status word and completion.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxN = 8;
constexpr size_t kAlign = 256;

size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

bool device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct Request {
    uint64_t ticket = 0;
    int which = 1;
    tucker_dtype dt = TUCKER_F32;
    const void* A = nullptr;
    int N = 0;
    int64_t dims[kMaxN] = {};
    int32_t ranks[kMaxN] = {};
    int32_t P = 0, q = 1;
    int64_t c = 0;
    tucker_prob prob = TUCKER_PROB_UNIFORM;
    uint64_t seed = 0;
    void* U[kMaxN] = {};
    void* G = nullptr;
    bool hostA = false, hostU[kMaxN] = {}, hostG = false;
    size_t ws = 0, a_bytes = 0, u_bytes[kMaxN] = {}, g_bytes = 0, need = 0;
    Clock::time_point t_submit, t_done;
    void* block = nullptr;
    tucker_status result = TUCKER_OK;
    bool done = false;
    bool tickable = false;        // the work list takes it (ticks on, small enough)
};

struct Slot {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t ev_alloc = nullptr;   // the request's block is allocated (on s)
    cudaEvent_t ev_copy = nullptr;    // its input has landed (on the copy stream)
    int* h_status = nullptr;      // pinned word the request's device status is copied into
    Request* r = nullptr;
    // a tick: its requests, their pinned status words, the pinned descriptor image
    std::vector<Request*> tick;
    int* h_tick_status = nullptr;
    void* h_desc = nullptr;
    size_t desc_cap = 0;
    size_t tick_extra = 0;        // budget bytes of the tick beyond its requests' own (the descriptor area)
    cudaEvent_t ev_upload = nullptr;
    bool busy() const { return r != nullptr || !tick.empty(); }
};

}  // namespace

struct tucker_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::vector<std::unique_ptr<Request>> reqs;      // index ticket - 1
    std::vector<Slot> slots;
    cudaMemPool_t pool = nullptr;
    cudaStream_t copy_s = nullptr;    // host-to-device staging of every request's input
    int device = 0;
    size_t budget = 0, in_use = 0, peak = 0;
    int inflight = 0, peak_inflight = 0;
    int32_t form = 0, prec = 0;
    int tick_max = 0;
    int64_t tick_elems = 0;
    uint64_t ticks = 0, tick_requests = 0;
    bool stop = false;
    std::vector<double> lat_ms;
    uint64_t failed = 0;
    bool any_submit = false;
    Clock::time_point t_first, t_last;
    std::thread worker;

    void run();
    bool launch(Slot& sl, Request* r);
    void retire(Slot& sl, tucker_status st);
    // ticks
    size_t tick_plan(const std::vector<Request*>& rs, tk::WorklistPlan* wp, std::vector<tucker_request>* treqs,
                     std::vector<size_t>* offsets, size_t* area_off, char* base, void** dU_store);
    bool launch_tick(Slot& sl, std::vector<Request*>& rs, size_t extra);
    void retire_tick(Slot& sl, tucker_status st);
};

// The block layout of a tick (each request: workspace slice, staged input, staged
// outputs; then the work-list area) and its plan, from base (null: sizes only).
// dU_store holds kMaxN device pointers per request. Returns the block's bytes, 0 if
// the work list refuses the set.
size_t tucker_server::tick_plan(const std::vector<Request*>& rs, tk::WorklistPlan* wp,
                                std::vector<tucker_request>* treqs, std::vector<size_t>* offsets, size_t* area_off,
                                char* base, void** dU_store) {
    const int n = (int)rs.size();
    treqs->assign(n, tucker_request{});
    offsets->assign(n, 0);
    size_t off = 0;
    for (int k = 0; k < n; ++k) {
        Request* r = rs[k];
        (*offsets)[k] = off;
        off += up(r->ws);
        tucker_request& t = (*treqs)[k];
        t.struct_size = sizeof(tucker_request);
        t.which = r->which;
        t.dt = r->dt;
        t.A = r->A;
        if (r->hostA) {
            t.A = base ? base + off : nullptr;
            off += up(r->a_bytes);
        }
        t.dims = r->dims;
        t.N = r->N;
        t.ranks = r->ranks;
        t.P = r->P;
        t.q = r->q;
        t.c = r->c;
        t.prob = r->prob;
        t.seed = r->seed;
        void** dU = dU_store + (size_t)k * kMaxN;
        for (int m = 0; m < r->N; ++m) {
            dU[m] = r->U[m];
            if (r->hostU[m]) {
                dU[m] = base ? base + off : (void*)(uintptr_t)256;
                off += up(r->u_bytes[m]);
            }
        }
        t.U = dU;
        t.G = r->G;
        if (r->hostG) {
            t.G = base ? base + off : (void*)(uintptr_t)256;
            off += up(r->g_bytes);
        }
    }
    tucker_opts o;
    std::memset(&o, 0, sizeof(o));
    o.struct_size = sizeof(o);
    o.form = form;
    o.prec = prec;
    if (tk::worklist_plan(n, treqs->data(), o, base, *offsets, *wp, 1) != TUCKER_OK) return 0;
    *area_off = off;
    return off + up(wp->area_bytes);
}

bool tucker_server::launch(Slot& sl, Request* r) {
    cudaStream_t s = sl.s;
    if (cudaMallocFromPoolAsync(&r->block, r->need, pool, s) != cudaSuccess) {
        cudaGetLastError();
        r->block = nullptr;
        r->result = TUCKER_ERR_OOM;
        return false;
    }
    char* b = (char*)r->block;
    void* ws = b;
    b += up(r->ws);
    const void* dA = r->A;
    if (r->hostA) {
        dA = b;
        cudaEventRecord(sl.ev_alloc, s);
        cudaStreamWaitEvent(copy_s, sl.ev_alloc, 0);
        cudaMemcpyAsync(b, r->A, r->a_bytes, cudaMemcpyHostToDevice, copy_s);
        cudaEventRecord(sl.ev_copy, copy_s);
        cudaStreamWaitEvent(s, sl.ev_copy, 0);
        b += up(r->a_bytes);
    }
    void* dU[kMaxN];
    for (int n = 0; n < r->N; ++n) {
        dU[n] = r->U[n];
        if (r->hostU[n]) {
            dU[n] = b;
            b += up(r->u_bytes[n]);
        }
    }
    void* dG = r->G;
    if (r->hostG) dG = b;
    tucker_opts o;
    std::memset(&o, 0, sizeof(o));
    o.struct_size = sizeof(o);
    o.form = form;
    o.prec = prec;
    o.flags = TUCKER_FLAG_ASYNC;
    o.stream = s;
    o.workspace = ws;
    o.workspace_bytes = r->ws;
    const tucker_status st =
        r->which ? tucker_rsthosvd(dA, r->dt, r->dims, r->N, r->ranks, r->P, r->q, r->c, r->prob, r->seed, dU, dG, &o)
                 : tucker_rthosvd(dA, r->dt, r->dims, r->N, r->ranks, r->P, r->q, r->c, r->prob, r->seed, dU, dG, &o);
    if (st != TUCKER_OK) {
        r->result = st;
        *sl.h_status = 0;
    } else {
        for (int n = 0; n < r->N; ++n)
            if (r->hostU[n]) cudaMemcpyAsync(r->U[n], dU[n], r->u_bytes[n], cudaMemcpyDeviceToHost, s);
        if (r->hostG) cudaMemcpyAsync(r->G, dG, r->g_bytes, cudaMemcpyDeviceToHost, s);
        // the status word sits at the start of an asynchronous call's workspace
        cudaMemcpyAsync(sl.h_status, ws, sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    cudaFreeAsync(r->block, s);
    if (cudaEventRecord(sl.ev, s) != cudaSuccess) {
        cudaGetLastError();
        if (r->result == TUCKER_OK) r->result = TUCKER_ERR_CUDA;
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return false;
    }
    sl.r = r;
    return true;
}

bool tucker_server::launch_tick(Slot& sl, std::vector<Request*>& rs, size_t extra) {
    cudaStream_t s = sl.s;
    const int n = (int)rs.size();
    tk::WorklistPlan wp;
    std::vector<tucker_request> treqs;
    std::vector<size_t> offsets;
    std::vector<void*> dU((size_t)n * kMaxN);
    size_t area_off = 0;
    const size_t bytes = tick_plan(rs, &wp, &treqs, &offsets, &area_off, nullptr, dU.data());
    void* block = nullptr;
    auto fail = [&](tucker_status st) {
        for (Request* r : rs) r->result = st;
        for (int k = 0; k < n; ++k) sl.h_tick_status[k] = 0;
        return false;
    };
    if (!bytes) return fail(TUCKER_ERR_UNSUPPORTED);
    if (cudaMallocFromPoolAsync(&block, bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(TUCKER_ERR_OOM);
    }
    char* b = (char*)block;
    if (!tick_plan(rs, &wp, &treqs, &offsets, &area_off, b, dU.data())) {
        cudaFreeAsync(block, s);
        return fail(TUCKER_ERR_UNSUPPORTED);
    }
    // the descriptor image: the slot's pinned buffer (free: the slot's last work has completed)
    if (sl.desc_cap < wp.desc_bytes) {
        if (sl.h_desc) cudaFreeHost(sl.h_desc);
        sl.h_desc = nullptr;
        sl.desc_cap = 0;
        if (cudaMallocHost(&sl.h_desc, wp.desc_bytes) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeAsync(block, s);
            return fail(TUCKER_ERR_OOM);
        }
        sl.desc_cap = wp.desc_bytes;
    }
    tk::worklist_pack(wp, sl.h_desc);
    tk::worklist_prepare(wp);
    // host inputs through the copy stream, in admission order
    bool staged = false;
    for (int k = 0; k < n; ++k) {
        Request* r = rs[k];
        if (!r->hostA) continue;
        if (!staged) {
            cudaEventRecord(sl.ev_alloc, s);
            cudaStreamWaitEvent(copy_s, sl.ev_alloc, 0);
            staged = true;
        }
        cudaMemcpyAsync((void*)treqs[k].A, r->A, r->a_bytes, cudaMemcpyHostToDevice, copy_s);
    }
    if (staged) {
        cudaEventRecord(sl.ev_copy, copy_s);
        cudaStreamWaitEvent(s, sl.ev_copy, 0);
    }
    std::vector<cudaStream_t> lanes{s};
    cudaError_t e = tk::worklist_enqueue(wp, b + area_off, sl.h_desc, lanes, sl.ev_upload);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        Request* r = rs[k];
        for (int m = 0; m < r->N; ++m)
            if (r->hostU[m]) cudaMemcpyAsync(r->U[m], treqs[k].U[m], r->u_bytes[m], cudaMemcpyDeviceToHost, s);
        if (r->hostG) cudaMemcpyAsync(r->G, treqs[k].G, r->g_bytes, cudaMemcpyDeviceToHost, s);
        // each request's status word sits at the start of its workspace slice
        e = cudaMemcpyAsync(sl.h_tick_status + k, b + offsets[k], sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    cudaFreeAsync(block, s);
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev, s);
    sl.tick = rs;
    sl.tick_extra = extra;
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (Request* r : rs)
            if (r->result == TUCKER_OK) r->result = tk::status_from_cuda(e);
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return false;
    }
    return true;
}

void tucker_server::retire_tick(Slot& sl, tucker_status st) {
    std::vector<Request*> rs;
    rs.swap(sl.tick);
    std::lock_guard<std::mutex> g(mu);
    in_use -= sl.tick_extra;
    sl.tick_extra = 0;
    const auto now = Clock::now();
    for (size_t k = 0; k < rs.size(); ++k) {
        Request* r = rs[k];
        if (r->result == TUCKER_OK) {
            if (st != TUCKER_OK) r->result = st;
            else if (sl.h_tick_status[k] & 2) r->result = TUCKER_ERR_TIMEOUT;
            else if (sl.h_tick_status[k] & 1) r->result = TUCKER_ERR_NUMERICAL;
        }
        in_use -= r->need;
        --inflight;
        r->t_done = now;
        r->done = true;
        if (r->result == TUCKER_OK)
            lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
        else
            ++failed;
    }
    t_last = now;
    cv_done.notify_all();
}

void tucker_server::retire(Slot& sl, tucker_status st) {
    Request* r = sl.r;
    if (r->result == TUCKER_OK) {
        if (st != TUCKER_OK) r->result = st;
        else if (*sl.h_status & 2) r->result = TUCKER_ERR_TIMEOUT;
        else if (*sl.h_status & 1) r->result = TUCKER_ERR_NUMERICAL;
    }
    sl.r = nullptr;
    std::lock_guard<std::mutex> g(mu);
    in_use -= r->need;
    --inflight;
    r->t_done = Clock::now();
    r->done = true;
    if (r->result == TUCKER_OK)
        lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    else
        ++failed;
    t_last = r->t_done;
    cv_done.notify_all();
}

void tucker_server::run() {
    cudaSetDevice(device);
    for (;;) {
        // retire what has finished
        for (Slot& sl : slots) {
            if (!sl.busy()) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) cudaGetLastError();
            if (sl.r) retire(sl, q == cudaSuccess ? TUCKER_OK : TUCKER_ERR_CUDA);
            else retire_tick(sl, q == cudaSuccess ? TUCKER_OK : TUCKER_ERR_CUDA);
        }
        // admit from the head of the queue while a stream and memory are free
        for (;;) {
            Request* r = nullptr;
            Slot* free_slot = nullptr;
            std::vector<Request*> tick;
            size_t extra = 0;
            {
                std::lock_guard<std::mutex> g(mu);
                if (pending.empty()) break;
                for (Slot& sl : slots)
                    if (!sl.busy()) { free_slot = &sl; break; }
                if (!free_slot || in_use + pending.front()->need > budget) break;
                if (pending.front()->tickable) {
                    // the tickable requests at the head (one element type), as many as
                    // fit the budget with the tick's descriptor area
                    size_t sum = 0;
                    const tucker_dtype dt = pending.front()->dt;
                    for (size_t i = 0; i < pending.size() && (int)tick.size() < tick_max; ++i) {
                        Request* c = pending[i];
                        if (!c->tickable || c->dt != dt || in_use + sum + c->need > budget) break;
                        tick.push_back(c);
                        sum += c->need;
                    }
                    while (!tick.empty()) {
                        tk::WorklistPlan wp;
                        std::vector<tucker_request> t;
                        std::vector<size_t> offs;
                        size_t area_off = 0;
                        std::vector<void*> dU(tick.size() * kMaxN);
                        const size_t bytes = tick_plan(tick, &wp, &t, &offs, &area_off, nullptr, dU.data());
                        extra = bytes > sum ? bytes - sum : 0;
                        if (bytes && in_use + sum + extra <= budget) break;
                        sum -= tick.back()->need;
                        tick.pop_back();
                    }
                }
                if (!tick.empty()) {
                    ++ticks;
                    tick_requests += tick.size();
                    pending.erase(pending.begin(), pending.begin() + (long)tick.size());
                    in_use += extra;
                    for (Request* c : tick) in_use += c->need;
                    inflight += (int)tick.size();
                } else {
                    r = pending.front();
                    pending.pop_front();
                    in_use += r->need;
                    ++inflight;
                }
                peak = std::max(peak, in_use);
                peak_inflight = std::max(peak_inflight, inflight);
            }
            if (!tick.empty()) {
                if (!launch_tick(*free_slot, tick, extra)) {
                    free_slot->tick = tick;
                    free_slot->tick_extra = extra;
                    retire_tick(*free_slot, TUCKER_OK);
                }
                continue;
            }
            if (!launch(*free_slot, r)) {
                free_slot->r = r;
                retire(*free_slot, r->result);
            }
        }
        std::unique_lock<std::mutex> lk(mu);
        if (inflight == 0 && pending.empty()) {
            if (stop) break;
            cv_work.wait(lk, [&] { return stop || !pending.empty(); });
        } else {
            // work on the device: poll at a short interval (or sooner on a submission)
            cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

extern "C" {

tucker_status tucker_server_create(const tucker_server_opts* opts, tucker_server** out) {
    if (!opts || !out || opts->struct_size < sizeof(tucker_server_opts)) return TUCKER_ERR_INVALID_ARG;
    if (opts->max_inflight < 1 || opts->max_inflight > 256 || opts->budget_bytes == 0) return TUCKER_ERR_INVALID_ARG;
    if (opts->form != TUCKER_FORM_PAPER && opts->form != TUCKER_FORM_RANGE && opts->form != TUCKER_FORM_RELATED)
        return TUCKER_ERR_INVALID_ARG;
    if (opts->prec < TUCKER_SK_FP32 || opts->prec > TUCKER_SK_BF16X1) return TUCKER_ERR_INVALID_ARG;
    if (opts->tick_max < 0 || opts->tick_max > 256 || (opts->tick_max > 1 && opts->tick_elems < 1))
        return TUCKER_ERR_INVALID_ARG;
    // ticks run the work-list path, which is planned but not run: see the header
    if (opts->tick_max > 1) return TUCKER_ERR_UNSUPPORTED;
    std::unique_ptr<tucker_server> s(new tucker_server());
    s->budget = opts->budget_bytes;
    s->form = opts->form;
    s->prec = opts->prec;
    s->tick_max = opts->tick_max > 1 ? opts->tick_max : 0;
    s->tick_elems = opts->tick_elems;
    cudaError_t e = cudaGetDevice(&s->device);
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if (e == cudaSuccess) e = cudaMemPoolCreate(&s->pool, &props);
    if (e == cudaSuccess) {
        // the pool keeps every block it has mapped until the server is destroyed: blocks of
        // recurring request sizes are then reused instead of being unmapped at a
        // synchronisation and mapped again (tens of milliseconds for GB-sized blocks); the
        // budget, not the pool, bounds what is admitted
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_s, cudaStreamNonBlocking);
    s->slots.resize(opts->max_inflight);
    for (Slot& sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_alloc, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_copy, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_upload, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.h_status, sizeof(int));
        if (e == cudaSuccess) *sl.h_status = 0;
        if (e == cudaSuccess && s->tick_max > 1)
            e = cudaMallocHost((void**)&sl.h_tick_status, sizeof(int) * (size_t)s->tick_max);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (Slot& sl : s->slots) {
            if (sl.s) cudaStreamDestroy(sl.s);
            if (sl.ev) cudaEventDestroy(sl.ev);
            if (sl.ev_alloc) cudaEventDestroy(sl.ev_alloc);
            if (sl.ev_copy) cudaEventDestroy(sl.ev_copy);
            if (sl.ev_upload) cudaEventDestroy(sl.ev_upload);
            if (sl.h_status) cudaFreeHost(sl.h_status);
            if (sl.h_tick_status) cudaFreeHost(sl.h_tick_status);
        }
        if (s->copy_s) cudaStreamDestroy(s->copy_s);
        if (s->pool) cudaMemPoolDestroy(s->pool);
        return e == cudaErrorMemoryAllocation ? TUCKER_ERR_OOM : TUCKER_ERR_CUDA;
    }
    tucker_server* raw = s.release();
    raw->worker = std::thread([raw] { raw->run(); });
    *out = raw;
    return TUCKER_OK;
}

tucker_status tucker_server_submit(tucker_server* srv, const tucker_request* req, uint64_t* ticket) {
    if (!srv || !req || !ticket || req->struct_size < sizeof(tucker_request)) return TUCKER_ERR_INVALID_ARG;
    if (req->N < 1 || req->N > kMaxN || !req->A || !req->dims || !req->ranks || !req->U || !req->G)
        return TUCKER_ERR_INVALID_ARG;
    if (req->which != 0 && req->which != 1) return TUCKER_ERR_INVALID_ARG;
    if (req->dt != TUCKER_F32 && req->dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    std::unique_ptr<Request> r(new Request());
    r->which = req->which;
    r->dt = req->dt;
    r->A = req->A;
    r->N = req->N;
    r->P = req->P;
    r->q = req->q;
    r->c = req->c;
    r->prob = req->prob;
    r->seed = req->seed;
    r->G = req->G;
    const size_t elem = req->dt == TUCKER_F64 ? 8 : 4;
    size_t E = 1, Gn = 1;
    for (int n = 0; n < r->N; ++n) {
        if (!req->U[n]) return TUCKER_ERR_INVALID_ARG;
        r->dims[n] = req->dims[n];
        r->ranks[n] = req->ranks[n];
        r->U[n] = req->U[n];
        if (r->dims[n] < 1 || r->ranks[n] < 1 || r->ranks[n] > r->dims[n]) return TUCKER_ERR_INVALID_ARG;
        E *= (size_t)r->dims[n];
        Gn *= (size_t)r->ranks[n];
    }
    tucker_opts o;
    std::memset(&o, 0, sizeof(o));
    o.struct_size = sizeof(o);
    o.form = srv->form;
    o.prec = srv->prec;
    const tucker_status ws = tucker_workspace_size(r->which, r->dt, r->dims, r->N, r->ranks, r->P, r->q, r->c, &o,
                                                   &r->ws);
    if (ws != TUCKER_OK) return ws;
    {
        // pointer classification makes CUDA calls: keep it off the worker's lock
        r->hostA = !device_ptr(r->A);
        r->hostG = !device_ptr(r->G);
        for (int n = 0; n < r->N; ++n) r->hostU[n] = !device_ptr(r->U[n]);
    }
    r->a_bytes = E * elem;
    r->g_bytes = Gn * elem;
    r->need = up(r->ws) + (r->hostA ? up(r->a_bytes) : 0) + (r->hostG ? up(r->g_bytes) : 0);
    for (int n = 0; n < r->N; ++n) {
        r->u_bytes[n] = (size_t)r->dims[n] * r->ranks[n] * elem;
        if (r->hostU[n]) r->need += up(r->u_bytes[n]);
    }
    if (r->need > srv->budget) return TUCKER_ERR_BUDGET;
    if (srv->tick_max > 1 && r->c == 0 && (int64_t)E <= srv->tick_elems) {
        // the work list takes it alone, so it takes it beside others of its type
        std::vector<Request*> one{r.get()};
        tk::WorklistPlan wp;
        std::vector<tucker_request> t;
        std::vector<size_t> offs;
        size_t area_off = 0;
        void* dU[kMaxN];
        r->tickable = srv->tick_plan(one, &wp, &t, &offs, &area_off, nullptr, dU) > 0;
    }
    std::lock_guard<std::mutex> g(srv->mu);
    r->t_submit = Clock::now();
    if (!srv->any_submit) {
        srv->any_submit = true;
        srv->t_first = r->t_submit;
    }
    r->ticket = srv->reqs.size() + 1;
    *ticket = r->ticket;
    srv->pending.push_back(r.get());
    srv->reqs.push_back(std::move(r));
    srv->cv_work.notify_one();
    return TUCKER_OK;
}

tucker_status tucker_server_wait(tucker_server* srv, uint64_t ticket, int64_t timeout_ms, tucker_status* result) {
    if (!srv || !result) return TUCKER_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (ticket < 1 || ticket > srv->reqs.size()) return TUCKER_ERR_INVALID_ARG;
    Request* r = srv->reqs[ticket - 1].get();
    if (timeout_ms < 0) {
        srv->cv_done.wait(lk, [&] { return r->done; });
    } else if (!r->done) {
        srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; });
    }
    if (!r->done) return TUCKER_ERR_TIMEOUT;
    *result = r->result;
    return TUCKER_OK;
}

tucker_status tucker_server_stats_get(tucker_server* srv, tucker_server_stats* out) {
    if (!srv || !out) return TUCKER_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(srv->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = srv->reqs.size();
    out->completed = srv->lat_ms.size();
    out->failed = srv->failed;
    out->peak_bytes = srv->peak;
    out->peak_inflight = srv->peak_inflight;
    out->ticks = srv->ticks;
    out->tick_requests = srv->tick_requests;
    if (!srv->lat_ms.empty()) {
        std::vector<double> v = srv->lat_ms;
        std::sort(v.begin(), v.end());
        // nearest-rank percentiles
        auto pct = [&](double p) {
            size_t k = (size_t)std::ceil(p / 100.0 * (double)v.size());
            return v[std::min(v.size() - 1, k ? k - 1 : 0)];
        };
        out->p50_ms = pct(50.0);
        out->p99_ms = pct(99.0);
        out->max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_ms = sum / (double)v.size();
        const double span = std::chrono::duration<double>(srv->t_last - srv->t_first).count();
        out->throughput = span > 0 ? (double)v.size() / span : 0.0;
    }
    return TUCKER_OK;
}

tucker_status tucker_server_destroy(tucker_server* srv) {
    if (!srv) return TUCKER_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    srv->worker.join();
    for (Slot& sl : srv->slots) {
        cudaStreamSynchronize(sl.s);
        cudaStreamDestroy(sl.s);
        cudaEventDestroy(sl.ev);
        cudaEventDestroy(sl.ev_alloc);
        cudaEventDestroy(sl.ev_copy);
        cudaEventDestroy(sl.ev_upload);
        cudaFreeHost(sl.h_status);
        if (sl.h_tick_status) cudaFreeHost(sl.h_tick_status);
        if (sl.h_desc) cudaFreeHost(sl.h_desc);
    }
    cudaStreamSynchronize(srv->copy_s);
    cudaStreamDestroy(srv->copy_s);
    cudaMemPoolDestroy(srv->pool);
    delete srv;
    return TUCKER_OK;
}

}  // extern "C"
