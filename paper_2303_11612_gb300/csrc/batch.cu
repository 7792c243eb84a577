// Batched decompositions as one CUDA graph launch. The first call with a given
// batch signature (every request's algorithm, type, shape, ranks, parameters,
// seed and buffer addresses, plus the options and workspace) captures the
// requests' asynchronous launch sequences, each on its own stream forked from an
// origin stream, into one graph and instantiates it; later calls with the same
// signature replay it with a single cudaGraphLaunch. Instantiated graphs are
// kept in a small least-recently-used cache. With TUCKER_FLAG_WORKLIST the
// graph instead holds the batch's work-list steps and grouped
// orthonormalisations (worklist.cu, api.cu: worklist_plan): one launch per step
// for every request together.
#include <cstdio>
#include <cstring>
#include <string>
#include <list>
#include <mutex>
#include <vector>

#include "internal.h"

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kCacheSize = 16;
size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Cached {
    std::vector<unsigned char> sig;
    cudaGraphExec_t exec;
    std::vector<size_t> offsets;       // each request's workspace offset
    int64_t kernels;                   // kernel launches one replay makes
    void* desc = nullptr;              // work-list batches: pinned host image of the descriptors
};

void release(Cached& c) {
    cudaGraphExecDestroy(c.exec);
    if (c.desc) cudaFreeHost(c.desc);
}

std::mutex g_mu;
std::list<Cached> g_cache;             // front = most recently used
std::vector<cudaStream_t> g_side;
cudaStream_t g_origin = nullptr;
cudaEvent_t g_join = nullptr;

bool device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename V> void put(std::vector<unsigned char>& s, const V& v) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    s.insert(s.end(), p, p + sizeof(V));
}

std::vector<unsigned char> signature(int n, const tucker_request* r, const tucker_opts& o) {
    std::vector<unsigned char> s;
    put(s, n);
    put(s, o.form);
    put(s, o.prec);
    put(s, o.workspace);
    put(s, o.workspace_bytes);
    put(s, o.flags & TUCKER_FLAG_WORKLIST);
    for (int k = 0; k < n; ++k) {
        put(s, r[k].which);
        put(s, r[k].dt);
        put(s, r[k].A);
        put(s, r[k].N);
        for (int m = 0; m < r[k].N; ++m) {
            put(s, r[k].dims[m]);
            put(s, r[k].ranks[m]);
            put(s, r[k].U[m]);
        }
        put(s, r[k].P);
        put(s, r[k].q);
        put(s, r[k].c);
        put(s, r[k].prob);
        put(s, r[k].seed);
        put(s, r[k].G);
    }
    return s;
}

// Each request's workspace offset and the total; work-list batches add the
// descriptor area after the requests' slices (at area_off).
tucker_status check(int n, const tucker_request* reqs, const tucker_opts* opts, bool check_ptrs,
                    std::vector<size_t>& offsets, size_t& total, size_t* area_off = nullptr) {
    if (n < 1 || !reqs) return TUCKER_ERR_INVALID_ARG;
    tucker_opts o;
    std::memset(&o, 0, sizeof(o));
    o.struct_size = sizeof(o);
    if (opts) {
        o.form = opts->form;
        o.prec = opts->prec;
    }
    offsets.resize(n);
    total = 0;
    for (int k = 0; k < n; ++k) {
        const tucker_request& r = reqs[k];
        if (r.struct_size < sizeof(tucker_request) || (r.which != 0 && r.which != 1) || !r.A || !r.dims ||
            !r.ranks || !r.U || !r.G || r.N < 1)
            return TUCKER_ERR_INVALID_ARG;
        size_t ws = 0;
        const tucker_status st = tucker_workspace_size(r.which, r.dt, r.dims, r.N, r.ranks, r.P, r.q, r.c, &o, &ws);
        if (st != TUCKER_OK) return st;
        if (check_ptrs) {
            bool dev = device_ptr(r.A) && device_ptr(r.G);
            for (int m = 0; m < r.N && dev; ++m) dev = device_ptr(r.U[m]);
            if (!dev) return TUCKER_ERR_INVALID_ARG;
        }
        offsets[k] = total;
        total += up(ws);
    }
    if (area_off) *area_off = total;
    if (opts && (opts->flags & TUCKER_FLAG_WORKLIST)) {
        tk::WorklistPlan wp;
        const tucker_status st = tk::worklist_plan(n, reqs, *opts, nullptr, offsets, wp);
        if (st != TUCKER_OK) return st;
        total += up(wp.area_bytes);
    }
    return TUCKER_OK;
}

}  // namespace

extern "C" {

tucker_status tucker_batch_workspace_size(int n, const tucker_request* reqs, const tucker_opts* opts, size_t* bytes) {
    if (!bytes) return TUCKER_ERR_INVALID_ARG;
    std::vector<size_t> off;
    size_t total = 0;
    const tucker_status st = check(n, reqs, opts, false, off, total);
    if (st == TUCKER_OK) *bytes = total;
    return st;
}

tucker_status tucker_batch_describe(int n, const tucker_request* reqs, const tucker_opts* opts, char* buf,
                                    size_t len) {
    if (!opts || opts->struct_size < sizeof(tucker_opts) || !(opts->flags & TUCKER_FLAG_WORKLIST) || !buf || len < 1)
        return TUCKER_ERR_INVALID_ARG;
    std::vector<size_t> offsets;
    size_t total = 0;
    tucker_status st = check(n, reqs, opts, false, offsets, total);
    if (st != TUCKER_OK) return st;
    tk::WorklistPlan wp;
    st = tk::worklist_plan(n, reqs, *opts, nullptr, offsets, wp);
    if (st != TUCKER_OK) return st;
    static const char* kNames[] = {"init", "gaussian", "power", "sum", "product"};
    std::string out;
    char line[256];
    for (const tk::WorklistOp& op : wp.ops) {
        if (op.kind == 0) {
            int count[5] = {0, 0, 0, 0, 0};
            int last = -1;
            for (int i = op.a; i < op.b; ++i)
                if (wp.items[i].task != last) {
                    last = wp.items[i].task;
                    ++count[wp.tasks[last].kind];
                }
            snprintf(line, sizeof line, "step %d lane %d: items=%d", op.step, op.lane, op.b - op.a);
            out += line;
            for (int k = 0; k < 5; ++k) {
                snprintf(line, sizeof line, " %s=%d", kNames[k], count[k]);
                out += line;
            }
            snprintf(line, sizeof line, " smem=%zu heavy=%d\n", op.smem, op.heavy);
            out += line;
        } else {
            snprintf(line, sizeof line, "%s lane %d: jobs=%d\n", op.kind == 1 ? "cholqr" : "extract", op.lane,
                     op.b - op.a);
            out += line;
        }
    }
    snprintf(line, sizeof line, "lanes=%d tasks=%zu items=%zu area=%zu\n", wp.lanes, wp.tasks.size(), wp.items.size(),
             wp.area_bytes);
    out += line;
    if (out.size() + 1 > len) return TUCKER_ERR_INVALID_ARG;
    std::memcpy(buf, out.c_str(), out.size() + 1);
    return TUCKER_OK;
}

tucker_status tucker_batch_run(int n, const tucker_request* reqs, const tucker_opts* opts) {
    if (!opts || opts->struct_size < sizeof(tucker_opts) || !opts->workspace) return TUCKER_ERR_INVALID_ARG;
    // the work-list path is planned (tucker_batch_describe) but not run: see the header
    if (opts->flags & TUCKER_FLAG_WORKLIST) return TUCKER_ERR_UNSUPPORTED;
    std::vector<size_t> offsets;
    size_t total = 0, area_off = 0;
    tucker_status st = check(n, reqs, opts, false, offsets, total, &area_off);
    if (st != TUCKER_OK) return st;
    if (opts->workspace_bytes < total) return TUCKER_ERR_INVALID_ARG;
    const bool worklist = (opts->flags & TUCKER_FLAG_WORKLIST) != 0;
    cudaStream_t user = (cudaStream_t)opts->stream;
    const std::vector<unsigned char> sig = signature(n, reqs, *opts);
    std::lock_guard<std::mutex> g(g_mu);
    cudaError_t e = cudaSuccess;
    if (!g_origin) {
        e = cudaStreamCreateWithFlags(&g_origin, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g_join, cudaEventDisableTiming);
        if (e != cudaSuccess) return TUCKER_ERR_CUDA;
    }
    bool replay = true;
    auto hit = g_cache.end();
    for (auto it = g_cache.begin(); it != g_cache.end(); ++it)
        if (it->sig == sig) { hit = it; break; }
    if (hit == g_cache.end()) {
        // addresses are part of the signature: they are checked once, here
        std::vector<size_t> unused;
        size_t t2 = 0;
        if (!device_ptr(opts->workspace)) return TUCKER_ERR_INVALID_ARG;
        st = check(n, reqs, opts, true, unused, t2);
        if (st != TUCKER_OK) return st;
        while ((int)g_side.size() < n) {
            cudaStream_t s2;
            if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess) return TUCKER_ERR_CUDA;
            g_side.push_back(s2);
        }
        std::vector<cudaEvent_t> ev(n + 1, nullptr);
        for (auto& x : ev)
            if (cudaEventCreateWithFlags(&x, cudaEventDisableTiming) != cudaSuccess) {
                x = nullptr;
                for (auto& y : ev)
                    if (y) cudaEventDestroy(y);
                cudaGetLastError();
                return TUCKER_ERR_CUDA;
            }
        cudaGraph_t graph = nullptr;
        Cached c;
        tk::WorklistPlan wp;
        if (worklist) {
            // the descriptors point into this workspace; their host image is pinned
            // (the graph's upload node reads it on every replay)
            st = tk::worklist_plan(n, reqs, *opts, (char*)opts->workspace, offsets, wp);
            if (st == TUCKER_OK && cudaMallocHost(&c.desc, wp.desc_bytes ? wp.desc_bytes : 1) != cudaSuccess) {
                c.desc = nullptr;
                cudaGetLastError();
                st = TUCKER_ERR_OOM;
            }
            if (st != TUCKER_OK) {
                for (auto& x : ev) cudaEventDestroy(x);
                return st;
            }
            tk::worklist_pack(wp, c.desc);
            tk::worklist_prepare(wp);
        }
        const int64_t k0 = tucker_launch_count();
        e = cudaStreamBeginCapture(g_origin, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess && worklist) {
            // lane 0 on the origin stream, the others forked from it after the
            // upload (ev[n]) and joined back through ev[1..]
            std::vector<cudaStream_t> lanes(wp.lanes);
            lanes[0] = g_origin;
            for (int l = 1; l < wp.lanes; ++l) lanes[l] = g_side[l - 1];
            e = tk::worklist_enqueue(wp, (char*)opts->workspace + area_off, c.desc, lanes, ev[n]);
            for (int l = 1; l < wp.lanes && e == cudaSuccess; ++l) {
                e = cudaEventRecord(ev[l - 1], lanes[l]);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(g_origin, ev[l - 1], 0);
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev[n], g_origin);
        for (int k = 0; k < n && !worklist && st == TUCKER_OK && e == cudaSuccess; ++k) {
            const tucker_request& r = reqs[k];
            e = cudaStreamWaitEvent(g_side[k], ev[n], 0);
            if (e != cudaSuccess) break;
            tucker_opts o = *opts;
            o.flags |= TUCKER_FLAG_ASYNC;
            o.stream = g_side[k];
            o.workspace = (char*)opts->workspace + offsets[k];
            o.workspace_bytes = total - offsets[k];
            o.rel_error = nullptr;
            o.sample_idx = nullptr;
            st = r.which ? tucker_rsthosvd(r.A, r.dt, r.dims, r.N, r.ranks, r.P, r.q, r.c, r.prob, r.seed, r.U, r.G, &o)
                         : tucker_rthosvd(r.A, r.dt, r.dims, r.N, r.ranks, r.P, r.q, r.c, r.prob, r.seed, r.U, r.G, &o);
            if (st == TUCKER_OK) e = cudaEventRecord(ev[k], g_side[k]);
            if (e == cudaSuccess && st == TUCKER_OK) e = cudaStreamWaitEvent(g_origin, ev[k], 0);
        }
        const cudaError_t ee = cudaStreamEndCapture(g_origin, &graph);
        if (e == cudaSuccess) e = ee;
        c.offsets = offsets;
        c.sig = sig;
        c.kernels = tucker_launch_count() - k0;   // counted once, for the launch below
        if (e == cudaSuccess && st == TUCKER_OK) e = cudaGraphInstantiate(&c.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        for (auto& x : ev) cudaEventDestroy(x);
        if (st != TUCKER_OK || e != cudaSuccess) {
            if (c.desc) cudaFreeHost(c.desc);
            if (st != TUCKER_OK) return st;
            cudaGetLastError();
            return tk::status_from_cuda(e);          // records the error for tucker_last_cuda_error
        }
        g_cache.push_front(std::move(c));
        if (g_cache.size() > kCacheSize) {
            release(g_cache.back());
            g_cache.pop_back();
        }
        hit = g_cache.begin();
        replay = false;
    } else {
        g_cache.splice(g_cache.begin(), g_cache, hit);
        hit = g_cache.begin();
    }
    // one graph launch (each request's first node zeroes its status word),
    // ordered after the caller's stream and before whatever it enqueues next
    e = cudaEventRecord(g_join, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g_origin, g_join, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(hit->exec, g_origin);
    if (e == cudaSuccess) e = cudaEventRecord(g_join, g_origin);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, g_join, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TUCKER_ERR_CUDA;
    }
    if (replay) tk::note_launches(hit->kernels);
    if (opts->flags & TUCKER_FLAG_ASYNC) return TUCKER_OK;
    if (cudaStreamSynchronize(user) != cudaSuccess) {
        cudaGetLastError();
        return TUCKER_ERR_CUDA;
    }
    for (int k = 0; k < n; ++k) {
        int w = 0;
        if (cudaMemcpy(&w, (char*)opts->workspace + hit->offsets[k], sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return TUCKER_ERR_CUDA;
        if (w & 2) return TUCKER_ERR_TIMEOUT;
        if (w & 1) return TUCKER_ERR_NUMERICAL;
    }
    return TUCKER_OK;
}

}  // extern "C"
