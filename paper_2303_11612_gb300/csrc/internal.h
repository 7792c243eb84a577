// Host-side launchers shared between the translation units of the library.
#pragma once

#include <functional>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace tk {

// Bump allocator over a caller- or library-provided device block. With a null
// base it only measures, which is how the workspace size is computed.
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t used = 0;
    bool ok = true;
    void* take(size_t bytes) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + ((bytes + 255) & ~size_t(255));
        if (!base) return nullptr;
        if (used > cap) { ok = false; return nullptr; }
        return base + off;
    }
};

// ---- sketch (kernels_sketch.cu)
struct PowerPlan {
    int groups, parts, jb, lg;
    size_t smem;
    int64_t tiles;
};
PowerPlan power_plan(const ModeView& v, int L, int elem_size, int num_sms);
size_t power_partials_bytes(const PowerPlan& p, const ModeView& v, int L, int elem_size);

template <typename T>
cudaError_t launch_gaussian(T* out, int64_t rows, int64_t cols, uint64_t seed, uint32_t stream_id,
                            cudaStream_t s);
// X_out = A_(n) (A_(n)^T X_in) (range == false) or Y = A_(n) Omega (range == true).
template <typename T>
cudaError_t launch_power(const T* A, const ModeView& v, const T* X_in, int L, T* X_out,
                         void* partials, const PowerPlan& plan, bool range, uint64_t seed,
                         uint32_t stream_id, cudaStream_t s);

// out[e] = sum_{p < parts} partial[p * count + e], summed in part order.
template <typename T>
cudaError_t launch_reduce_partials(const T* partial, int parts, int64_t count, T* out, cudaStream_t s);

// ---- tensor-core power step, bf16 operands / fp32 accumulation (kernels_tc.cu)
bool power_tc_supported(const ModeView& v, int L);
size_t power_tc_partials_bytes(const ModeView& v, int L, int num_sms);
cudaError_t launch_power_tc(const float* A, const ModeView& v, const float* X_in, int L, float* X_out, void* partials,
                            int* status, int num_sms, cudaStream_t s);

// ---- tensor-core power step, tf32 operands / fp32 accumulation, contiguous
// fibers (kernels_tf32.cu). Returns cudaErrorNotSupported (nothing launched)
// when the shape is outside power_tf32_supported or A is not 16-byte aligned;
// partials as for launch_power_tc.
bool power_tf32_supported(const ModeView& v, int L);
cudaError_t launch_power_tf32(const float* A, const ModeView& v, const float* X_in, int L, float* X_out,
                              void* partials, int* status, int num_sms, cudaStream_t s);

// ---- tensor-core power step, single-pass bf16 operands / fp32 accumulation,
// contiguous fibers (kernels_bf16x1.cu); contract as launch_power_tf32.
bool power_bf16x1_supported(const ModeView& v, int L);
cudaError_t launch_power_bf16x1(const float* A, const ModeView& v, const float* X_in, int L, float* X_out,
                                void* partials, int* status, int num_sms, cudaStream_t s);

// ---- mode-n product on the tensor cores, split-bf16 operands / fp32
// accumulation, contiguous fibers (kernels_ttm_tc.cu); M(i, o) = Mp[i ld_i + o ld_k],
// out as launch_ttm. Returns cudaErrorNotSupported (nothing launched) outside
// ttm_tc_supported or when A is not 16-byte aligned.
bool ttm_tc_supported(const ModeView& v, int64_t K_out);
cudaError_t launch_ttm_tc(const float* A, const ModeView& v, const float* Mp, int64_t K_out, int64_t ld_i,
                          int64_t ld_k, float* out, int* status, int num_sms, cudaStream_t s);

// ---- tensor-core passes for contiguous fibers at large shapes (kernels_wide.cu):
// I_n % 4 == 0, columns (L or K_out) <= 128. Return cudaErrorNotSupported (nothing
// launched) outside wide_supported or when A is not 16-byte aligned.
bool wide_supported(const ModeView& v, int64_t cols);          // power step (both passes)
bool wide_ttm_supported(const ModeView& v, int64_t K_out);      // mode product
size_t wide_ttm_scratch_bytes(const ModeView& v, int64_t K_out);
size_t wide_power_scratch_bytes(const ModeView& v, int L, int num_sms);
// out = A x_n M (split bf16, FP32 accumulate), out[j K_out + o] as launch_ttm.
// FP32 ring depth of the wide kernels: kWideStagesShared (3) keeps a wide CTA's
// shared memory small enough that another decomposition's extraction CTA fits
// on the same SM (batches and served requests run many decompositions at
// once); a call that runs alone takes as many stages as shared memory holds.
constexpr int kWideStagesShared = 3;
constexpr int kWideStagesAlone = 6;
cudaError_t launch_ttm_wide(const float* A, const ModeView& v, const float* Mp, int64_t K_out, int64_t ld_i,
                            int64_t ld_k, float* out, void* scratch, int* status, int num_sms, cudaStream_t s,
                            int max_stages = kWideStagesAlone);
// X_out = A_(n) (A_(n)^T X_in) in two passes (range == false), or Y = A_(n) Omega
// with Omega J_n x L from the Philox stream (range == true, X_in unused); split:
// split-bf16 operands, else single-pass bf16.
cudaError_t launch_power_wide(const float* A, const ModeView& v, const float* X_in, int L, float* X_out, bool split,
                              bool range, uint64_t seed, uint32_t stream_id, void* scratch, int* status, int num_sms,
                              cudaStream_t s, int max_stages = kWideStagesAlone);

// Strategy B: G = A_(n) A_(n)^T (I_n x I_n, column-major, I_n <= 128) in one tensor-core pass;
// scratch of gram_wide_scratch_bytes (per-CTA partials, summed in a fixed order).
bool gram_wide_supported(const ModeView& v);
size_t gram_wide_scratch_bytes(const ModeView& v, int num_sms);
cudaError_t launch_gram_wide(const float* A, const ModeView& v, float* G, bool split, void* scratch, int* status,
                             int num_sms, cudaStream_t s, int max_stages = kWideStagesAlone);

// half steps of the AMM sketch on the tensor cores (split bf16), scratch as launch_power_wide:
// Y (J x L, column-major) = A_(n)^T X, and X_out = A_(n) Q with Q J x L column-major
cudaError_t launch_wide_tn(const float* A, const ModeView& v, const float* X, int L, float* Y, void* scratch,
                           int* status, int num_sms, cudaStream_t s, int max_stages = kWideStagesAlone);
cudaError_t launch_wide_nn(const float* A, const ModeView& v, const float* Q, int L, float* X_out, void* scratch,
                           int* status, int num_sms, cudaStream_t s, int max_stages = kWideStagesAlone);

// ---- half steps of the power scheme on the gathered AMM sample (kernels_half.cu)
bool half_supported(int L);
size_t half_partials_bytes(int64_t I, int L, int64_t Tn, int num_sms, int elem_size);
// Y (Tn x L) = M^T X with M I x Tn, X I x L (all column-major).
template <typename T>
cudaError_t launch_gemm_tn(const T* M, int64_t I, int64_t Tn, const T* X, int L, T* Y, cudaStream_t s);
// X (I x L) = M Q with Q Tn x L, split over Tn (partials of half_partials_bytes).
template <typename T>
cudaError_t launch_gemm_nn(const T* M, int64_t I, int64_t Tn, const T* Q, int L, T* X, void* partials, int num_sms,
                           cudaStream_t s);

// Sign rule on U's columns (largest-magnitude entry positive, lowest row on ties).
template <typename T>
cudaError_t launch_sign_fix(T* U, int64_t I, int R, cudaStream_t s);

// ---- sampling (kernels_amm.cu)
template <typename T>
cudaError_t launch_fiber_norms(const T* A, const ModeView& v, double* w, cudaStream_t s);
// Mode-1 and mode-2 fiber norms in one pass over the tensor read as I1 x I2 x rest:
// w1[i2 + I2 r] (the mode-1 fibers' order), w2[i1 + I1 r] (the mode-2 fibers'); I1 <= 1024.
bool fiber_norms12_supported(int64_t I1);
// Order-3 tensors: all three modes' fiber norms from one pass (norms123_kernel),
// through partials in scratch (fiber_norms123_scratch_bytes), summed in order.
bool fiber_norms123_supported(int64_t I1);
size_t fiber_norms123_scratch_bytes(int64_t I1, int64_t I2, int64_t I3);
template <typename T>
cudaError_t launch_fiber_norms123(const T* A, int64_t I1, int64_t I2, int64_t I3, double* w1, double* w2,
                                  double* w3, void* scratch, cudaStream_t s);
template <typename T>
cudaError_t launch_fiber_norms12(const T* A, int64_t I1, int64_t I2, int64_t rest, double* w1, double* w2,
                                 cudaStream_t s);
size_t quantize_scratch_bytes(int64_t J);
cudaError_t launch_quantize(const double* w, int64_t J, int prob, uint64_t* W, void* scratch,
                            cudaStream_t s);
size_t sample_scratch_bytes(int64_t J);
cudaError_t launch_sample(const uint64_t* W, int64_t J, int64_t T, uint64_t seed, uint32_t stream_id,
                          int64_t* idx, double* scale, void* scratch, cudaStream_t s);
template <typename T>
cudaError_t launch_gather(const T* A, const ModeView& v, const int64_t* idx, const double* scale,
                          int64_t T_, T* Cp, cudaStream_t s);
// sharded calls: quantisation against a given maximum, and one slab's draws
cudaError_t launch_quantize_max(const double* w, int64_t J, double wmax, uint64_t* W, cudaStream_t s);
cudaError_t launch_sample_slab(const uint64_t* W, int64_t J, int64_t T_, uint64_t seed, uint32_t stream_id,
                               uint64_t S_offset, uint64_t S_total, int64_t fiber_offset, int64_t* idx, double* scale,
                               void* scratch, cudaStream_t s);

// ---- orthonormalisation and extraction (kernels_orth.cu)
struct OrthPlan {
    int64_t I;
    int L;
    int gram_blocks;
};
OrthPlan orth_plan(int64_t I, int L, int num_sms);
size_t orth_scratch_bytes(const OrthPlan& p, int elem_size);
// True when the extraction of R columns fits the shared-memory limits.
bool orth_supported(const OrthPlan& p, int R, int elem_size);
// One CholeskyQR pass: X (I x L) = Q F, F upper triangular (packed rows in the
// first L(L+1)/2 of the L^2 doubles at `factor`: a double-float pair per entry
// for FP32 data, FP64 for FP64 data), Q = X F^-1. X and Q may not alias.
template <typename T>
cudaError_t launch_cholqr(const T* X, T* Q, const OrthPlan& p, double* factor, void* scratch, int* status,
                          cudaStream_t s);
// U (I x R) = the R leading left singular vectors of C = X P, P = factors[nprev-1]
// ... factors[0] (factors of earlier steps, in L^2-double slots as written by
// launch_cholqr; nprev may be 0), sign-fixed. Q1 (I x L) is scratch; factors must have room for nprev + 1
// factors (the extraction stores its own CholeskyQR factor after them).
template <typename T>
cudaError_t launch_extract(const T* X, T* Q1, const OrthPlan& p, double* factors, int nprev, int R, T* U,
                           void* scratch, int* status, cudaStream_t s);

// Grouped orthonormalisations (a batch's requests side by side in one launch,
// job = blockIdx.y): the same block programs and results as launch_cholqr /
// launch_extract of each job alone.
struct OrthJob {
    const void* X;          // I x L sketch
    void* Q;                // I x L: the CholeskyQR output (cholqr), the extraction's Q1 (extract)
    int64_t I;
    int L, R;               // R: columns extracted
    int rows, nblk;         // Gram rows per CTA, Gram CTAs (the plan's)
    int nprev;              // extraction: earlier factors in the slots from `factor` on
    int staged;             // extraction: the final pass keeps U in shared memory (orth_group_staged)
    void* partial;          // orthonormalisation scratch (orth_job)
    int* flag;
    unsigned* ticket;
    void* W;
    double* factor;         // cholqr: the factor slot; extract: the first factor slot
    int64_t fofs;           // doubles from `factor` to the slot this CholeskyQR pass writes (extract: nprev L^2)
    void* U;                // extraction output, I x R
    int* status;
};
// A job with the plan's sizes and the scratch regions filled in.
OrthJob orth_job(const OrthPlan& p, void* scratch);
bool orth_group_staged(const OrthJob& j, int elem_size);
// d_jobs: the jobs in device memory; h_jobs: the same on the host (sizes of the launches).
template <typename T>
cudaError_t launch_cholqr_group(const OrthJob* d_jobs, const std::vector<OrthJob>& h_jobs, cudaStream_t s);
template <typename T>
cudaError_t launch_extract_group(const OrthJob* d_jobs, const std::vector<OrthJob>& h_jobs, cudaStream_t s);

// ---- work-list kernel of batched runs (worklist.cu)
enum WKind : int { kWInit = 0, kWGen = 1, kWPow = 2, kWRed = 3, kWTtm = 4 };
// One stage of one request's mode; its items are the blocks the stage's own
// kernel would launch.
struct WTask {
    int kind;               // WKind
    int nitems;             // items of this task
    int dep[2];             // tasks whose output it reads (-1: none): always in an earlier phase of its lane
    int* status;            // the request's status word
    const void* in;         // kWPow, kWTtm: the tensor; kWRed: the partials
    const void* X;          // kWPow: X_in (I x L); kWTtm: the factor U (I x K)
    void* out;              // kWGen: Omega; kWPow: the partials; kWRed: X_out; kWTtm: the product
    ModeView v;             // kWPow, kWTtm
    int64_t tiles;          // kWPow: fiber tiles of jb fibers
    int64_t count;          // kWRed: I L
    int64_t K;              // kWTtm: outputs per fiber (R_n)
    int64_t rows, cols;     // kWGen
    uint64_t seed;
    uint32_t sid;
    int L, parts, jb, lg, opt;
};
// kWPow: x = column group, y = part; kWTtm: (x, y) = the product kernel's block;
// kWGen, kWRed: x = block of the task's nitems.
struct WItem {
    int task, x, y, pad;
};
// Shared memory of a power-step item (jb fixed by the type: 32 FP32, 16 FP64), of
// a mode-product item; the outputs-per-thread choice of a mode product with K
// outputs (0 when K > 32, which the work list does not take).
size_t worklist_pow_smem(int elem, int I, int lg);
size_t worklist_ttm_smem(int elem, int opt);
// Whether a task needs the kernel's heavy register class (column groups of 32, more than 16 outputs per block).
bool worklist_heavy(const WTask& t);
int worklist_ttm_opt(int64_t K);
// The grid of a step with `items` items and `smem` bytes of dynamic shared
// memory (the SMs times the CTAs that fit on one, at most one CTA per item);
// also raises the kernel's shared-memory limit. Not for use under stream capture.
int worklist_grid(int elem, bool heavy, size_t smem, int items);
// Items [begin, end) of one phase (independent of one another); the claim word
// zeroed before the launch.
template <typename T>
cudaError_t launch_worklist(const WTask* tasks, const WItem* items, int begin, int end, unsigned* claim, bool heavy,
                            size_t smem, int grid, cudaStream_t s);

// A batch as work-list steps and grouped orthonormalisations (api.cu).
struct WorklistOp {
    int kind;               // 0: work-list step over items [a, b); 1: CholeskyQR of jobs [a, b); 2: extraction of jobs [a, b)
    int a, b;
    int step;               // kind 0: the step's claim word
    size_t smem;            // kind 0: dynamic shared memory
    int grid = 0;           // kind 0: CTAs (worklist_prepare)
    int heavy = 0;          // kind 0: a task needs the heavy register class
    int lane = 0;           // the stream of the batch's graph it runs on
};
struct WorklistPlan {
    int elem = 4;
    std::vector<WTask> tasks;
    std::vector<WItem> items;
    std::vector<OrthJob> jobs;
    std::vector<WorklistOp> ops;
    int steps = 0;
    int lanes = 1;          // requests k with k % lanes == l run their steps on stream l
    // device area: tasks, items and jobs (uploaded from the host image), then the
    // claim words (one per phase)
    size_t tasks_off = 0, items_off = 0, jobs_off = 0, desc_bytes = 0;
    size_t counters_off = 0, counter_bytes = 0, area_bytes = 0;
};
// The plan of n requests whose workspace slices start at ws + offsets[k] (ws may be
// null: sizes only). TUCKER_ERR_UNSUPPORTED unless every request is Algorithm 1 or 2
// in the paper form with the exact FMA arithmetic, no sampling, one element type,
// every extent <= 256 and every rank <= 32.
tucker_status worklist_plan(int n, const tucker_request* reqs, const tucker_opts& opts, char* ws,
                            const std::vector<size_t>& offsets, WorklistPlan& wp, int max_lanes = 8);
// Fills each step's grid (queries the device: call before stream capture).
void worklist_prepare(WorklistPlan& wp);
// The host image of the descriptors (wp.desc_bytes bytes at host).
void worklist_pack(const WorklistPlan& wp, void* host);
// Uploads the image to area (wp.area_bytes of device memory) and zeroes the
// counters on lane_streams[0], then enqueues each lane's steps and grouped
// launches on its stream (lane l on lane_streams[l], ordered after the upload;
// the caller joins the lanes).
cudaError_t worklist_enqueue(const WorklistPlan& wp, char* area, const void* host_desc,
                             const std::vector<cudaStream_t>& lane_streams, cudaEvent_t uploaded);

// ---- mode products and norms (kernels_ttm.cu)
// out = A x_n M: M(k_out, i) read as Mp[i * ld_i + k_out * ld_k]. With a
// device status word (FP32) the TMA-fed kernel is used where the shape allows;
// a bounded wait that times out sets kStatTimeout there.
template <typename T>
cudaError_t launch_ttm(const T* A, const ModeView& v, const T* Mp, int64_t K_out, int64_t ld_i,
                       int64_t ld_k, T* out, cudaStream_t s, int* status = nullptr);
size_t sumsq_scratch_bytes();
// One CTA whose bounded wait on an mbarrier nothing completes runs out after
// `iters` polls: sets kStatTimeout in *status, frees its tensor memory, returns.
cudaError_t launch_wait_timeout(int iters, int* status, cudaStream_t s);
// Energies e_k = ||Y(slice k of mode n)||^2 (Y viewed through v with v.i = K slices).
size_t slice_sumsq_scratch_bytes(const ModeView& v, int num_sms);
template <typename T>
cudaError_t launch_slice_sumsq(const T* Y, const ModeView& v, double* e, void* scratch, int num_sms,
                               cudaStream_t s);
// *out (device double) = sum (a - b)^2 (b may be null).
template <typename T>
cudaError_t launch_sumsq(const T* a, const T* b, int64_t n, double* out, void* scratch,
                         cudaStream_t s);

int num_sms();

// The status a CUDA error maps to; records the error for tucker_last_cuda_error.
tucker_status status_from_cuda(cudaError_t e);

// ---- launch counting and profiling (profile.cu)
enum KernelClass { kKPower = 0, kKTtm = 1, kKGather = 2, kKNorms = 3, kKExtract = 4, kKSample = 5,
                   kKPowerBf16 = 6, kKPowerTf32 = 7, kKTtmBf16 = 8, kKPowerBf16x1 = 9, kKTtmWide = 10,
                   kKPowerWide1 = 11, kKPowerWide2 = 12, kKRangeWide = 13,
                   kKGramWide = 14, kKWorklist = 15, kKernelClasses = 16 };
void note_launch();
void note_launches(int64_t n);   // a graph replay's kernels
void profile_drain();
// Brackets one launch with CUDA events when profiling is on.
class ProfScope {
  public:
    ProfScope(int cls, double bytes, double flops, cudaStream_t s);
    ~ProfScope();
  private:
    int cls_;
    double bytes_, flops_;
    cudaStream_t s_;
    void* a_ = nullptr;
    void* b_ = nullptr;
};

// ---- autotuner (autotune.cu)
enum TuneSite : int { kTuneTtm = 0, kTunePower = 1 };
struct TuneKey {
    int site;
    int64_t k[4];
};
bool operator<(const TuneKey& a, const TuneKey& b);
// Marks the calling thread as inside a synchronous library call (tuning may
// synchronise its stream) for the object's lifetime.
class TuneAllow {
public:
    explicit TuneAllow(bool allow);
    ~TuneAllow();
    TuneAllow(const TuneAllow&) = delete;
    TuneAllow& operator=(const TuneAllow&) = delete;
private:
    bool on_;
};
bool tune_active(cudaStream_t s);
int tune_get(const TuneKey& k);            // the kept choice, or -1
// Times every candidate (warm-up + one timed launch), keeps and returns the fastest.
int tune_pick(cudaStream_t s, const TuneKey& key, const char* what, const std::vector<std::string>& names,
              const std::function<cudaError_t(int)>& launch_candidate, int fallback);

}  // namespace tk

