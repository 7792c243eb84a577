// C ABI of the library: argument checks, workspace planning, host/device
// staging and the per-mode orchestration of Algorithms 1, 2, 4 and 5.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace tk {

int num_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    return n;
}

namespace {

constexpr int kMaxOrder = 8;
constexpr int64_t kMaxI = 1024;      // power-step register tiling (4 rows per thread)
constexpr int kMaxL = 110;           // packed L x L factors of the extraction in shared memory

thread_local cudaStream_t g_async_stream = nullptr;
thread_local int* g_async_status = nullptr;

thread_local cudaError_t g_last_cuda_error = cudaSuccess;

tucker_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return TUCKER_OK;
    g_last_cuda_error = e;
    if (e == cudaErrorMemoryAllocation) return TUCKER_ERR_OOM;
    return TUCKER_ERR_CUDA;
}

bool on_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

ModeView view_of(const int64_t* dims, int N, int n) {
    ModeView v{1, dims[n], 1};
    for (int m = 0; m < n; ++m) v.lf *= dims[m];
    for (int m = n + 1; m < N; ++m) v.rt *= dims[m];
    return v;
}

int64_t prod(const int64_t* d, int N) {
    int64_t p = 1;
    for (int k = 0; k < N; ++k) p *= d[k];
    return p;
}

uint32_t stream_id(int purpose, int mode) { return ((uint32_t)purpose << 8) | (uint32_t)(mode & 0xFF); }

struct Opts {
    int form = TUCKER_FORM_PAPER;
    int prec = TUCKER_SK_FP32;
    uint32_t flags = 0;
    double alpha = 0.0;
    cudaStream_t stream = nullptr;
    void* workspace = nullptr;
    size_t workspace_bytes = 0;
    double* rel_error = nullptr;
    int64_t* const* sample_idx = nullptr;
};

tucker_status read_opts(const tucker_opts* o, Opts& out) {
    if (!o) return TUCKER_OK;
    if (o->struct_size < sizeof(tucker_opts)) return TUCKER_ERR_INVALID_ARG;
    out.form = o->form;
    out.prec = o->prec;
    out.flags = o->flags;
    out.alpha = o->alpha;
    out.stream = reinterpret_cast<cudaStream_t>(o->stream);
    out.workspace = o->workspace;
    out.workspace_bytes = o->workspace_bytes;
    out.rel_error = o->rel_error;
    out.sample_idx = o->sample_idx;
    if (out.form != TUCKER_FORM_PAPER && out.form != TUCKER_FORM_RANGE && out.form != TUCKER_FORM_RELATED)
        return TUCKER_ERR_INVALID_ARG;
    if (out.prec < TUCKER_SK_FP32 || out.prec > TUCKER_SK_BF16X1) return TUCKER_ERR_INVALID_ARG;
    if (!(out.alpha >= 0.0) || out.alpha > 1.0) return TUCKER_ERR_INVALID_ARG;
    return TUCKER_OK;
}

int64_t sample_count(int64_t c, double alpha, int64_t J) {
    if (c > 0) return std::min(c, J);
    if (alpha > 0.0) {
        double t = alpha * (double)J;
        int64_t T = (int64_t)t;
        if ((double)T < t) ++T;
        return std::min(T, J);
    }
    return 0;
}

// ------------------------------------------------------------------ plan
struct ModePlan {
    ModeView v;        // view of the tensor the mode works on
    ModeView mv;       // view of the matrix that is sketched (v, or the I x T gather)
    int L;
    int R;
    int64_t T;         // AMM samples (0 = none)
    bool tc;           // power steps on the tensor cores (split-bf16 operands)
    bool tf32;         // power steps on the tensor cores (tf32 operands, contiguous fibers)
    bool bf16x1;       // power steps on the tensor cores (single-pass bf16 operands, contiguous fibers)
    bool wide;         // power steps as two tensor-core passes (contiguous fibers beyond the fused tiles)
    bool wide_split;   //   with split-bf16 operands (else single-pass bf16)
    bool wide_range;   // range form: first pass Y = A Omega on the tensor cores, Omega generated in-kernel
    bool half;         // AMM, paper form: power steps on C' as two orthonormalised half steps
    bool half_tc;      //   on the tensor cores (split bf16; the tensor-core forms, large samples)
    bool gram;         // Strategy B: G = B_(n) B_(n)^T in one tensor-core pass, then G^q Omega
    OrthPlan opT;      //   orthonormalisation of the T x L half-step product
    OrthPlan opL;      // related form: extraction from the L x L matrix P^T A A^T P
    PowerPlan pp;
    OrthPlan op;
};

struct Plan {
    int N = 0;
    int prec = TUCKER_SK_FP32;
    bool st = false;
    int elem = 4;
    int form = 0;
    int q = 1;
    int64_t dims[kMaxOrder];
    int64_t cur[kMaxOrder][kMaxOrder];   // dims of the tensor each mode works on (ST shrinks)
    ModePlan m[kMaxOrder];
    int64_t maxI = 0, maxL = 0, maxJ = 0, maxT = 0, maxIT = 0, maxTL = 0, maxGram = 0;
    bool half = false;
    size_t max_partials = 0, max_orth = 0;
    int64_t inter_elems = 0;             // largest intermediate tensor of the TTM chain
};

// The plan of mode n of the tensor d (rank R, oversampling P, c samples): fills
// p.m[n] and raises the plan's buffer maxima.
tucker_status plan_mode(Plan& p, const int64_t* d, int N, int n, int64_t R, int32_t P, int64_t c, bool st, int elem,
                        const Opts& o, int sms) {
    ModePlan& mp = p.m[n];
    mp.v = view_of(d, N, n);
    mp.R = R;
    mp.L = (int)std::min<int64_t>((int64_t)R + P, d[n]);
    const int64_t J = mp.v.fibers();
    mp.T = sample_count(c, o.alpha, J);
    mp.mv = mp.T > 0 ? ModeView{1, d[n], mp.T} : mp.v;
    if (d[n] > kMaxI || mp.L > kMaxL) return TUCKER_ERR_UNSUPPORTED;
    if (elem == 8 && d[n] > 512) return TUCKER_ERR_UNSUPPORTED;
    mp.pp = power_plan(mp.mv, mp.L, elem, sms);
    // tensor-core power steps where the tile fits: TF32 on contiguous fibers, split
    // BF16 (also the TF32 form's choice for strided fibers); the FP32 kernel elsewhere.
    // Single-pass BF16 sketches the input tensor only (every mode of T-HOSVD, the
    // first of ST-HOSVD): ST-HOSVD's later modes see the truncated tensor, small by
    // then, where the split form's accuracy costs little.
    mp.tf32 = o.prec == TUCKER_SK_TF32 && elem == 4 && power_tf32_supported(mp.mv, mp.L);
    mp.bf16x1 = o.prec == TUCKER_SK_BF16X1 && elem == 4 && (!st || n == 0) &&
                power_bf16x1_supported(mp.mv, mp.L);
    // beyond the fused kernels' tiles (I_n > 512 or wide sketches; contiguous fibers, the
    // gathered AMM sample, or strides that are multiples of 32): two tensor-core passes,
    // single-pass bf16 where the form sketches in single-pass BF16 (preferred there over
    // the fused split kernel), split bf16 elsewhere
    mp.wide_split = !(o.prec == TUCKER_SK_BF16X1 && (!st || n == 0));
    mp.wide = o.prec != TUCKER_SK_FP32 && elem == 4 && !mp.tf32 && !mp.bf16x1 &&
              wide_supported(mp.mv, mp.L) && (!mp.wide_split || !power_tc_supported(mp.mv, mp.L));
    mp.tc = o.prec != TUCKER_SK_FP32 && elem == 4 && !mp.wide && power_tc_supported(mp.mv, mp.L);
    if (mp.tc || mp.tf32 || mp.bf16x1)
        p.max_partials = std::max(p.max_partials, power_tc_partials_bytes(mp.mv, mp.L, sms));
    mp.wide_range = o.form == TUCKER_FORM_RANGE && o.prec != TUCKER_SK_FP32 && elem == 4 &&
                    wide_supported(mp.mv, mp.L);
    if (mp.wide || mp.wide_range)
        p.max_partials = std::max(p.max_partials, wide_power_scratch_bytes(mp.mv, mp.L, sms));
    if (o.prec != TUCKER_SK_FP32 && elem == 4 && st && !ttm_tc_supported(mp.v, mp.R) &&
        wide_ttm_supported(mp.v, mp.R))
        p.max_partials = std::max(p.max_partials, wide_ttm_scratch_bytes(mp.v, mp.R));
    mp.op = orth_plan(d[n], mp.L, sms);
    if (!orth_supported(mp.op, mp.R, elem)) return TUCKER_ERR_UNSUPPORTED;
    // AMM in the paper form: C_n = (C' C'^T)^q Omega evaluated in half steps (Y = C'^T Q,
    // Y = Q_Y R_Y, X = C' Q_Y), every stored product orthonormalised, so that FP32 keeps
    // the sample's directions down to sigma_i / sigma_1 ~ 2^-24 rather than 2^-12
    if (o.form == TUCKER_FORM_RELATED) {
        // Algorithms 6/7: defined without AMM; the leading vectors of P^T A_(n) come from
        // the L x L matrix P^T A A^T P, and Q_n = P U is an I x L by L x R product
        if (mp.T > 0 || !half_supported(mp.L)) return TUCKER_ERR_UNSUPPORTED;
        mp.opL = orth_plan(mp.L, mp.L, sms);
        if (!orth_supported(mp.opL, mp.R, elem)) return TUCKER_ERR_UNSUPPORTED;
        p.max_orth = std::max(p.max_orth, orth_scratch_bytes(mp.opL, elem));
        p.max_partials = std::max(p.max_partials, half_partials_bytes(d[n], mp.R, mp.L, sms, elem));
    }
    mp.half = mp.T > 0 && o.form == TUCKER_FORM_PAPER && mp.T >= mp.L && half_supported(mp.L);
    // the tensor-core forms run the half steps of large samples (beyond the fused
    // kernels' tiles) on the tensor cores in split bf16, FP32-class like the FMA form
    mp.half_tc = mp.half && o.prec != TUCKER_SK_FP32 && elem == 4 && wide_supported(mp.mv, mp.L) &&
                 !power_tc_supported(mp.mv, mp.L);
    if (mp.half_tc) p.max_partials = std::max(p.max_partials, wide_power_scratch_bytes(mp.mv, mp.L, sms));
    // Strategy B (remark after Algorithm 1) where it saves passes over the tensor: with q >= 2
    // power steps and I_n <= 128, G = B_(n) B_(n)^T in one tensor-core pass (split bf16, FP32
    // accumulation) and C_n = G^q Omega_n on the I_n x I_n matrix, where Strategy A reads the
    // tensor q times; the same C_n, in the same factored form
    mp.gram = o.form == TUCKER_FORM_PAPER && mp.T == 0 && p.q >= 2 && o.prec != TUCKER_SK_FP32 && elem == 4 &&
              gram_wide_supported(mp.v);
    if (mp.gram) {
        p.maxGram = std::max(p.maxGram, d[n] * d[n]);
        p.max_partials = std::max(p.max_partials, gram_wide_scratch_bytes(mp.v, sms));
        p.max_partials = std::max(p.max_partials, half_partials_bytes(d[n], mp.L, d[n], sms, elem));
    }
    if (mp.half) {
        mp.opT = orth_plan(mp.T, mp.L, sms);
        p.half = true;
        p.maxTL = std::max(p.maxTL, mp.T * (int64_t)mp.L);
        p.max_orth = std::max(p.max_orth, orth_scratch_bytes(mp.opT, elem));
        p.max_partials = std::max(p.max_partials, half_partials_bytes(d[n], mp.L, mp.T, sms, elem));
    }
    p.maxI = std::max(p.maxI, d[n]);
    p.maxL = std::max<int64_t>(p.maxL, mp.L);
    p.maxJ = std::max(p.maxJ, J);
    p.maxT = std::max(p.maxT, mp.T);
    p.maxIT = std::max(p.maxIT, d[n] * mp.T);
    p.max_partials = std::max(p.max_partials, power_partials_bytes(mp.pp, mp.mv, mp.L, elem));
    p.max_orth = std::max(p.max_orth, orth_scratch_bytes(mp.op, elem));
    return TUCKER_OK;
}

tucker_status make_plan(bool st, int elem, const int64_t* dims, int N, const int32_t* ranks, int32_t P, int32_t q,
                        int64_t c, const Opts& o, Plan& p) {
    if (N < 1 || N > kMaxOrder || !dims || !ranks) return TUCKER_ERR_INVALID_ARG;
    if (q < 1 || P < 0 || c < 0) return TUCKER_ERR_INVALID_ARG;
    for (int n = 0; n < N; ++n) {
        if (dims[n] < 1 || ranks[n] < 1 || ranks[n] > dims[n]) return TUCKER_ERR_INVALID_ARG;
    }
    p.N = N;
    p.st = st;
    p.elem = elem;
    p.form = o.form;
    p.prec = o.prec;
    p.q = q;
    const int sms = num_sms();
    int64_t d[kMaxOrder];
    for (int n = 0; n < N; ++n) d[n] = p.dims[n] = dims[n];
    for (int n = 0; n < N; ++n) {
        for (int k = 0; k < N; ++k) p.cur[n][k] = d[k];
        const tucker_status ms = plan_mode(p, d, N, n, ranks[n], P, c, st, elem, o, sms);
        if (ms != TUCKER_OK) return ms;
        if (st) d[n] = ranks[n];
        if (st && n < N - 1) p.inter_elems = std::max(p.inter_elems, prod(d, N));
    }
    if (!st) {
        int64_t e[kMaxOrder];
        for (int n = 0; n < N; ++n) e[n] = dims[n];
        for (int n = 0; n < N; ++n) {
            const ModeView tv = view_of(e, N, n);
            if (o.prec != TUCKER_SK_FP32 && elem == 4 && !ttm_tc_supported(tv, ranks[n]) &&
                wide_ttm_supported(tv, ranks[n]))
                p.max_partials = std::max(p.max_partials, wide_ttm_scratch_bytes(tv, ranks[n]));
            if (n == N - 1) break;
            e[n] = ranks[n];
            p.inter_elems = std::max(p.inter_elems, prod(e, N));
        }
    }
    return TUCKER_OK;
}

struct Work {
    int* status;
    void* X0; void* X1; void* Q; void* Qt;
    double* factors;
    void* partials;
    void* orth;
    double* w; uint64_t* W; void* samp; int64_t* idx; double* scale; void* Cp;
    double* w2;            // T-HOSVD with sampling: mode 2's fiber norms, formed beside mode 1's
    double* w3;            // order 3: mode 3's, with the partials of the pass that forms all three
    void* nscr;
    void* inter[2];
    void* Y; void* QY;     // half steps: T x L product and its orthonormal factor
    void* Gn;              // Strategy B: the I_n x I_n Gram matrix (FP32)
    void* sumsq;
    double* norms;     // [2]: ||A||^2, ||G||^2
    int wide_stages = kWideStagesAlone;   // FP32 ring depth of the wide tensor-core kernels
};

void carve(const Plan& p, Arena& a, Work& w) {
    const size_t IL = (size_t)p.maxI * p.maxL * p.elem;
    // factor slots: paper form q (2q with half steps: one per half step and per step), range form 1
    // related form: q for the power steps, 2 for P's CholeskyQR2, 1 for the extraction from H
    const int slots = p.form == TUCKER_FORM_PAPER     ? (p.half ? 2 * p.q : p.q)
                      : p.form == TUCKER_FORM_RELATED ? p.q + 3
                                                      : 1;
    w.status = (int*)a.take(sizeof(int) * 64);
    w.X0 = a.take(IL);
    w.X1 = a.take(IL);
    w.Q = a.take(IL);
    w.Qt = a.take(IL);
    w.factors = (double*)a.take(sizeof(double) * slots * (size_t)p.maxL * p.maxL);
    w.partials = a.take(p.max_partials);
    w.orth = a.take(p.max_orth);
    if (p.maxT > 0) {
        w.w = (double*)a.take(sizeof(double) * (size_t)p.maxJ);
        w.W = (uint64_t*)a.take(sizeof(uint64_t) * (size_t)p.maxJ);
        w.samp = a.take(std::max(sample_scratch_bytes(p.maxJ), quantize_scratch_bytes(p.maxJ)));
        w.idx = (int64_t*)a.take(sizeof(int64_t) * (size_t)p.maxT);
        w.scale = (double*)a.take(sizeof(double) * (size_t)p.maxT);
        w.Cp = a.take((size_t)p.maxIT * p.elem);
        w.w2 = p.st ? nullptr : (double*)a.take(sizeof(double) * (size_t)p.maxJ);
        const bool all3 = !p.st && p.N == 3 && fiber_norms123_supported(p.dims[0]);
        w.w3 = all3 ? (double*)a.take(sizeof(double) * (size_t)p.maxJ) : nullptr;
        w.nscr = all3 ? a.take(fiber_norms123_scratch_bytes(p.dims[0], p.dims[1], p.dims[2])) : nullptr;
    } else {
        w.w = nullptr; w.W = nullptr; w.samp = nullptr; w.idx = nullptr; w.scale = nullptr; w.Cp = nullptr;
        w.w2 = nullptr;
        w.w3 = nullptr;
        w.nscr = nullptr;
    }
    w.Y = p.maxTL ? a.take((size_t)p.maxTL * p.elem) : nullptr;
    w.QY = p.maxTL ? a.take((size_t)p.maxTL * p.elem) : nullptr;
    w.Gn = p.maxGram ? a.take((size_t)p.maxGram * sizeof(float)) : nullptr;
    w.inter[0] = a.take((size_t)p.inter_elems * p.elem);
    w.inter[1] = a.take((size_t)p.inter_elems * p.elem);
    w.sumsq = a.take(sumsq_scratch_bytes());
    w.norms = (double*)a.take(sizeof(double) * 2);
}

#define TK_TRY(x)                                   \
    do {                                            \
        cudaError_t _e = (x);                       \
        if (_e != cudaSuccess) return _e;           \
    } while (0)

// X_out = M M^T X_in on the tensor cores (tf32 or split bf16) or with FP32/FP64 FMA.
template <typename T>
cudaError_t power_step(const T* M, const ModePlan& mp, const T* X_in, T* X_out, const Work& w, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (mp.tf32 || mp.bf16x1) {
            // cudaErrorNotSupported: M not 16-byte aligned for TMA; the next form runs
            const cudaError_t e =
                mp.tf32 ? launch_power_tf32(M, mp.mv, X_in, mp.L, X_out, w.partials, w.status, num_sms(), s)
                        : launch_power_bf16x1(M, mp.mv, X_in, mp.L, X_out, w.partials, w.status, num_sms(), s);
            if (e != cudaErrorNotSupported) return e;
        }
        if (mp.tc)
            return launch_power_tc(M, mp.mv, X_in, mp.L, X_out, w.partials, w.status, num_sms(), s);
        if (mp.wide) {
            const cudaError_t e = launch_power_wide(M, mp.mv, X_in, mp.L, X_out, mp.wide_split, false, 0, 0,
                                                    w.partials, w.status, num_sms(), s, w.wide_stages);
            if (e != cudaErrorNotSupported) return e;
        }
    }
    return launch_power<T>(M, mp.mv, X_in, mp.L, X_out, w.partials, mp.pp, false, 0, 0, s);
}

template <typename T>
cudaError_t sketch_factor(const T* M, const ModePlan& mp, int n, int q, uint64_t seed, int form, T* U,
                          const Work& w, cudaStream_t s);

// One mode's factor U (I_n x R_n) from the tensor B (view mp.v); with sampling,
// `norms` holds B's mode-n fiber norms when they were formed already (else w.w
// receives them here).
template <typename T>
cudaError_t factor_mode(const T* B, const ModePlan& mp, int n, int q, int prob, uint64_t seed, int form, T* U,
                        const Work& w, int64_t* sample_out, cudaStream_t s, const double* norms = nullptr) {
    const T* M = B;
    if (mp.T > 0) {
        const int64_t J = mp.v.fibers();
        if (prob == TUCKER_PROB_NEARLY_OPTIMAL && !norms) TK_TRY(launch_fiber_norms<T>(B, mp.v, w.w, s));
        const double* wn = norms ? norms : w.w;
        {
            ProfScope prof(kKSample, 0.0, 0.0, s);
            TK_TRY(launch_quantize(wn, J, prob, w.W, w.samp, s));
            TK_TRY(launch_sample(w.W, J, mp.T, seed, stream_id(1, n), w.idx, w.scale, w.samp, s));
        }
        TK_TRY(launch_gather<T>(B, mp.v, w.idx, w.scale, mp.T, (T*)w.Cp, s));
        if (sample_out) TK_TRY(cudaMemcpyAsync(sample_out, w.idx, sizeof(int64_t) * mp.T, cudaMemcpyDefault, s));
        M = (const T*)w.Cp;
    }
    return sketch_factor<T>(M, mp, n, q, seed, form, U, w, s);
}

// U from the sketch of M: the tensor's unfolding, or the gathered AMM sample
// C' (I_n x T) when mp.T > 0.
template <typename T>
cudaError_t sketch_factor(const T* M, const ModePlan& mp, int n, int q, uint64_t seed, int form, T* U,
                          const Work& w, cudaStream_t s) {
    const int L = mp.L;
    T* X0 = (T*)w.X0; T* X1 = (T*)w.X1; T* Q = (T*)w.Q;
    const size_t LL = (size_t)L * L;
    if (form == TUCKER_FORM_RELATED) {
        // Algorithms 6/7: the sketch as in the paper form (its span is that of X_q), P its
        // orthonormal basis by CholeskyQR2, Z = M (M^T P) by one more power step, and
        // H = P^T Z = (P^T M)(P^T M)^T, whose leading eigenvectors are the leading left
        // singular vectors of P^T M; Q_n = P U_H with the sign rule
        TK_TRY(launch_gaussian<T>(X0, mp.v.i, L, seed, stream_id(0, n), s));
        for (int k = 0; k < q; ++k) {
            const T* xin = X0;
            if (k > 0) {
                TK_TRY(launch_cholqr<T>(X1, Q, mp.op, w.factors + (size_t)(k - 1) * LL, w.orth, w.status, s));
                xin = Q;
            }
            TK_TRY(power_step<T>(M, mp, xin, X1, w, s));
        }
        T* P = (T*)w.Qt;
        double* fs = w.factors + (size_t)q * LL;
        TK_TRY(launch_cholqr<T>(X1, Q, mp.op, fs, w.orth, w.status, s));
        TK_TRY(launch_cholqr<T>(Q, P, mp.op, fs + LL, w.orth, w.status, s));
        TK_TRY(power_step<T>(M, mp, P, X1, w, s));                     // Z (I x L)
        T* H = X0;                                                    // L x L
        TK_TRY(launch_gemm_tn<T>(P, mp.v.i, L, X1, L, H, s));
        T* UH = Q;                                                    // L x R
        {
            ProfScope prof(kKExtract, 0.0, 0.0, s);
            TK_TRY(launch_extract<T>(H, X1, mp.opL, fs + 2 * LL, 0, mp.R, UH, w.orth, w.status, s));
        }
        TK_TRY(launch_gemm_nn<T>(P, mp.v.i, L, UH, mp.R, U, w.partials, num_sms(), s));
        return launch_sign_fix<T>(U, mp.v.i, mp.R, s);
    }
    if (form == TUCKER_FORM_PAPER && mp.half) {
        // C = (C' C'^T)^q Omega in half steps: from Q_{k-1} (Q_0 = Omega), Y_k = C'^T Q_{k-1}
        // = Q_Y R_Y and X_k = C' Q_Y, so C' C'^T Q_{k-1} = X_k R_Y; between steps X_k = Q_k F_k.
        // Hence C = X_q R_Y,q F_{q-1} R_Y,q-1 ... F_1 R_Y,1, the factors kept in that order.
        TK_TRY(launch_gaussian<T>(X0, mp.v.i, L, seed, stream_id(0, n), s));
        T* Y = (T*)w.Y;
        T* QY = (T*)w.QY;
        int f = 0;
        const T* xin = X0;
        for (int k = 0; k < q; ++k) {
            if (k > 0) {
                TK_TRY(launch_cholqr<T>(X1, Q, mp.op, w.factors + (size_t)f * LL, w.orth, w.status, s));
                ++f;
                xin = Q;
            }
            cudaError_t e = cudaErrorNotSupported;
            if constexpr (sizeof(T) == 4) {
                if (mp.half_tc) e = launch_wide_tn(M, mp.mv, xin, L, Y, w.partials, w.status, num_sms(), s,
                                                   w.wide_stages);
            }
            if (e == cudaErrorNotSupported) e = launch_gemm_tn<T>(M, mp.v.i, mp.T, xin, L, Y, s);
            TK_TRY(e);
            TK_TRY(launch_cholqr<T>(Y, QY, mp.opT, w.factors + (size_t)f * LL, w.orth, w.status, s));
            ++f;
            e = cudaErrorNotSupported;
            if constexpr (sizeof(T) == 4) {
                if (mp.half_tc) e = launch_wide_nn(M, mp.mv, QY, L, X1, w.partials, w.status, num_sms(), s,
                                                   w.wide_stages);
            }
            if (e == cudaErrorNotSupported) e = launch_gemm_nn<T>(M, mp.v.i, mp.T, QY, L, X1, w.partials, num_sms(), s);
            TK_TRY(e);
        }
        ProfScope prof(kKExtract, 0.0, 0.0, s);
        return launch_extract<T>(X1, Q, mp.op, w.factors, f, mp.R, U, w.orth, w.status, s);
    }
    if (form == TUCKER_FORM_PAPER) {
        // C = (M M^T)^q Omega in factored form: after each step X_k = Q_k F_k and
        // the next step multiplies Q_k, so C = X_q F_{q-1} ... F_1 with no overflow
        // and no loss of the weaker directions to FP32 rounding. Strategy B forms
        // G = M M^T once and multiplies it instead of passing over M each step.
        const T* Gm = nullptr;
        if constexpr (sizeof(T) == 4) {
            if (mp.gram) {
                const cudaError_t e = launch_gram_wide(M, mp.mv, (float*)w.Gn, true, w.partials, w.status, num_sms(),
                                                       s, w.wide_stages);
                if (e == cudaSuccess) Gm = (const T*)w.Gn;
                else if (e != cudaErrorNotSupported) return e;
            }
        }
        TK_TRY(launch_gaussian<T>(X0, mp.v.i, L, seed, stream_id(0, n), s));
        for (int k = 0; k < q; ++k) {
            const T* xin = X0;
            if (k > 0) {
                TK_TRY(launch_cholqr<T>(X1, Q, mp.op, w.factors + (size_t)(k - 1) * LL, w.orth, w.status, s));
                xin = Q;
            }
            if (Gm) TK_TRY(launch_gemm_nn<T>(Gm, mp.v.i, mp.v.i, xin, L, X1, w.partials, num_sms(), s));
            else TK_TRY(power_step<T>(M, mp, xin, X1, w, s));
        }
        ProfScope prof(kKExtract, 0.0, 0.0, s);
        return launch_extract<T>(X1, Q, mp.op, w.factors, q - 1, mp.R, U, w.orth, w.status, s);
    }
    cudaError_t first = cudaErrorNotSupported;
    if constexpr (sizeof(T) == 4) {
        if (mp.wide_range)
            first = launch_power_wide(M, mp.mv, nullptr, L, X1, mp.wide_split, true, seed, stream_id(0, n),
                                      w.partials, w.status, num_sms(), s, w.wide_stages);
    }
    if (first == cudaErrorNotSupported)
        first = launch_power<T>(M, mp.mv, nullptr, L, X1, w.partials, mp.pp, true, seed, stream_id(0, n), s);
    TK_TRY(first);
    for (int k = 0; k < q; ++k) {
        TK_TRY(launch_cholqr<T>(X1, Q, mp.op, w.factors, w.orth, w.status, s));
        TK_TRY(power_step<T>(M, mp, Q, X1, w, s));
    }
    ProfScope prof(kKExtract, 0.0, 0.0, s);
    return launch_extract<T>(X1, Q, mp.op, w.factors, 0, mp.R, U, w.orth, w.status, s);
}

// Mode-n product of the TTM chain: on the tensor cores (split bf16) for
// contiguous fibers when the plan's arithmetic is BF16 or TF32, else FP32/FP64 FMA.
template <typename T>
cudaError_t mode_product(const Plan& p, const T* A, const ModeView& v, const T* U, int64_t K, T* out,
                         const Work& w, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (p.prec != TUCKER_SK_FP32) {
            cudaError_t e = launch_ttm_tc(A, v, U, K, 1, v.i, out, w.status, num_sms(), s);
            if (e == cudaErrorNotSupported && wide_ttm_supported(v, K))
                e = launch_ttm_wide(A, v, U, K, 1, v.i, out, w.partials, w.status, num_sms(), s, w.wide_stages);
            if (e != cudaErrorNotSupported) return e;
        }
    }
    return launch_ttm<T>(A, v, U, K, 1, v.i, out, s, w.status);
}

template <typename T>
cudaError_t run_driver(const Plan& p, const T* A, const int32_t* ranks, int q, int prob, uint64_t seed, T* const* U,
                       T* G, const Work& w, int64_t* const* sample_out, bool want_re, cudaStream_t s) {
    const int N = p.N;
    if (want_re) TK_TRY(launch_sumsq<T>(A, nullptr, prod(p.dims, N), &w.norms[0], w.sumsq, s));
    if (p.st) {
        const T* cur = A;
        for (int n = 0; n < N; ++n) {
            const ModePlan& mp = p.m[n];
            TK_TRY(factor_mode<T>(cur, mp, n, q, prob, seed, p.form, U[n], w,
                                  sample_out ? sample_out[n] : nullptr, s));
            T* out = n == N - 1 ? G : (T*)w.inter[n & 1];
            TK_TRY(mode_product<T>(p, cur, mp.v, U[n], ranks[n], out, w, s));
            cur = out;
        }
    } else {
        // Algorithm 4 with the nearly-optimal probabilities: every mode samples the same
        // tensor, so an order-3 tensor's three modes take their fiber norms from one pass
        // over it, and modes 1 and 2 of higher orders from one pass
        const double* pre[3] = {nullptr, nullptr, nullptr};
        if (prob == TUCKER_PROB_NEARLY_OPTIMAL && N == 3 && p.m[0].T > 0 && p.m[1].T > 0 && p.m[2].T > 0 && w.w3 &&
            w.nscr) {
            TK_TRY(launch_fiber_norms123<T>(A, p.dims[0], p.dims[1], p.dims[2], w.w, w.w2, w.w3, w.nscr, s));
            pre[0] = w.w;
            pre[1] = w.w2;
            pre[2] = w.w3;
        } else if (prob == TUCKER_PROB_NEARLY_OPTIMAL && N >= 2 && p.m[0].T > 0 && p.m[1].T > 0 && w.w2 &&
                   fiber_norms12_supported(p.dims[0])) {
            TK_TRY(launch_fiber_norms12<T>(A, p.dims[0], p.dims[1], prod(p.dims, N) / (p.dims[0] * p.dims[1]), w.w,
                                           w.w2, s));
            pre[0] = w.w;
            pre[1] = w.w2;
        }
        for (int n = 0; n < N; ++n)
            TK_TRY(factor_mode<T>(A, p.m[n], n, q, prob, seed, p.form, U[n], w,
                                  sample_out ? sample_out[n] : nullptr, s, n < 3 ? pre[n] : nullptr));
        int64_t e[kMaxOrder];
        for (int n = 0; n < N; ++n) e[n] = p.dims[n];
        const T* cur = A;
        for (int n = 0; n < N; ++n) {
            const ModeView v = view_of(e, N, n);
            T* out = n == N - 1 ? G : (T*)w.inter[n & 1];
            TK_TRY(mode_product<T>(p, cur, v, U[n], ranks[n], out, w, s));
            e[n] = ranks[n];
            cur = out;
        }
    }
    if (want_re) {
        int64_t r = 1;
        for (int n = 0; n < N; ++n) r *= ranks[n];
        TK_TRY(launch_sumsq<T>(G, nullptr, r, &w.norms[1], w.sumsq, s));
    }
    return cudaSuccess;
}

tucker_status finish(cudaStream_t s, int* dev_status, const Opts& o, double* dev_norms) {
    if (o.flags & TUCKER_FLAG_ASYNC) {
        g_async_stream = s;
        g_async_status = dev_status;
        return TUCKER_OK;
    }
    int st = 0;
    double nrm[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(&st, dev_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && o.rel_error && dev_norms)
        e = cudaMemcpyAsync(nrm, dev_norms, sizeof(nrm), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    if (o.rel_error && dev_norms) {
        const double r = nrm[0] > 0 ? 1.0 - nrm[1] / nrm[0] : 0.0;
        *o.rel_error = r > 0 ? sqrt(r) : 0.0;
    }
    if (st & kStatTimeout) return TUCKER_ERR_TIMEOUT;
    if (st & kStatNumerical) return TUCKER_ERR_NUMERICAL;
    return TUCKER_OK;
}

tucker_status driver(bool st, const void* A, tucker_dtype dt, const int64_t* dims, int N, const int32_t* ranks,
                     int32_t P, int32_t q, int64_t c, tucker_prob prob, uint64_t seed, void* const* U, void* G,
                     const tucker_opts* opts) {
    cudaGetLastError();      // a failed call of other code must not be reported as ours
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    if (prob != TUCKER_PROB_NEARLY_OPTIMAL && prob != TUCKER_PROB_UNIFORM) return TUCKER_ERR_INVALID_ARG;
    if (!A || !U || !G) return TUCKER_ERR_INVALID_ARG;
    if (o.prec != TUCKER_SK_FP32 && dt != TUCKER_F32) return TUCKER_ERR_UNSUPPORTED;
    for (int n = 0; n < N && n < kMaxOrder; ++n)
        if (!U[n]) return TUCKER_ERR_INVALID_ARG;
    const int elem = dt == TUCKER_F64 ? 8 : 4;
    Plan p;
    rs = make_plan(st, elem, dims, N, ranks, P, q, c, o, p);
    if (rs != TUCKER_OK) return rs;
    if ((o.flags & TUCKER_FLAG_ASYNC) && !o.workspace) return TUCKER_ERR_INVALID_ARG;

    cudaStream_t s = o.stream;
    // stage host buffers
    const int64_t E = prod(dims, N);
    int64_t Gn = 1, Un = 0;
    for (int n = 0; n < N; ++n) { Gn *= ranks[n]; Un += dims[n] * ranks[n]; }
    // asynchronous calls take device buffers as given (no driver queries, so the
    // call can be captured into a CUDA graph); synchronous calls stage host buffers
    const bool async = (o.flags & TUCKER_FLAG_ASYNC) != 0;
    TuneAllow tune(!async);                // a synchronous call may time kernel candidates
    const bool hA = !async && !on_device(A), hG = !async && !on_device(G);
    bool hU = false;
    for (int n = 0; n < N && !async; ++n) hU = hU || !on_device(U[n]);

    Arena a;
    Work w;
    carve(p, a, w);      // measure
    size_t need = a.used;
    size_t stage = 0;
    if (hA) stage += ((size_t)E * elem + 255) & ~size_t(255);
    if (hU) stage += ((size_t)Un * elem + 255) & ~size_t(255);
    if (hG) stage += ((size_t)Gn * elem + 255) & ~size_t(255);

    void* owned = nullptr;
    char* base;
    if (o.workspace) {
        if (o.workspace_bytes < need) return TUCKER_ERR_INVALID_ARG;
        base = (char*)o.workspace;
    } else {
        cudaError_t e = cudaMallocAsync(&owned, need, s);
        if (e != cudaSuccess) return from_cuda(e);
        base = (char*)owned;
    }
    void* stage_buf = nullptr;
    if (stage) {
        cudaError_t e = cudaMallocAsync(&stage_buf, stage, s);
        if (e != cudaSuccess) {
            if (owned) cudaFreeAsync(owned, s);
            return from_cuda(e);
        }
    }
    Arena b;
    b.base = base;
    b.cap = need;
    carve(p, b, w);
    // asynchronous calls run beside others (batches, the serving loop): keep the shallow rings
    w.wide_stages = async ? kWideStagesShared : kWideStagesAlone;

    char* sp = (char*)stage_buf;
    const void* dA = A;
    void* dU[kMaxOrder];
    void* dG = G;
    cudaError_t e = cudaSuccess;
    if (hA) {
        dA = sp;
        e = cudaMemcpyAsync(sp, A, (size_t)E * elem, cudaMemcpyHostToDevice, s);
        sp += ((size_t)E * elem + 255) & ~size_t(255);
    }
    for (int n = 0; n < N; ++n) dU[n] = U[n];
    if (hU) {
        for (int n = 0; n < N; ++n) {
            dU[n] = sp;
            sp += (size_t)dims[n] * ranks[n] * elem;
        }
        sp = (char*)(((uintptr_t)sp + 255) & ~uintptr_t(255));
    }
    if (hG) dG = sp;

    if (e == cudaSuccess) e = cudaMemsetAsync(w.status, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        if (elem == 4)
            e = run_driver<float>(p, (const float*)dA, ranks, q, prob, seed, (float* const*)dU, (float*)dG, w,
                                  o.sample_idx, o.rel_error != nullptr, s);
        else
            e = run_driver<double>(p, (const double*)dA, ranks, q, prob, seed, (double* const*)dU, (double*)dG, w,
                                   o.sample_idx, o.rel_error != nullptr, s);
    }
    if (e == cudaSuccess && hU)
        for (int n = 0; n < N && e == cudaSuccess; ++n)
            e = cudaMemcpyAsync(U[n], dU[n], (size_t)dims[n] * ranks[n] * elem, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && hG) e = cudaMemcpyAsync(G, dG, (size_t)Gn * elem, cudaMemcpyDeviceToHost, s);
    tucker_status out = e == cudaSuccess ? finish(s, w.status, o, w.norms) : from_cuda(e);
    if (owned) cudaFreeAsync(owned, s);
    if (stage_buf) cudaFreeAsync(stage_buf, s);
    if (owned || stage_buf) cudaStreamSynchronize(s);
    return out;
}

// Scratch for a single step entry point.
struct Scratch {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    tucker_status get(size_t n, cudaStream_t st) {
        s = st;
        return from_cuda(cudaMallocAsync(&p, n ? n : 256, st));
    }
    ~Scratch() {
        if (p) {
            cudaFreeAsync(p, s);
            cudaStreamSynchronize(s);
        }
    }
};

tucker_status sync_status(cudaStream_t s, const int* dev_status) {
    int st = 0;
    cudaError_t e = cudaSuccess;
    if (dev_status) e = cudaMemcpyAsync(&st, dev_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    if (st & kStatTimeout) return TUCKER_ERR_TIMEOUT;
    if (st & kStatNumerical) return TUCKER_ERR_NUMERICAL;
    return TUCKER_OK;
}

bool mode_args_ok(const void* A, const int64_t* dims, int N, int mode) {
    if (!A || !dims || N < 1 || N > kMaxOrder || mode < 0 || mode >= N) return false;
    for (int n = 0; n < N; ++n)
        if (dims[n] < 1) return false;
    return true;
}

// ------------------------------------------------------------------ fixed-precision ranks
// Problem 2 (concluding section): ranks r_n and factors Q_n with
// ||A - A x_1 Q_1 Q_1^T ... x_N Q_N Q_N^T||_F <= eps ||A||_F, in ST-HOSVD order.
// The energies the modes discard add up exactly (each truncation is an
// orthogonal projection of the tensor the previous ones left), so mode n
// (0-based) may discard budget_n = (eps^2 ||A||^2 - discarded so far) / (N - n).
// For mode n an L-column sketch (L = L0, doubled up to I_n) gives the L leading
// left singular vectors U_L of the paper form's C_n; Y = B x_n U_L^T gives the
// kept energies e_k = ||slice k of Y||^2, and r is the smallest count with
// ||B||^2 - (e_1 + ... + e_r) <= budget_n. Without one the sketch is widened; at
// L = I_n nothing is discarded. Q_n = U_L(:, 1:r) and the next B is the first r
// slices of Y. The decisions are taken on the host, in FP64, from the device's
// energies.
template <typename T>
tucker_status adaptive_run(const T* A, const int64_t* dims, int N, double eps, int q, int L0, uint64_t seed,
                           const Opts& o, T* const* U, T* G, int32_t* ranks) {
    cudaStream_t s = o.stream;
    const int elem = (int)sizeof(T);
    const int sms = num_sms();
    const int64_t E = prod(dims, N);
    int64_t maxI = 0;
    for (int n = 0; n < N; ++n) maxI = std::max(maxI, dims[n]);
    tucker_status rs;
    Scratch bY, bB0, bB1, bU, bS;
    if ((rs = bY.get((size_t)E * elem, s)) != TUCKER_OK) return rs;
    if ((rs = bB0.get((size_t)E * elem, s)) != TUCKER_OK) return rs;
    if ((rs = bB1.get((size_t)E * elem, s)) != TUCKER_OK) return rs;
    if ((rs = bU.get((size_t)maxI * std::min<int64_t>(maxI, kMaxL) * elem, s)) != TUCKER_OK) return rs;
    if ((rs = bS.get(sizeof(double) * 256 + sumsq_scratch_bytes(), s)) != TUCKER_OK) return rs;
    T* Y = (T*)bY.p;
    T* Bb[2] = {(T*)bB0.p, (T*)bB1.p};
    T* UL = (T*)bU.p;
    double* de = (double*)bS.p;              // [128] energies
    double* dn = de + 128;                   // [1] a norm
    void* sumsq_scr = de + 256;
    auto sumsq_host = [&](const T* x, int64_t n, double* out) -> tucker_status {
        cudaError_t e = launch_sumsq<T>(x, nullptr, n, dn, sumsq_scr, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, dn, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return from_cuda(e);
    };
    double total = 0.0;
    if ((rs = sumsq_host(A, E, &total)) != TUCKER_OK) return rs;
    const double allowed = eps * eps * total;
    double spent = 0.0;
    int64_t cd[kMaxOrder];
    for (int n = 0; n < N; ++n) cd[n] = dims[n];
    const T* cur = A;
    for (int n = 0; n < N; ++n) {
        const ModeView v = view_of(cd, N, n);
        const int64_t I = cd[n];
        double normB = total;
        if (n > 0 && (rs = sumsq_host(cur, prod(cd, N), &normB)) != TUCKER_OK) return rs;
        const double budget = (allowed - spent) / (double)(N - n);
        int64_t L = std::min<int64_t>(L0, I);
        int64_t r = 0;
        double kept = 0.0;
        for (;;) {
            if (L > kMaxL) return TUCKER_ERR_UNSUPPORTED;
            Plan p;
            p.N = N;
            p.st = true;
            p.elem = elem;
            p.form = o.form;
            p.prec = o.prec;
            p.q = q;
            for (int k = 0; k < N; ++k) p.dims[k] = cd[k];
            if ((rs = plan_mode(p, cd, N, n, L, 0, 0, true, elem, o, sms)) != TUCKER_OK) return rs;
            Arena a;
            Work w;
            carve(p, a, w);
            ModeView vy = v;
            vy.i = L;
            const size_t wbytes = (a.used + 255) & ~size_t(255);
            Scratch ws;
            if ((rs = ws.get(wbytes + slice_sumsq_scratch_bytes(vy, sms), s)) != TUCKER_OK) return rs;
            Arena b;
            b.base = (char*)ws.p;
            b.cap = a.used;
            carve(p, b, w);
            double e[128];
            int st = 0;
            cudaError_t ce = cudaMemsetAsync(w.status, 0, sizeof(int), s);
            if (ce == cudaSuccess)
                ce = factor_mode<T>(cur, p.m[n], n, q, TUCKER_PROB_UNIFORM, seed, o.form, UL, w, nullptr, s);
            if (ce == cudaSuccess) ce = mode_product<T>(p, cur, v, UL, L, Y, w, s);
            if (ce == cudaSuccess) ce = launch_slice_sumsq<T>(Y, vy, de, (char*)ws.p + wbytes, sms, s);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(e, de, sizeof(double) * L, cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(&st, w.status, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) return from_cuda(ce);
            if (st & kStatTimeout) return TUCKER_ERR_TIMEOUT;
            if (st & kStatNumerical) return TUCKER_ERR_NUMERICAL;
            double acc = 0.0;
            r = 0;
            for (int64_t k = 0; k < L; ++k) {
                acc += e[k];
                if (normB - acc <= budget) {
                    r = k + 1;
                    break;
                }
            }
            if (r > 0 || L == I) {
                if (r == 0) r = L;
                kept = 0.0;
                for (int64_t k = 0; k < r; ++k) kept += e[k];
                break;
            }
            L = std::min<int64_t>(2 * L, I);
        }
        ranks[n] = (int32_t)r;
        spent += normB - kept;
        T* dst = n == N - 1 ? G : Bb[n & 1];
        const size_t run = (size_t)v.lf * elem;
        cudaError_t ce = cudaMemcpyAsync(U[n], UL, (size_t)I * r * elem, cudaMemcpyDeviceToDevice, s);
        if (ce == cudaSuccess)
            ce = cudaMemcpy2DAsync(dst, run * r, Y, run * L, run * r, (size_t)v.rt, cudaMemcpyDeviceToDevice, s);
        if (ce != cudaSuccess) return from_cuda(ce);
        cur = dst;
        cd[n] = r;
    }
    if (o.rel_error) {
        double g2 = 0.0;
        if ((rs = sumsq_host(G, prod(cd, N), &g2)) != TUCKER_OK) return rs;
        const double r2 = total > 0.0 ? 1.0 - g2 / total : 0.0;
        *o.rel_error = r2 > 0.0 ? sqrt(r2) : 0.0;
    }
    return from_cuda(cudaStreamSynchronize(s));
}

}  // namespace

tucker_status status_from_cuda(cudaError_t e) { return from_cuda(e); }

// ------------------------------------------------------------------ work-list batches
// The requests of a batch as phases of the work-list kernel and grouped
// orthonormalisations, in the order of the drivers' own launches: for each mode
// n one phase with every request's truncation by U_{n-1} (ST-HOSVD), status
// reset and Omega_n, then per power step a phase of partials and a phase of
// their sums, then the orthonormalisation of every request's sketch in one
// launch; last, the cores (T-HOSVD's chain a phase per position). Items of one
// phase never depend on one another: what a task reads was written by an
// earlier phase, an earlier launch on the lane's stream. The requests are dealt to lanes (request k
// to lane k mod lanes; a lane per four requests, at most eight), each lane a
// sequence of its own on a stream of its own,
// so one lane's orthonormalisations (a few CTAs each) overlap another lane's
// streaming steps. Each request keeps its own workspace slice (the layout of an
// asynchronous call), so its results are those of the request alone (FP32
// power-step tiles as planned, without autotuning).
tucker_status worklist_plan(int n, const tucker_request* reqs, const tucker_opts& opts, char* ws,
                            const std::vector<size_t>& offsets, WorklistPlan& wp, int max_lanes) {
    wp = WorklistPlan();
    Opts o;
    tucker_status rs = read_opts(&opts, o);
    if (rs != TUCKER_OK) return rs;
    if (o.form != TUCKER_FORM_PAPER || o.prec != TUCKER_SK_FP32 || o.alpha != 0.0) return TUCKER_ERR_UNSUPPORTED;
    if (n < 1 || (int)offsets.size() < n) return TUCKER_ERR_INVALID_ARG;
    const int elem = reqs[0].dt == TUCKER_F64 ? 8 : 4;
    wp.elem = elem;
    std::vector<Plan> plans(n);
    std::vector<Work> works(n);
    for (int k = 0; k < n; ++k) {
        const tucker_request& r = reqs[k];
        if ((r.dt != TUCKER_F32 && r.dt != TUCKER_F64) || (r.dt == TUCKER_F64 ? 8 : 4) != elem) return TUCKER_ERR_UNSUPPORTED;
        if (r.c != 0) return TUCKER_ERR_UNSUPPORTED;
        rs = make_plan(r.which == 1, elem, r.dims, r.N, r.ranks, r.P, r.q, 0, o, plans[k]);
        if (rs != TUCKER_OK) return rs;
        const Plan& p = plans[k];
        for (int m = 0; m < r.N; ++m) {
            const ModePlan& mp = p.m[m];
            if (mp.v.i > kThreads || r.dims[m] > kThreads || worklist_ttm_opt(r.ranks[m]) == 0 || mp.T != 0 ||
                mp.gram || mp.half || mp.tc || mp.tf32 || mp.bf16x1 || mp.wide)
                return TUCKER_ERR_UNSUPPORTED;
            if (mp.pp.jb != (elem == 4 ? 32 : 16)) return TUCKER_ERR_UNSUPPORTED;
        }
        Arena a;
        a.base = ws ? ws + offsets[k] : nullptr;
        a.cap = ~size_t(0) >> 1;
        carve(p, a, works[k]);
    }
    // every extent a block program will touch, checked against the buffer it
    // targets (elements): what the items and jobs read and write stays inside
    // the request's buffers whatever the shapes
    bool fits = true;
    auto need = [&](bool ok) { fits = fits && ok; };
    std::vector<int64_t> cap_il(n), cap_part(n), cap_inter(n), cap_fac(n), cap_A(n), cap_G(n);
    for (int k = 0; k < n; ++k) {
        const Plan& p = plans[k];
        const tucker_request& r = reqs[k];
        cap_il[k] = p.maxI * p.maxL;
        cap_part[k] = (int64_t)(p.max_partials / elem);
        cap_inter[k] = p.inter_elems;
        cap_fac[k] = (int64_t)r.q * p.maxL * p.maxL;        // paper form without half steps: q slots
        cap_A[k] = prod(r.dims, r.N);
        int64_t g = 1;
        for (int m = 0; m < r.N; ++m) g *= r.ranks[m];
        cap_G[k] = g;
    }
    // four requests or more per lane, at most eight lanes
    wp.lanes = std::max(1, std::min(std::min(8, max_lanes), n / 4));
    std::vector<WTask>& tasks = wp.tasks;
    std::vector<WItem>& items = wp.items;
    auto add = [&](WTask t, int gx, int gy) -> int {
        t.nitems = gx * gy;
        const int id = (int)tasks.size();
        tasks.push_back(t);
        for (int x = 0; x < gx; ++x)
            for (int y = 0; y < gy; ++y) items.push_back(WItem{id, x, y, 0});
        return id;
    };
    auto base_task = [&](int kind, int k) {
        WTask t{};
        t.kind = kind;
        t.dep[0] = t.dep[1] = -1;
        t.status = works[k].status;
        return t;
    };
    const int NF = elem == 4 ? 2 : 1;
    for (int lane = 0; lane < wp.lanes; ++lane) {
        std::vector<int> mem;
        for (int k = lane; k < n; k += wp.lanes) mem.push_back(k);
        int maxN = 0, maxq = 0;
        for (int k : mem) {
            maxN = std::max(maxN, reqs[k].N);
            maxq = std::max(maxq, reqs[k].q);
        }
        size_t step_smem = 0;
        int step_heavy = 0;
        int step_begin = (int)items.size();
        auto note = [&](const WTask& t, size_t smem) {
            step_smem = std::max(step_smem, smem);
            step_heavy |= worklist_heavy(t) ? 1 : 0;
        };
        auto close_step = [&]() {
            if ((int)items.size() > step_begin)
                wp.ops.push_back(
                    WorklistOp{0, step_begin, (int)items.size(), wp.steps++, step_smem, 0, step_heavy, lane});
            step_begin = (int)items.size();
            step_smem = 0;
            step_heavy = 0;
        };
        // the mode product out = in x_m U (fibers of view v), as one task
        auto ttm_task = [&](int k, const void* in, const ModeView& v, const void* U, int64_t K, void* out, int dep,
                            int64_t in_cap, int64_t out_cap) {
            need(v.fibers() * v.i <= in_cap && v.fibers() * K <= out_cap && v.i <= kThreads);
            WTask t = base_task(kWTtm, k);
            t.in = in;
            t.X = U;
            t.out = out;
            t.v = v;
            t.K = K;
            t.opt = worklist_ttm_opt(K);
            t.dep[0] = dep;
            note(t, worklist_ttm_smem(elem, t.opt));
            const int64_t gx = (v.fibers() + 64 * NF - 1) / (64 * NF), gy = (K + 4 * t.opt - 1) / (4 * t.opt);
            return add(t, (int)gx, (int)gy);
        };
        std::vector<const void*> cur(n);
        for (int k : mem) cur[k] = reqs[k].A;
        std::vector<int> init(n, -1), prev(n, -1);
        for (int m = 0; m < maxN; ++m) {
            // step: [truncation by U_{m-1}], [status reset], Omega_m, power step 1, its sum
            std::vector<int> ttm(n, -1), gen(n, -1), pw(n, -1);
            for (int k : mem) {
                const tucker_request& r = reqs[k];
                if (r.which == 1 && m > 0 && m < r.N) {
                    void* out = (void*)works[k].inter[(m - 1) & 1];
                    ttm[k] = ttm_task(k, cur[k], plans[k].m[m - 1].v, r.U[m - 1], r.ranks[m - 1], out, -1,
                                      m == 1 ? cap_A[k] : cap_inter[k], cap_inter[k]);
                    cur[k] = out;
                }
            }
            for (int k : mem) {
                const tucker_request& r = reqs[k];
                if (m >= r.N) continue;
                const ModePlan& mp = plans[k].m[m];
                if (m == 0) init[k] = add(base_task(kWInit, k), 1, 1);
                WTask t = base_task(kWGen, k);
                t.out = works[k].X0;
                t.rows = mp.v.i;
                t.cols = mp.L;
                t.seed = r.seed;
                t.sid = stream_id(0, m);
                (void)init;
                const int64_t ne = mp.v.i * (int64_t)mp.L;
                need(ne <= cap_il[k]);
                gen[k] = add(t, (int)std::max<int64_t>(1, (ne + 4 * kThreads - 1) / (4 * kThreads)), 1);
            }
            close_step();                    // phase 1: truncation, status reset, Omega_m
            for (int q = 0; q < maxq; ++q) {
                if (q > 0) {
                    // CholeskyQR of every sketch that takes another power step, in one launch
                    const int j0 = (int)wp.jobs.size();
                    for (int k : mem) {
                        const tucker_request& r = reqs[k];
                        if (m >= r.N || q >= r.q) continue;
                        const ModePlan& mp = plans[k].m[m];
                        OrthJob j = orth_job(mp.op, works[k].orth);
                        j.X = works[k].X1;
                        j.Q = works[k].Q;
                        j.R = mp.R;
                        j.factor = works[k].factors + (size_t)(q - 1) * mp.L * mp.L;
                        j.fofs = 0;
                        need(mp.v.i * (int64_t)mp.L <= cap_il[k] && (int64_t)q * mp.L * mp.L <= cap_fac[k]);
                        j.status = works[k].status;
                        wp.jobs.push_back(j);
                    }
                    if ((int)wp.jobs.size() > j0)
                        wp.ops.push_back(WorklistOp{1, j0, (int)wp.jobs.size(), -1, 0, 0, 0, lane});
                }
                for (int k : mem) {
                    const tucker_request& r = reqs[k];
                    if (m >= r.N || q >= r.q) continue;
                    const ModePlan& mp = plans[k].m[m];
                    WTask t = base_task(kWPow, k);
                    t.in = r.which == 1 ? cur[k] : r.A;
                    t.v = mp.v;
                    t.X = q == 0 ? works[k].X0 : works[k].Q;
                    t.L = mp.L;
                    t.out = works[k].partials;
                    t.tiles = mp.pp.tiles;
                    t.parts = mp.pp.parts;
                    t.jb = mp.pp.jb;
                    t.lg = mp.pp.lg;
                    if (q == 0) {
                        t.dep[0] = gen[k];
                        t.dep[1] = ttm[k];
                    }
                    need(mp.v.fibers() * mp.v.i <= (r.which == 1 && m > 0 ? cap_inter[k] : cap_A[k]) &&
                         mp.v.i * (int64_t)mp.L <= cap_il[k] &&
                         (int64_t)mp.pp.parts * mp.v.i * mp.L <= cap_part[k] && mp.v.i <= kThreads &&
                         mp.pp.tiles * mp.pp.jb >= mp.v.fibers() && mp.pp.groups * mp.pp.lg >= mp.L);
                    note(t, worklist_pow_smem(elem, (int)mp.v.i, mp.pp.lg));
                    pw[k] = add(t, mp.pp.groups, mp.pp.parts);
                }
                close_step();                // phase 2: the power step's partials
                for (int k : mem) {
                    const tucker_request& r = reqs[k];
                    if (m >= r.N || q >= r.q) continue;
                    const ModePlan& mp = plans[k].m[m];
                    WTask t = base_task(kWRed, k);
                    t.in = works[k].partials;
                    t.out = works[k].X1;
                    t.parts = mp.pp.parts;
                    t.count = mp.v.i * (int64_t)mp.L;
                    t.dep[0] = pw[k];
                    need((int64_t)t.parts * t.count <= cap_part[k] && t.count <= cap_il[k]);
                    add(t, (int)std::max<int64_t>(1, (t.count + 255) / 256), 1);
                }
                close_step();                // phase 3: their sums
            }
            // the leading factor of every sketch, in one launch
            const int j0 = (int)wp.jobs.size();
            for (int k : mem) {
                const tucker_request& r = reqs[k];
                if (m >= r.N) continue;
                const ModePlan& mp = plans[k].m[m];
                OrthJob j = orth_job(mp.op, works[k].orth);
                j.X = works[k].X1;
                j.Q = works[k].Q;
                j.R = mp.R;
                j.factor = works[k].factors;
                j.nprev = r.q - 1;
                j.fofs = (int64_t)(r.q - 1) * mp.L * mp.L;
                j.U = r.U[m];
                j.status = works[k].status;
                j.staged = orth_group_staged(j, elem) ? 1 : 0;
                need(mp.v.i * (int64_t)mp.L <= cap_il[k] && (int64_t)r.q * mp.L * mp.L <= cap_fac[k] &&
                     mp.v.i == r.dims[m] && mp.R == r.ranks[m]);
                wp.jobs.push_back(j);
            }
            wp.ops.push_back(WorklistOp{2, j0, (int)wp.jobs.size(), -1, 0, 0, 0, lane});
        }
        // the cores: ST-HOSVD's last truncation; T-HOSVD's chain x_1 U_1^T ... x_N U_N^T
        for (int m = 0; m < maxN; ++m) {
            for (int k : mem) {
                const tucker_request& r = reqs[k];
                if (r.which == 1) {
                    if (m == r.N - 1)
                        ttm_task(k, cur[k], plans[k].m[m].v, r.U[m], r.ranks[m], r.G, -1,
                                 m == 0 ? cap_A[k] : cap_inter[k], cap_G[k]);
                    continue;
                }
                if (m >= r.N) continue;
                int64_t e[kMaxOrder];
                for (int a = 0; a < r.N; ++a) e[a] = a < m ? r.ranks[a] : r.dims[a];
                void* out = m == r.N - 1 ? r.G : works[k].inter[m & 1];
                prev[k] = ttm_task(k, cur[k], view_of(e, r.N, m), r.U[m], r.ranks[m], out, prev[k],
                                   m == 0 ? cap_A[k] : cap_inter[k], m == r.N - 1 ? cap_G[k] : cap_inter[k]);
                cur[k] = out;
            }
            close_step();                    // a phase per position of the chain
        }
    }
    if (!fits) return TUCKER_ERR_INVALID_ARG;
    // every task a task reads the output of runs in an earlier phase of the same
    // lane (an earlier launch on the lane's stream): no item waits for another
    std::vector<int> phase_of(items.size(), -1), lane_of(items.size(), -1), first(tasks.size(), -1);
    for (const WorklistOp& op : wp.ops)
        if (op.kind == 0)
            for (int i = op.a; i < op.b; ++i) {
                phase_of[i] = op.step;
                lane_of[i] = op.lane;
            }
    for (int i = 0; i < (int)items.size(); ++i)
        if (first[items[i].task] < 0) first[items[i].task] = i;
    for (int i = 0; i < (int)items.size(); ++i)
        for (int d : tasks[items[i].task].dep)
            if (d >= 0 && (d >= items[i].task || lane_of[first[d]] != lane_of[i] || phase_of[first[d]] >= phase_of[i]))
                return TUCKER_ERR_INVALID_ARG;
    const size_t a256 = 255;
    wp.tasks_off = 0;
    wp.items_off = (sizeof(WTask) * tasks.size() + a256) & ~a256;
    wp.jobs_off = wp.items_off + ((sizeof(WItem) * items.size() + a256) & ~a256);
    wp.desc_bytes = wp.jobs_off + sizeof(OrthJob) * wp.jobs.size();
    wp.counters_off = (wp.desc_bytes + a256) & ~a256;
    wp.counter_bytes = sizeof(unsigned) * (size_t)wp.steps;
    wp.area_bytes = wp.counters_off + ((wp.counter_bytes + a256) & ~a256);
    return TUCKER_OK;
}

void worklist_prepare(WorklistPlan& wp) {
    for (WorklistOp& op : wp.ops)
        if (op.kind == 0) op.grid = worklist_grid(wp.elem, op.heavy != 0, op.smem, op.b - op.a);
}

void worklist_pack(const WorklistPlan& wp, void* host) {
    char* h = (char*)host;
    std::memcpy(h + wp.tasks_off, wp.tasks.data(), sizeof(WTask) * wp.tasks.size());
    std::memcpy(h + wp.items_off, wp.items.data(), sizeof(WItem) * wp.items.size());
    if (!wp.jobs.empty()) std::memcpy(h + wp.jobs_off, wp.jobs.data(), sizeof(OrthJob) * wp.jobs.size());
}

cudaError_t worklist_enqueue(const WorklistPlan& wp, char* area, const void* host_desc,
                             const std::vector<cudaStream_t>& lane_streams, cudaEvent_t uploaded) {
    if ((int)lane_streams.size() < wp.lanes) return cudaErrorInvalidValue;
    cudaStream_t s0 = lane_streams[0];
    cudaError_t e = cudaMemcpyAsync(area, host_desc, wp.desc_bytes, cudaMemcpyHostToDevice, s0);
    unsigned* counters = (unsigned*)(area + wp.counters_off);
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, wp.counter_bytes, s0);
    if (e == cudaSuccess) e = cudaEventRecord(uploaded, s0);
    for (int l = 1; l < wp.lanes && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(lane_streams[l], uploaded, 0);
    const WTask* tasks = (const WTask*)(area + wp.tasks_off);
    const WItem* items = (const WItem*)(area + wp.items_off);
    const OrthJob* jobs = (const OrthJob*)(area + wp.jobs_off);
    for (const WorklistOp& op : wp.ops) {
        if (e != cudaSuccess) break;
        cudaStream_t s = lane_streams[op.lane];
        if (op.kind == 0) {
            e = wp.elem == 4 ? launch_worklist<float>(tasks, items, op.a, op.b, counters + op.step, op.heavy != 0,
                                                      op.smem, op.grid, s)
                             : launch_worklist<double>(tasks, items, op.a, op.b, counters + op.step, op.heavy != 0,
                                                       op.smem, op.grid, s);
        } else {
            const std::vector<OrthJob> h(wp.jobs.begin() + op.a, wp.jobs.begin() + op.b);
            ProfScope prof(kKExtract, 0.0, 0.0, s);
            if (op.kind == 1)
                e = wp.elem == 4 ? launch_cholqr_group<float>(jobs + op.a, h, s)
                                 : launch_cholqr_group<double>(jobs + op.a, h, s);
            else
                e = wp.elem == 4 ? launch_extract_group<float>(jobs + op.a, h, s)
                                 : launch_extract_group<double>(jobs + op.a, h, s);
        }
    }
    return e;
}

}  // namespace tk

using namespace tk;

extern "C" {

tucker_status tucker_rthosvd(const void* A, tucker_dtype dt, const int64_t* dims, int N, const int32_t* ranks,
                             int32_t P, int32_t q, int64_t c, tucker_prob prob, uint64_t seed, void* const* U, void* G,
                             const tucker_opts* opts) {
    return driver(false, A, dt, dims, N, ranks, P, q, c, prob, seed, U, G, opts);
}

tucker_status tucker_rsthosvd(const void* A, tucker_dtype dt, const int64_t* dims, int N, const int32_t* ranks,
                              int32_t P, int32_t q, int64_t c, tucker_prob prob, uint64_t seed, void* const* U,
                              void* G, const tucker_opts* opts) {
    return driver(true, A, dt, dims, N, ranks, P, q, c, prob, seed, U, G, opts);
}

tucker_status tucker_workspace_size(int which, tucker_dtype dt, const int64_t* dims, int N, const int32_t* ranks,
                                    int32_t P, int32_t q, int64_t c, const tucker_opts* opts, size_t* bytes) {
    if (!bytes || (which != 0 && which != 1)) return TUCKER_ERR_INVALID_ARG;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    Plan p;
    rs = make_plan(which == 1, dt == TUCKER_F64 ? 8 : 4, dims, N, ranks, P, q, c, o, p);
    if (rs != TUCKER_OK) return rs;
    Arena a;
    Work w;
    carve(p, a, w);
    *bytes = a.used;
    return TUCKER_OK;
}

tucker_status tucker_plan_describe(int which, tucker_dtype dt, const int64_t* dims, int N, const int32_t* ranks,
                                   int32_t P, int32_t q, int64_t c, const tucker_opts* opts, char* buf,
                                   size_t buf_bytes) {
    if (!buf || buf_bytes == 0 || (which != 0 && which != 1)) return TUCKER_ERR_INVALID_ARG;
    buf[0] = 0;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    Plan p;
    rs = make_plan(which == 1, dt == TUCKER_F64 ? 8 : 4, dims, N, ranks, P, q, c, o, p);
    if (rs != TUCKER_OK) return rs;
    // the same choices power_step() and mode_product() make, for 16-byte aligned tensors
    std::string text;
    int64_t e[kMaxOrder];
    for (int n = 0; n < N; ++n) e[n] = p.dims[n];
    for (int n = 0; n < N; ++n) {
        const ModePlan& mp = p.m[n];
        const char* power = p.elem == 8 ? "fp64"
                            : mp.gram   ? "gram-split-bf16"
                            : mp.tf32   ? "tf32"
                            : mp.bf16x1 ? "bf16x1"
                            : mp.tc     ? "split-bf16"
                            : mp.wide   ? (mp.wide_split ? "wide-split-bf16" : "wide-bf16x1")
                                        : "fp32";
        const ModeView tv = p.st ? mp.v : view_of(e, N, n);
        const bool tc_ttm = p.elem == 4 && p.prec != TUCKER_SK_FP32;
        const char* ttm = p.elem == 8                                       ? "fp64"
                          : (tc_ttm && ttm_tc_supported(tv, ranks[n]))     ? "split-bf16"
                          : (tc_ttm && wide_ttm_supported(tv, ranks[n]))   ? "wide-split-bf16"
                                                                           : "fp32";
        const char* range = p.form != TUCKER_FORM_RANGE ? ""
                            : p.elem == 8               ? " range-sketch=fp64"
                            : mp.wide_range ? (mp.wide_split ? " range-sketch=wide-split-bf16" : " range-sketch=wide-bf16x1")
                                            : " range-sketch=fp32";
        char line[256];
        snprintf(line, sizeof(line), "mode %d: I=%lld L=%d J=%lld T=%lld sketch=%s power=%s ttm=%s%s%s\n", n,
                 (long long)mp.v.i, mp.L, (long long)mp.v.fibers(), (long long)mp.T,
                 mp.mv.lf == 1 ? "contiguous" : "strided",
                 mp.half ? (mp.half_tc ? "wide-split-bf16" : p.elem == 8 ? "fp64" : "fp32") : power, ttm,
                 range, mp.half ? " amm=half-steps" : p.form == TUCKER_FORM_RELATED ? " factor=related" : "");
        text += line;
        if (!p.st) e[n] = ranks[n];
    }
    if (text.size() >= buf_bytes) return TUCKER_ERR_INVALID_ARG;
    memcpy(buf, text.c_str(), text.size() + 1);
    return TUCKER_OK;
}

const char* tucker_status_string(tucker_status s) {
    switch (s) {
        case TUCKER_OK: return "ok";
        case TUCKER_ERR_INVALID_ARG: return "invalid argument";
        case TUCKER_ERR_OOM: return "out of device memory";
        case TUCKER_ERR_CUDA: return "CUDA error";
        case TUCKER_ERR_NUMERICAL: return "numerical failure (non-finite values or unrepaired breakdown)";
        case TUCKER_ERR_TIMEOUT: return "a bounded device wait timed out";
        case TUCKER_ERR_UNSUPPORTED: return "request outside the supported sizes or options";
        case TUCKER_ERR_BUDGET: return "request larger than the memory budget";
    }
    return "unknown status";
}

const char* tucker_last_cuda_error(void) {
    static thread_local char buf[256];
    const cudaError_t e = g_last_cuda_error;
    snprintf(buf, sizeof(buf), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return buf;
}

tucker_status tucker_last_device_status(void) {
    if (!g_async_status) return TUCKER_OK;
    return sync_status(g_async_stream, g_async_status);
}

tucker_status tucker_gaussian(void* out, tucker_dtype dt, int64_t rows, int64_t cols, uint64_t seed,
                              uint32_t stream_id, const tucker_opts* opts) {
    Opts o;
    if (read_opts(opts, o) != TUCKER_OK) return TUCKER_ERR_INVALID_ARG;
    if (!out || rows < 0 || cols < 0 || (dt != TUCKER_F32 && dt != TUCKER_F64)) return TUCKER_ERR_INVALID_ARG;
    if (!on_device(out)) return TUCKER_ERR_INVALID_ARG;
    cudaError_t e = dt == TUCKER_F32 ? launch_gaussian<float>((float*)out, rows, cols, seed, stream_id, o.stream)
                                     : launch_gaussian<double>((double*)out, rows, cols, seed, stream_id, o.stream);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, nullptr);
}

tucker_status tucker_power_step(const void* A, tucker_dtype dt, const int64_t* dims, int N, int mode,
                                const void* X_in, int64_t L, void* X_out, const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!mode_args_ok(A, dims, N, mode) || !X_in || !X_out || L < 1) return TUCKER_ERR_INVALID_ARG;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    TuneAllow tune((o.flags & TUCKER_FLAG_ASYNC) == 0);
    const ModeView v = view_of(dims, N, mode);
    const int elem = dt == TUCKER_F64 ? 8 : 4;
    if (v.i > kMaxI || L > 4096 || (elem == 8 && v.i > 512)) return TUCKER_ERR_UNSUPPORTED;
    const PowerPlan pp = power_plan(v, (int)L, elem, num_sms());
    if (o.prec != TUCKER_SK_FP32 && elem == 4 && wide_supported(v, L) &&
        !(o.prec == TUCKER_SK_TF32 ? power_tf32_supported(v, (int)L)
          : o.prec == TUCKER_SK_BF16X1 ? power_bf16x1_supported(v, (int)L)
                                       : power_tc_supported(v, (int)L))) {
        // beyond the fused kernels' tiles: two tensor-core passes
        Scratch sc;
        if ((rs = sc.get(wide_power_scratch_bytes(v, (int)L, num_sms()) + 256, o.stream)) != TUCKER_OK) return rs;
        int* status = reinterpret_cast<int*>(sc.p);
        cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), o.stream);
        if (e == cudaSuccess)
            e = launch_power_wide((const float*)A, v, (const float*)X_in, (int)L, (float*)X_out,
                                  o.prec != TUCKER_SK_BF16X1, false, 0, 0, reinterpret_cast<char*>(sc.p) + 256,
                                  status, num_sms(), o.stream);
        if (e == cudaErrorNotSupported) return TUCKER_ERR_UNSUPPORTED;
        if (e != cudaSuccess) return from_cuda(e);
        return sync_status(o.stream, status);
    }
    if (o.prec == TUCKER_SK_TF32 || o.prec == TUCKER_SK_BF16X1) {
        const bool tf = o.prec == TUCKER_SK_TF32;
        if (elem != 4 || !(tf ? power_tf32_supported(v, (int)L) : power_bf16x1_supported(v, (int)L)))
            return TUCKER_ERR_UNSUPPORTED;
        Scratch sc;
        if ((rs = sc.get(power_tc_partials_bytes(v, (int)L, num_sms()) + 256, o.stream)) != TUCKER_OK) return rs;
        int* status = reinterpret_cast<int*>(sc.p);
        cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), o.stream);
        if (e == cudaSuccess)
            e = (tf ? launch_power_tf32 : launch_power_bf16x1)((const float*)A, v, (const float*)X_in, (int)L,
                                                               (float*)X_out, reinterpret_cast<char*>(sc.p) + 256,
                                                               status, num_sms(), o.stream);
        if (e == cudaErrorNotSupported) return TUCKER_ERR_UNSUPPORTED;
        if (e != cudaSuccess) return from_cuda(e);
        return sync_status(o.stream, status);
    }
    if (o.prec == TUCKER_SK_BF16) {
        if (elem != 4 || !power_tc_supported(v, (int)L)) return TUCKER_ERR_UNSUPPORTED;
        Scratch sc;
        if ((rs = sc.get(power_tc_partials_bytes(v, (int)L, num_sms()) + 256, o.stream)) != TUCKER_OK) return rs;
        int* status = reinterpret_cast<int*>(sc.p);
        cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), o.stream);
        if (e == cudaSuccess)
            e = launch_power_tc((const float*)A, v, (const float*)X_in, (int)L, (float*)X_out,
                                reinterpret_cast<char*>(sc.p) + 256, status, num_sms(), o.stream);
        if (e != cudaSuccess) return from_cuda(e);
        return sync_status(o.stream, status);
    }
    Scratch sc;
    if ((rs = sc.get(power_partials_bytes(pp, v, (int)L, elem), o.stream)) != TUCKER_OK) return rs;
    cudaError_t e = elem == 4 ? launch_power<float>((const float*)A, v, (const float*)X_in, (int)L, (float*)X_out,
                                                    sc.p, pp, false, 0, 0, o.stream)
                              : launch_power<double>((const double*)A, v, (const double*)X_in, (int)L,
                                                     (double*)X_out, sc.p, pp, false, 0, 0, o.stream);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, nullptr);
}

tucker_status tucker_range_sketch(const void* A, tucker_dtype dt, const int64_t* dims, int N, int mode, int64_t L,
                                  uint64_t seed, void* Y, const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!mode_args_ok(A, dims, N, mode) || !Y || L < 1) return TUCKER_ERR_INVALID_ARG;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    const ModeView v = view_of(dims, N, mode);
    const int elem = dt == TUCKER_F64 ? 8 : 4;
    if (v.i > kMaxI || L > 4096 || (elem == 8 && v.i > 512)) return TUCKER_ERR_UNSUPPORTED;
    const uint32_t sid = stream_id(0, mode);
    if (o.prec != TUCKER_SK_FP32) {
        // Y = A_(n) Omega on the tensor cores, Omega generated inside the kernel
        if (elem != 4 || !wide_supported(v, L)) return TUCKER_ERR_UNSUPPORTED;
        Scratch sc;
        if ((rs = sc.get(wide_power_scratch_bytes(v, (int)L, num_sms()) + 256, o.stream)) != TUCKER_OK) return rs;
        int* status = reinterpret_cast<int*>(sc.p);
        cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), o.stream);
        if (e == cudaSuccess)
            e = launch_power_wide((const float*)A, v, nullptr, (int)L, (float*)Y, o.prec != TUCKER_SK_BF16X1, true,
                                  seed, sid, reinterpret_cast<char*>(sc.p) + 256, status, num_sms(), o.stream);
        if (e == cudaErrorNotSupported) return TUCKER_ERR_UNSUPPORTED;
        if (e != cudaSuccess) return from_cuda(e);
        return sync_status(o.stream, status);
    }
    const PowerPlan pp = power_plan(v, (int)L, elem, num_sms());
    Scratch sc;
    if ((rs = sc.get(power_partials_bytes(pp, v, (int)L, elem), o.stream)) != TUCKER_OK) return rs;
    cudaError_t e = elem == 4 ? launch_power<float>((const float*)A, v, nullptr, (int)L, (float*)Y, sc.p, pp, true,
                                                    seed, sid, o.stream)
                              : launch_power<double>((const double*)A, v, nullptr, (int)L, (double*)Y, sc.p, pp,
                                                     true, seed, sid, o.stream);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, nullptr);
}

tucker_status tucker_fiber_norms12(const void* A, tucker_dtype dt, const int64_t* dims, int N, double* w1,
                                   double* w2, const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (N < 2 || !mode_args_ok(A, dims, N, 1) || !w1 || !w2) return TUCKER_ERR_INVALID_ARG;
    if (!fiber_norms12_supported(dims[0])) return TUCKER_ERR_UNSUPPORTED;
    const int64_t rest = prod(dims, N) / (dims[0] * dims[1]);
    cudaError_t e = dt == TUCKER_F32 ? launch_fiber_norms12<float>((const float*)A, dims[0], dims[1], rest, w1, w2,
                                                                   o.stream)
                  : dt == TUCKER_F64 ? launch_fiber_norms12<double>((const double*)A, dims[0], dims[1], rest, w1, w2,
                                                                    o.stream)
                                     : cudaErrorInvalidValue;
    if (e == cudaErrorInvalidValue) return TUCKER_ERR_INVALID_ARG;
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, nullptr);
}

tucker_status tucker_fiber_norms123(const void* A, tucker_dtype dt, const int64_t* dims, int N, double* w1,
                                    double* w2, double* w3, const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (N != 3 || !mode_args_ok(A, dims, N, 2) || !w1 || !w2 || !w3) return TUCKER_ERR_INVALID_ARG;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    if (!fiber_norms123_supported(dims[0])) return TUCKER_ERR_UNSUPPORTED;
    const size_t need = fiber_norms123_scratch_bytes(dims[0], dims[1], dims[2]);
    Scratch sc;
    void* scr = o.workspace;
    if (scr) {
        if (o.workspace_bytes < need) return TUCKER_ERR_INVALID_ARG;
    } else {
        rs = sc.get(need, o.stream);
        if (rs != TUCKER_OK) return rs;
        scr = sc.p;
    }
    const cudaError_t e =
        dt == TUCKER_F32 ? launch_fiber_norms123<float>((const float*)A, dims[0], dims[1], dims[2], w1, w2, w3, scr,
                                                        o.stream)
                         : launch_fiber_norms123<double>((const double*)A, dims[0], dims[1], dims[2], w1, w2, w3, scr,
                                                         o.stream);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, nullptr);
}

tucker_status tucker_fiber_norms123_workspace_size(const int64_t* dims, int N, size_t* bytes) {
    if (!dims || !bytes || N != 3 || dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return TUCKER_ERR_INVALID_ARG;
    if (!fiber_norms123_supported(dims[0])) return TUCKER_ERR_UNSUPPORTED;
    *bytes = fiber_norms123_scratch_bytes(dims[0], dims[1], dims[2]);
    return TUCKER_OK;
}

tucker_status tucker_fiber_norms(const void* A, tucker_dtype dt, const int64_t* dims, int N, int mode, double* w,
                                 const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!mode_args_ok(A, dims, N, mode) || !w) return TUCKER_ERR_INVALID_ARG;
    const ModeView v = view_of(dims, N, mode);
    cudaError_t e = dt == TUCKER_F32 ? launch_fiber_norms<float>((const float*)A, v, w, o.stream)
                  : dt == TUCKER_F64 ? launch_fiber_norms<double>((const double*)A, v, w, o.stream)
                                     : cudaErrorInvalidValue;
    if (e == cudaErrorInvalidValue) return TUCKER_ERR_INVALID_ARG;
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, nullptr);
}

tucker_status tucker_quantize_weights(const double* w, int64_t J, tucker_prob prob, uint64_t* W,
                                      const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!w || !W || J < 1) return TUCKER_ERR_INVALID_ARG;
    if (prob != TUCKER_PROB_NEARLY_OPTIMAL && prob != TUCKER_PROB_UNIFORM) return TUCKER_ERR_INVALID_ARG;
    Scratch sc;
    if ((rs = sc.get(quantize_scratch_bytes(J), o.stream)) != TUCKER_OK) return rs;
    cudaError_t e = launch_quantize(w, J, prob, W, sc.p, o.stream);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, nullptr);
}

tucker_status tucker_sample_fibers(const uint64_t* W, int64_t J, int64_t T, uint64_t seed, int mode, int64_t* idx,
                                   double* scale, const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!W || J < 1 || T < 0 || (T > 0 && (!idx || !scale)) || mode < 0 || mode > 255) return TUCKER_ERR_INVALID_ARG;
    Scratch sc;
    if ((rs = sc.get(sample_scratch_bytes(J), o.stream)) != TUCKER_OK) return rs;
    cudaError_t e = launch_sample(W, J, T, seed, stream_id(1, mode), idx, scale, sc.p, o.stream);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, nullptr);
}

tucker_status tucker_gather_fibers(const void* A, tucker_dtype dt, const int64_t* dims, int N, int mode,
                                   const int64_t* idx, const double* scale, int64_t T, void* Cp,
                                   const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!mode_args_ok(A, dims, N, mode) || T < 0 || (T > 0 && (!idx || !scale || !Cp))) return TUCKER_ERR_INVALID_ARG;
    const ModeView v = view_of(dims, N, mode);
    cudaError_t e = dt == TUCKER_F32 ? launch_gather<float>((const float*)A, v, idx, scale, T, (float*)Cp, o.stream)
                  : dt == TUCKER_F64 ? launch_gather<double>((const double*)A, v, idx, scale, T, (double*)Cp, o.stream)
                                     : cudaErrorInvalidValue;
    if (e == cudaErrorInvalidValue) return TUCKER_ERR_INVALID_ARG;
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, nullptr);
}

// ------------------------------------------------------------------ steps of a sharded call
tucker_status tucker_quantize_weights_max(const double* w, int64_t J, double wmax, uint64_t* W,
                                          const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!w || !W || J < 1 || !(wmax >= 0.0)) return TUCKER_ERR_INVALID_ARG;
    cudaError_t e = launch_quantize_max(w, J, wmax, W, o.stream);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, nullptr);
}

tucker_status tucker_sample_fibers_slab(const uint64_t* W, int64_t J, int64_t T, uint64_t seed, int mode,
                                        uint64_t S_offset, uint64_t S_total, int64_t fiber_offset, int64_t* idx,
                                        double* scale, const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!W || J < 1 || T < 0 || (T > 0 && (!idx || !scale)) || mode < 0 || mode > 255 || S_total == 0 ||
        S_offset >= S_total || fiber_offset < 0)
        return TUCKER_ERR_INVALID_ARG;
    Scratch sc;
    if ((rs = sc.get(sample_scratch_bytes(J), o.stream)) != TUCKER_OK) return rs;
    cudaError_t e = launch_sample_slab(W, J, T, seed, stream_id(1, mode), S_offset, S_total, fiber_offset, idx, scale,
                                       sc.p, o.stream);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, nullptr);
}

tucker_status tucker_cholqr(const void* X, tucker_dtype dt, int64_t I, int64_t L, void* Q, double* F,
                            const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!X || !Q || !F || X == Q || I < 1 || L < 1 || L > I) return TUCKER_ERR_INVALID_ARG;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    if (L > kMaxL) return TUCKER_ERR_UNSUPPORTED;
    const int elem = dt == TUCKER_F64 ? 8 : 4;
    const OrthPlan op = orth_plan(I, (int)L, num_sms());
    Scratch sc;
    if ((rs = sc.get(256 + orth_scratch_bytes(op, elem), o.stream)) != TUCKER_OK) return rs;
    int* status = (int*)sc.p;
    void* orth = (char*)sc.p + 256;
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), o.stream);
    if (e == cudaSuccess)
        e = elem == 4 ? launch_cholqr<float>((const float*)X, (float*)Q, op, F, orth, status, o.stream)
                      : launch_cholqr<double>((const double*)X, (double*)Q, op, F, orth, status, o.stream);
    if (e == cudaErrorInvalidValue) return TUCKER_ERR_UNSUPPORTED;
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, status);
}

tucker_status tucker_leading_factor_chain(const void* X, tucker_dtype dt, int64_t I, int64_t L, int64_t R,
                                          const double* factors, int nfactors, void* U, const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!X || !U || I < 1 || L < 1 || R < 1 || R > L || L > I || nfactors < 0 || nfactors > 64 ||
        (nfactors > 0 && !factors))
        return TUCKER_ERR_INVALID_ARG;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    if (L > kMaxL) return TUCKER_ERR_UNSUPPORTED;
    const int elem = dt == TUCKER_F64 ? 8 : 4;
    const OrthPlan op = orth_plan(I, (int)L, num_sms());
    if (!orth_supported(op, (int)R, elem)) return TUCKER_ERR_UNSUPPORTED;
    const size_t slot = (size_t)L * L;
    Arena a;
    a.take(sizeof(int) * 64);
    a.take(orth_scratch_bytes(op, elem));
    a.take((size_t)I * L * elem);
    a.take(sizeof(double) * slot * (size_t)(nfactors + 1));
    Scratch sc;
    if ((rs = sc.get(a.used, o.stream)) != TUCKER_OK) return rs;
    Arena b;
    b.base = (char*)sc.p;
    b.cap = a.used;
    int* status = (int*)b.take(sizeof(int) * 64);
    void* orth = b.take(orth_scratch_bytes(op, elem));
    void* Q1 = b.take((size_t)I * L * elem);
    double* F = (double*)b.take(sizeof(double) * slot * (size_t)(nfactors + 1));
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), o.stream);
    if (e == cudaSuccess && nfactors > 0)
        e = cudaMemcpyAsync(F, factors, sizeof(double) * slot * (size_t)nfactors, cudaMemcpyDeviceToDevice, o.stream);
    if (e == cudaSuccess)
        e = elem == 4 ? launch_extract<float>((const float*)X, (float*)Q1, op, F, nfactors, (int)R, (float*)U, orth,
                                              status, o.stream)
                      : launch_extract<double>((const double*)X, (double*)Q1, op, F, nfactors, (int)R, (double*)U,
                                               orth, status, o.stream);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, status);
}

tucker_status tucker_gram(const void* A, tucker_dtype dt, const int64_t* dims, int N, int mode, void* G,
                          const tucker_opts* opts) {
    cudaGetLastError();
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!mode_args_ok(A, dims, N, mode) || !G) return TUCKER_ERR_INVALID_ARG;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    const ModeView v = view_of(dims, N, mode);
    if (dt != TUCKER_F32 || o.prec == TUCKER_SK_FP32 || !gram_wide_supported(v)) return TUCKER_ERR_UNSUPPORTED;
    Scratch sc;
    if ((rs = sc.get(gram_wide_scratch_bytes(v, num_sms()) + 256, o.stream)) != TUCKER_OK) return rs;
    int* status = reinterpret_cast<int*>(sc.p);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), o.stream);
    if (e == cudaSuccess)
        e = launch_gram_wide((const float*)A, v, (float*)G, true, reinterpret_cast<char*>(sc.p) + 256, status,
                             num_sms(), o.stream);
    if (e == cudaErrorNotSupported) return TUCKER_ERR_UNSUPPORTED;
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, status);
}

tucker_status tucker_check_wait_timeout(int32_t iters, const tucker_opts* opts) {
    cudaGetLastError();
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (iters < 1 || iters > (1 << 24)) return TUCKER_ERR_INVALID_ARG;
    Scratch sc;
    if ((rs = sc.get(256, o.stream)) != TUCKER_OK) return rs;
    cudaError_t e = cudaMemsetAsync(sc.p, 0, sizeof(int), o.stream);
    if (e == cudaSuccess) e = launch_wait_timeout(iters, (int*)sc.p, o.stream);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, (const int*)sc.p);
}

tucker_status tucker_rsthosvd_adaptive(const void* A, tucker_dtype dt, const int64_t* dims, int N, double eps,
                                       int32_t q, int32_t L0, uint64_t seed, void* const* U, void* G, int32_t* ranks,
                                       const tucker_opts* opts) {
    cudaGetLastError();
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    if (!A || !dims || !U || !G || !ranks || N < 1 || N > kMaxOrder) return TUCKER_ERR_INVALID_ARG;
    if (!(eps >= 0.0) || !std::isfinite(eps) || q < 1 || L0 < 1) return TUCKER_ERR_INVALID_ARG;
    if ((o.flags & TUCKER_FLAG_ASYNC) || o.workspace) return TUCKER_ERR_INVALID_ARG;
    for (int n = 0; n < N; ++n)
        if (dims[n] < 1 || !U[n]) return TUCKER_ERR_INVALID_ARG;
    if (o.prec != TUCKER_SK_FP32 && dt != TUCKER_F32) return TUCKER_ERR_UNSUPPORTED;
    if (!on_device(A) || !on_device(G)) return TUCKER_ERR_INVALID_ARG;
    for (int n = 0; n < N; ++n)
        if (!on_device(U[n])) return TUCKER_ERR_INVALID_ARG;
    if (dt == TUCKER_F32)
        return adaptive_run<float>((const float*)A, dims, N, eps, q, L0, seed, o, (float* const*)U, (float*)G, ranks);
    return adaptive_run<double>((const double*)A, dims, N, eps, q, L0, seed, o, (double* const*)U, (double*)G,
                                ranks);
}

tucker_status tucker_sample_factor(const void* Cp, tucker_dtype dt, int64_t I, int64_t T, int64_t R, int32_t P,
                                   int32_t q, uint64_t seed, int mode, void* U, const tucker_opts* opts) {
    cudaGetLastError();
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!Cp || !U || I < 1 || T < 1 || R < 1 || R > I || P < 0 || q < 1 || mode < 0 || mode > 255)
        return TUCKER_ERR_INVALID_ARG;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    if (o.form != TUCKER_FORM_PAPER) return TUCKER_ERR_UNSUPPORTED;
    // the sample as the unfolding of an I x T matrix whose T fibers are all sampled
    const int elem = dt == TUCKER_F64 ? 8 : 4;
    const int64_t dims[2] = {I, T};
    const int32_t ranks[2] = {(int32_t)R, 1};
    Plan p;
    rs = make_plan(false, elem, dims, 2, ranks, P, q, T, o, p);
    if (rs != TUCKER_OK) return rs;
    Arena a;
    Work w;
    carve(p, a, w);
    Scratch sc;
    if ((rs = sc.get(a.used, o.stream)) != TUCKER_OK) return rs;
    Arena b;
    b.base = (char*)sc.p;
    b.cap = a.used;
    carve(p, b, w);
    cudaError_t e = cudaMemsetAsync(w.status, 0, sizeof(int), o.stream);
    if (e == cudaSuccess)
        e = elem == 4 ? sketch_factor<float>((const float*)Cp, p.m[0], mode, q, seed, TUCKER_FORM_PAPER, (float*)U, w,
                                             o.stream)
                      : sketch_factor<double>((const double*)Cp, p.m[0], mode, q, seed, TUCKER_FORM_PAPER,
                                              (double*)U, w, o.stream);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, w.status);
}

tucker_status tucker_leading_factor(const void* C, tucker_dtype dt, int64_t I, int64_t L, int64_t R, void* U,
                                    const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!C || !U || I < 1 || L < 1 || R < 1 || R > L || L > I) return TUCKER_ERR_INVALID_ARG;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    if (L > kMaxL) return TUCKER_ERR_UNSUPPORTED;
    const int elem = dt == TUCKER_F64 ? 8 : 4;
    const OrthPlan op = orth_plan(I, (int)L, num_sms());
    if (!orth_supported(op, (int)R, dt == TUCKER_F64 ? 8 : 4)) return TUCKER_ERR_UNSUPPORTED;
    Arena a;
    a.take(sizeof(int) * 64);
    a.take(orth_scratch_bytes(op, elem));
    a.take((size_t)I * L * elem);
    a.take(sizeof(double) * L * L);
    Scratch sc;
    if ((rs = sc.get(a.used, o.stream)) != TUCKER_OK) return rs;
    Arena b;
    b.base = (char*)sc.p;
    b.cap = a.used;
    int* status = (int*)b.take(sizeof(int) * 64);
    void* orth = b.take(orth_scratch_bytes(op, elem));
    void* Q1 = b.take((size_t)I * L * elem);
    double* F = (double*)b.take(sizeof(double) * L * L);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), o.stream);
    if (e == cudaSuccess)
        e = elem == 4 ? launch_extract<float>((const float*)C, (float*)Q1, op, F, 0, (int)R, (float*)U, orth, status,
                                              o.stream)
                      : launch_extract<double>((const double*)C, (double*)Q1, op, F, 0, (int)R, (double*)U, orth,
                                               status, o.stream);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, status);
}

tucker_status tucker_ttm(const void* A, tucker_dtype dt, const int64_t* dims, int N, int mode, const void* M_ptr,
                         int64_t K, int transpose, void* out, const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!mode_args_ok(A, dims, N, mode) || !M_ptr || !out || K < 1) return TUCKER_ERR_INVALID_ARG;
    const ModeView v = view_of(dims, N, mode);
    // M(k, i): transpose == 0: M_ptr is K x I_n (col-major) -> M_ptr[k + i K]
    //          transpose == 1: M_ptr is I_n x K               -> M_ptr[i + k I_n]
    const int64_t ld_i = transpose ? 1 : K, ld_k = transpose ? v.i : 1;
    TuneAllow tune(true);
    Scratch sc;
    const bool wide =
        o.prec != TUCKER_SK_FP32 && dt == TUCKER_F32 && !ttm_tc_supported(v, K) && wide_ttm_supported(v, K);
    if ((rs = sc.get(256 + (wide ? wide_ttm_scratch_bytes(v, K) : 0), o.stream)) != TUCKER_OK) return rs;
    if (cudaMemsetAsync(sc.p, 0, sizeof(int), o.stream) != cudaSuccess) return from_cuda(cudaGetLastError());
    if (o.prec != TUCKER_SK_FP32) {
        if (dt != TUCKER_F32) return TUCKER_ERR_UNSUPPORTED;
        const cudaError_t e =
            wide ? launch_ttm_wide((const float*)A, v, (const float*)M_ptr, K, ld_i, ld_k, (float*)out,
                                   reinterpret_cast<char*>(sc.p) + 256, (int*)sc.p, num_sms(), o.stream)
                 : launch_ttm_tc((const float*)A, v, (const float*)M_ptr, K, ld_i, ld_k, (float*)out, (int*)sc.p,
                                 num_sms(), o.stream);
        if (e == cudaErrorNotSupported) return TUCKER_ERR_UNSUPPORTED;
        if (e != cudaSuccess) return from_cuda(e);
        return sync_status(o.stream, (const int*)sc.p);
    }
    cudaError_t e = dt == TUCKER_F32 ? launch_ttm<float>((const float*)A, v, (const float*)M_ptr, K, ld_i, ld_k,
                                                         (float*)out, o.stream, (int*)sc.p)
                  : dt == TUCKER_F64 ? launch_ttm<double>((const double*)A, v, (const double*)M_ptr, K, ld_i, ld_k,
                                                          (double*)out, o.stream)
                                     : cudaErrorInvalidValue;
    if (e == cudaErrorInvalidValue) return TUCKER_ERR_INVALID_ARG;
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(o.stream, (const int*)sc.p);
}

tucker_status tucker_relative_error(const void* A, tucker_dtype dt, const int64_t* dims, int N, const int32_t* ranks,
                                    void* const* U, const void* G, double* re, const tucker_opts* opts) {
    Opts o;
    tucker_status rs = read_opts(opts, o);
    if (rs != TUCKER_OK) return rs;
    if (!A || !dims || !ranks || !U || !G || !re || N < 1 || N > kMaxOrder) return TUCKER_ERR_INVALID_ARG;
    if (dt != TUCKER_F32 && dt != TUCKER_F64) return TUCKER_ERR_INVALID_ARG;
    for (int n = 0; n < N; ++n)
        if (dims[n] < 1 || ranks[n] < 1 || ranks[n] > dims[n] || !U[n]) return TUCKER_ERR_INVALID_ARG;
    const int elem = dt == TUCKER_F64 ? 8 : 4;
    const int64_t E = prod(dims, N);
    // expand G x_1 U_1 ... x_N U_N through two buffers of at most E elements
    Arena a;
    a.take((size_t)E * elem); a.take((size_t)E * elem); a.take(sumsq_scratch_bytes()); a.take(sizeof(double) * 2);
    Scratch sc;
    if ((rs = sc.get(a.used, o.stream)) != TUCKER_OK) return rs;
    Arena b;
    b.base = (char*)sc.p;
    b.cap = a.used;
    void* buf[2] = {b.take((size_t)E * elem), b.take((size_t)E * elem)};
    void* ss = b.take(sumsq_scratch_bytes());
    double* nrm = (double*)b.take(sizeof(double) * 2);
    int64_t e_[kMaxOrder];
    for (int n = 0; n < N; ++n) e_[n] = ranks[n];
    const void* cur = G;
    cudaError_t e = cudaSuccess;
    for (int n = 0; n < N && e == cudaSuccess; ++n) {
        const ModeView v = view_of(e_, N, n);
        // out = cur x_n U_n, M(k = i_out, i = r) = U[i_out + r I_n]
        void* dst = buf[n & 1];
        e = elem == 4 ? launch_ttm<float>((const float*)cur, v, (const float*)U[n], dims[n], dims[n], 1, (float*)dst,
                                          o.stream)
                      : launch_ttm<double>((const double*)cur, v, (const double*)U[n], dims[n], dims[n], 1,
                                           (double*)dst, o.stream);
        e_[n] = dims[n];
        cur = dst;
    }
    if (e == cudaSuccess)
        e = elem == 4 ? launch_sumsq<float>((const float*)A, (const float*)cur, E, &nrm[0], ss, o.stream)
                      : launch_sumsq<double>((const double*)A, (const double*)cur, E, &nrm[0], ss, o.stream);
    if (e == cudaSuccess)
        e = elem == 4 ? launch_sumsq<float>((const float*)A, nullptr, E, &nrm[1], ss, o.stream)
                      : launch_sumsq<double>((const double*)A, nullptr, E, &nrm[1], ss, o.stream);
    double h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, o.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(o.stream);
    if (e != cudaSuccess) return from_cuda(e);
    *re = h[1] > 0 ? sqrt(h[0] / h[1]) : 0.0;
    return TUCKER_OK;
}

}  // extern "C"
