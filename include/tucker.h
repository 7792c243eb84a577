/*
 * tucker.h - C ABI of the GB300 (sm_103a) randomized Tucker library.
 *
 * Che, Wei, Yan, "Efficient algorithms for Tucker decomposition via
 * approximate matrix multiplication" (arXiv 2303.11612).
 *
 * Problem 1 (Section 1): given a tensor A of size I_1 x ... x I_N and target
 * multilinear ranks R_n (the paper's mu_n), find orthonormal U_n (I_n x R_n)
 * and the core G = A x_1 U_1^T ... x_N U_N^T (R_1 x ... x R_N).
 *
 * Conventions shared by every entry point
 *  - Tensors are dense, element (i_1, ..., i_N) at offset
 *    i_1 + I_1 (i_2 + I_2 (i_3 + ...)) (i_1 fastest), the order implied by the
 *    mode-n unfolding of Section 2. Mode indices are 0-based (mode 0 = the
 *    paper's mode 1). Matrices are column-major with leading dimension = rows.
 *  - The mode-n unfolding A_(n) is I_n x J_n with J_n = prod_{m != n} I_m; its
 *    column j = i_1 + I_1 (i_2 + ...) over the modes m != n in increasing order
 *    (Section 2). It is never materialised.
 *  - Pointers may be device or host memory (the library asks the CUDA driver):
 *    host buffers are staged through device copies inside the call. All
 *    buffers are owned by the caller; the library keeps no pointer after the
 *    call returns. A is never written.
 *  - Work is issued on opts->stream (NULL = the legacy default stream). Unless
 *    TUCKER_FLAG_ASYNC is set the call synchronises that stream before it
 *    returns and reports device-side failures (Cholesky breakdown that could not
 *    be repaired, non-finite values) in its status. With TUCKER_FLAG_ASYNC the
 *    call returns after enqueueing; the device status is then read by
 *    tucker_last_device_status(), or directly: the first 4 bytes of the
 *    caller's workspace hold it (0 = success; bit 0 numerical failure, bit 1 a
 *    bounded wait timed out) once the stream reaches the end of the call's
 *    work. An asynchronous call requires device buffers and a caller
 *    workspace, makes no allocation or synchronisation, and can therefore be
 *    captured into a CUDA graph.
 *  - Scratch memory: opts->workspace / workspace_bytes (device memory of at
 *    least tucker_workspace_size() bytes, 256-byte aligned) when given;
 *    otherwise the library allocates it from the stream-ordered pool and frees
 *    it before returning.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit
 *    seed, counter (block_lo, block_hi, stream, 0) with stream = purpose << 8 |
 *    mode; purpose 0 = Gaussian test matrix, 1 = fiber-sampling uniforms. A
 *    word x maps to u = ((x >> 9) + 0.5) 2^-23 in (0, 1); Gaussian element e
 *    uses block e / 4, lane e % 4 and Box-Muller on the lane pairs (0,1), (2,3).
 *  - Errors: argument errors are detected before any launch and return
 *    TUCKER_ERR_INVALID_ARG without side effects.
 */
#ifndef TUCKER_H
#define TUCKER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TUCKER_OK = 0,
    TUCKER_ERR_INVALID_ARG = 1,
    TUCKER_ERR_OOM = 2,
    TUCKER_ERR_CUDA = 3,
    TUCKER_ERR_NUMERICAL = 4,   /* non-finite values, or a breakdown not repaired */
    TUCKER_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
    TUCKER_ERR_UNSUPPORTED = 6, /* valid request outside what is built (e.g. a size limit) */
    TUCKER_ERR_BUDGET = 7       /* serving: request larger than the memory budget */
} tucker_status;

/* Sampling probabilities for approximate matrix multiplication (remark after
 * Algorithm 3): nearly-optimal p_j proportional to ||fiber_j||^2 (the optimal
 * probabilities for A_(n) A_(n)^T), or uniform p_j = 1 / J_n. */
typedef enum { TUCKER_PROB_NEARLY_OPTIMAL = 0, TUCKER_PROB_UNIFORM = 1 } tucker_prob;

/* Element type of tensors, factors and the core. With TUCKER_F64 every step
 * computes in FP64. With TUCKER_F32 the sketch and the mode-n products compute
 * in FP32 (or the tensor-core form opts->prec selects); the orthonormalisation
 * sums its Gram matrices of exact FP32 products in FP32 pairs and does the small
 * triangular algebra (Cholesky, inverses, triangle products) in double-float,
 * two FP32 words (about 2^-47); the small SVD is a QR with column pivoting
 * (Householder, FP32 with paired dot products) followed by a one-sided Jacobi
 * in FP32 with its coupling sums in FP32 pairs (tucker_leading_factor). */
typedef enum { TUCKER_F32 = 0, TUCKER_F64 = 1 } tucker_dtype;

/* Which sketch is taken.
 *  PAPER (default): C_n = (A_(n) A_(n)^T)^q Omega_n, Omega_n I_n x L_n Gaussian
 *    (Algorithms 1, 2, 4, 5; Strategy A of the remark after Algorithm 1).
 *  RANGE: Y = A_(n) Omega with Omega J_n x L_n, then q times
 *    Y = A_(n) (A_(n)^T orth(Y)) (the form the introduction contrasts, item (c)).
 * Either way U_n = the R_n leading left singular vectors of the sketch (remark
 * after Algorithm 5), each column's largest-magnitude entry made positive.
 *  RELATED: Algorithms 6 and 7 (the related forms of Algorithms 1 and 2): the
 *    paper form's C_n, its thin QR C_n = P_n R, U = the R_n leading left singular
 *    vectors of P_n^T A_(n), and the factor Q_n = P_n U with the sign rule; one
 *    more pass over the mode's tensor per mode. Without AMM only (c = 0, alpha = 0,
 *    else TUCKER_ERR_UNSUPPORTED). */
typedef enum { TUCKER_FORM_PAPER = 0, TUCKER_FORM_RANGE = 1, TUCKER_FORM_RELATED = 2 } tucker_form;

/* Arithmetic of the sketch / power products.
 *  FP32: exact FP32 FMA on the CUDA cores.
 *  TF32: tcgen05 tensor cores, kind::tf32, FP32 accumulation: A is read once by
 *    TMA, in FP32, straight into the tensor cores' operand layout, which use its
 *    top 19 bits (TF32, about 2^-11 relative), as for X and A^T X. Used for
 *    contiguous fibers (mode 1, or an AMM sample) with I_n % 4 == 0,
 *    I_n <= 512, L_n <= 32 and A 16-byte aligned; other modes take the BF16
 *    form where it fits, else FP32. tucker_power_step returns
 *    TUCKER_ERR_UNSUPPORTED outside those limits.
 *  BF16: tcgen05 tensor cores with FP32 accumulation, split form: A and the
 *    intermediate A^T X are each held as a bf16 high part plus a bf16 low part
 *    (about 16 significant bits), so the sketch is of A itself; A is still read
 *    once, in FP32. One fused pass where I_n <= 512 and L_n <= 64; beyond that
 *    (I_n <= 1024, L_n <= 128) two passes, W = A^T X then A W, on contiguous
 *    fibers or strides that are multiples of 32; other modes run FP32.
 *  BF16X1: tcgen05 tensor cores, kind::f16, single pass: A, X and A^T X each
 *    rounded to bf16 once (8 significant bits, to nearest), FP32 accumulation;
 *    the sketch is then good to about 2^-8, which the power steps win back
 *    (the factors' subspace moves by an angle of that order, the relative
 *    error of the decomposition only to second order). A is read once by TMA,
 *    in FP32. Used for sketches of the input tensor (every mode of T-HOSVD,
 *    the first of ST-HOSVD) on contiguous fibers (mode 0, or an AMM sample)
 *    and on strided fibers with Lf = I_1 ... I_{n-1} >= 64 and Lf % 4 == 0,
 *    where I_n % 4 == 0, I_n <= 512, L_n <= 32 and A is 16-byte aligned, and
 *    in the two-pass kernels beyond (contiguous fibers, I_n <= 1024);
 *    ST-HOSVD's later modes (on the truncated tensor, small by then) and other
 *    shapes take the BF16 form where it fits, else FP32.
 * In every tensor-core form, q >= 2 power steps in the paper form on a mode with
 * I_n <= 128 take Strategy B (tucker_gram: one pass for A_(n) A_(n)^T in split
 * bf16, then its powers) where the tensor-core kernels take the layout, and the
 * mode products run in split BF16 (see tucker_ttm). The tensor-core forms need
 * FP32 data (TUCKER_ERR_UNSUPPORTED for FP64). */
typedef enum { TUCKER_SK_FP32 = 0, TUCKER_SK_TF32 = 1, TUCKER_SK_BF16 = 2, TUCKER_SK_BF16X1 = 3 } tucker_sketch_prec;

#define TUCKER_FLAG_ASYNC 0x1u
/* tucker_batch_run only: run the batch through the work-list kernel (see the
 * batches section). */
#define TUCKER_FLAG_WORKLIST 0x2u

typedef struct {
    uint32_t struct_size;   /* sizeof(tucker_opts) */
    int32_t form;           /* tucker_form */
    int32_t prec;           /* tucker_sketch_prec */
    uint32_t flags;         /* TUCKER_FLAG_* */
    double alpha;           /* T_n = ceil(alpha J_n) when c == 0 and alpha > 0 (Section 3.3) */
    void* stream;           /* cudaStream_t; NULL = legacy default stream */
    void* workspace;        /* device scratch, may be NULL */
    size_t workspace_bytes;
    double* rel_error;      /* host out, may be NULL: RE = sqrt(1 - ||G||^2/||A||^2) (Eq. 8) */
    int64_t* const* sample_idx; /* may be NULL: N device/host arrays receiving the T_n
                                   sampled fiber indices of each mode (AMM only) */
} tucker_opts;

/* ---------------------------------------------------------------- drivers */

/* Randomized T-HOSVD with the power scheme: Algorithm 1 (c == 0 and alpha == 0)
 * or Algorithm 4 (c > 0: T_n = min(c, J_n) fibers of A_(n) sampled, Section 3.2).
 *   A      : tensor, dims[0] x ... x dims[N-1], element type dt (read only)
 *   dims   : host array of N extents, 1 <= N <= 8
 *   ranks  : host array of N target ranks, 1 <= R_n <= I_n
 *   P      : oversampling (the paper's K), >= 0; L_n = min(R_n + P, I_n)
 *   q      : power steps, >= 1
 *   c      : AMM sample count (0 = no sampling)
 *   prob   : sampling probabilities (ignored when no sampling)
 *   seed   : Philox key
 *   U      : host array of N pointers, U[n] receives I_n x R_n (column-major)
 *   G      : receives the R_1 x ... x R_N core (r_1 fastest)
 *   opts   : may be NULL (defaults: paper form, FP32 sketch, synchronous) */
tucker_status tucker_rthosvd(const void* A, tucker_dtype dt, const int64_t* dims, int N,
                             const int32_t* ranks, int32_t P, int32_t q, int64_t c,
                             tucker_prob prob, uint64_t seed, void* const* U, void* G,
                             const tucker_opts* opts);

/* Randomized ST-HOSVD with the power scheme: Algorithm 2 (no sampling) or
 * Algorithm 5 (sampling), processing order 1..N (Section 4). After U_n the
 * working tensor becomes B x_n U_n^T; the last one is the core. Arguments as
 * for tucker_rthosvd; for mode n, J_n = R_1 ... R_{n-1} I_{n+1} ... I_N. */
tucker_status tucker_rsthosvd(const void* A, tucker_dtype dt, const int64_t* dims, int N,
                              const int32_t* ranks, int32_t P, int32_t q, int64_t c,
                              tucker_prob prob, uint64_t seed, void* const* U, void* G,
                              const tucker_opts* opts);

/* Fixed-precision problem (Problem 2, concluding section): multilinear ranks
 * r_n and orthonormal factors Q_n with
 *   ||A - A x_1 Q_1 Q_1^T ... x_N Q_N Q_N^T||_F <= eps ||A||_F,
 * by randomized ST-HOSVD in processing order 1..N. The energies the modes
 * discard add up exactly (each truncation projects the tensor the previous ones
 * left), so mode n may discard (eps^2 ||A||^2 - energy discarded so far) / (N - n)
 * (0-based n). Mode n sketches L columns (L = min(L0, I_n), doubled up to I_n)
 * in the form opts->form with q power steps and no oversampling beyond L, takes
 * all L leading left singular vectors U_L, the kept energies
 * e_k = ||u_k^T B_(n)||^2 from Y = B x_n U_L^T, and the smallest r_n whose
 * remainder ||B||^2 - (e_1 + ... + e_r) is within the mode's share; without one
 * the sketch is widened, and at L = I_n nothing is discarded. Q_n = U_L(:, 1:r_n)
 * and B becomes the first r_n slices of Y. Decisions are taken on the host in
 * FP64 from energies summed in FP64 on the device; the call is synchronous.
 *   A, dims, N, dt: the tensor (device memory)
 *   eps   : relative tolerance, finite, >= 0
 *   q     : power steps, >= 1; L0: first sketch width, >= 1
 *   U     : host array of N device pointers, U[n] with room for I_n x I_n
 *           elements; receives I_n x r_n (column-major)
 *   G     : device buffer with room for I_1 ... I_N elements; receives the
 *           r_1 x ... x r_N core (r_1 fastest)
 *   ranks : host array of N, receives r_n
 *   opts  : stream, prec, form, rel_error as for the drivers; the call
 *           allocates its scratch itself (stream-ordered) and takes neither
 *           opts->workspace nor TUCKER_FLAG_ASYNC (TUCKER_ERR_INVALID_ARG).
 * Host pointers where device memory is required give
 * TUCKER_ERR_INVALID_ARG; a sketch wider than the extraction supports (110
 * columns) before the tolerance is met gives TUCKER_ERR_UNSUPPORTED. */
tucker_status tucker_rsthosvd_adaptive(const void* A, tucker_dtype dt, const int64_t* dims, int N, double eps,
                                       int32_t q, int32_t L0, uint64_t seed, void* const* U, void* G,
                                       int32_t* ranks, const tucker_opts* opts);

/* Scratch bytes a driver call needs. which = 0 (T-HOSVD) or 1 (ST-HOSVD). */
tucker_status tucker_workspace_size(int which, tucker_dtype dt, const int64_t* dims, int N,
                                    const int32_t* ranks, int32_t P, int32_t q, int64_t c,
                                    const tucker_opts* opts, size_t* bytes);

/* The arithmetic a driver call with these arguments takes in each mode, as
 * text, without running it (host only; no GPU needed): one line per mode,
 *   "mode n: I=.. L=.. J=.. T=.. sketch=contiguous|strided power=F ttm=F"
 * (plus " range-sketch=F" in the range form), F one of bf16x1, tf32,
 * split-bf16, fp32, fp64 - the choice made for a 16-byte aligned tensor (a
 * misaligned one falls back to the next form; see tucker_sketch_prec). I, J:
 * extent and fibers of the tensor the mode works on; T: AMM samples (0 = none),
 * whose I x T gather is then the sketched matrix. Writes a zero-terminated
 * string into buf (256 bytes per mode suffice); returns the drivers' argument
 * errors, and TUCKER_ERR_INVALID_ARG when buf is too small. */
tucker_status tucker_plan_describe(int which, tucker_dtype dt, const int64_t* dims, int N,
                                   const int32_t* ranks, int32_t P, int32_t q, int64_t c,
                                   const tucker_opts* opts, char* buf, size_t buf_bytes);

const char* tucker_status_string(tucker_status s);

/* Name and description of the last CUDA error that made a call on this host
 * thread return TUCKER_ERR_CUDA or TUCKER_ERR_OOM (thread-local storage). */
const char* tucker_last_cuda_error(void);

/* Device status word of the last TUCKER_FLAG_ASYNC call on this host thread
 * (synchronises its stream first). */
tucker_status tucker_last_device_status(void);

/* ---------------------------------------------------------------- steps
 * One entry point per step of the path, for tests and for callers that build
 * their own pipelines. "mode view" arguments (A, dt, dims, N, mode) describe
 * the mode-n unfolding of a tensor as above. */

/* Gaussian test matrix (Algorithm 1, "generate a standard Gaussian matrix"):
 * out (rows x cols, column-major, dt) gets element (i, l) = Gaussian element
 * e = i * cols + l of Philox stream `stream_id` under `seed`. */
tucker_status tucker_gaussian(void* out, tucker_dtype dt, int64_t rows, int64_t cols,
                              uint64_t seed, uint32_t stream_id, const tucker_opts* opts);

/* One power step of Strategy A fused into a single pass over the tensor:
 * X_out = A_(n) (A_(n)^T X_in), X_in and X_out I_n x L column-major.
 * opts->prec selects the arithmetic (see tucker_sketch_prec): FP32 for every
 * mode view; TF32 for contiguous fibers (mode 0) and BF16X1 for contiguous or
 * wide-strided fibers, within their limits; BF16 (split) for I_n <= 512 and
 * L <= 64. Outside a form's limits the
 * call returns TUCKER_ERR_UNSUPPORTED (it never substitutes another form). */
tucker_status tucker_power_step(const void* A, tucker_dtype dt, const int64_t* dims, int N,
                                int mode, const void* X_in, int64_t L, void* X_out,
                                const tucker_opts* opts);

/* Range-form sketch Y = A_(n) Omega (Omega J_n x L Gaussian, element (j, l) =
 * e = j * L + l of stream (0 << 8 | mode)), Omega generated inside the kernel. */
tucker_status tucker_range_sketch(const void* A, tucker_dtype dt, const int64_t* dims, int N,
                                  int mode, int64_t L, uint64_t seed, void* Y,
                                  const tucker_opts* opts);

/* Squared fiber norms w_j = ||A_(n)(:, j)||^2, j < J_n (FP64 out; the sum is
 * carried in paired FP32 words or FP64, about 2^-44 relative). */
tucker_status tucker_fiber_norms(const void* A, tucker_dtype dt, const int64_t* dims, int N,
                                 int mode, double* w, const tucker_opts* opts);

/* The squared norms of the mode-1 and the mode-2 fibers (as tucker_fiber_norms
 * with mode 0 and 1) in one pass over A (N >= 2, I_1 <= 1024, else
 * TUCKER_ERR_UNSUPPORTED): w1 receives J_1 = I_2 ... I_N values, bitwise those
 * of tucker_fiber_norms for mode 0 when I_1 >= 64 (the same summation order);
 * w2 receives J_2 = I_1 I_3 ... I_N values, summed in a fixed order of its own
 * (within about 2^-44 relative of tucker_fiber_norms for mode 1). Algorithm 4
 * with the nearly-optimal probabilities samples modes 1 and 2 of the same
 * tensor; the T-HOSVD driver forms both from this pass. Not in the paper as a
 * separate step (a fusion of the remark after Algorithm 3's norms). */
tucker_status tucker_fiber_norms12(const void* A, tucker_dtype dt, const int64_t* dims, int N,
                                   double* w1, double* w2, const tucker_opts* opts);

/* All three modes' squared fiber norms of an order-3 tensor (N == 3, else
 * TUCKER_ERR_INVALID_ARG; I_1 <= 1024, else TUCKER_ERR_UNSUPPORTED) in one pass
 * over A: w1 (J_1 = I_2 I_3 values) bitwise those of tucker_fiber_norms for
 * mode 0 when I_1 >= 64; w2 (J_2 = I_1 I_3) and w3 (J_3 = I_1 I_2) summed from
 * partials over bands of rows and chunks of slabs in a fixed order (within
 * about 2^-44 relative of tucker_fiber_norms for modes 1 and 2). The partials
 * go to opts->workspace when it is set (device memory of
 * tucker_fiber_norms123_workspace_size bytes; fewer is TUCKER_ERR_INVALID_ARG),
 * else to a block the call allocates on opts->stream and frees. Algorithm 4
 * with the nearly-optimal probabilities samples every mode of the same tensor;
 * the T-HOSVD driver forms an order-3 tensor's three weight vectors from this
 * pass. Not in the paper as a separate step. */
tucker_status tucker_fiber_norms123(const void* A, tucker_dtype dt, const int64_t* dims, int N,
                                    double* w1, double* w2, double* w3, const tucker_opts* opts);
/* Device bytes of tucker_fiber_norms123's partials for dims (N == 3). */
tucker_status tucker_fiber_norms123_workspace_size(const int64_t* dims, int N, size_t* bytes);

/* Integer sampling weights W_j = ceil(w_j / max(w) * 2^24) (0 where w_j == 0;
 * all ones if every w_j is 0), or all ones for uniform probabilities. */
tucker_status tucker_quantize_weights(const double* w, int64_t J, tucker_prob prob,
                                      uint64_t* W, const tucker_opts* opts);

/* RANDSAMPLE(T, p) with p_j = W_j / S, S = sum W (Section 3.2): draw t uses the
 * 64-bit Philox word r_t of stream (1 << 8 | mode) (block t / 2; words (x0,x1)
 * for even t, (x2,x3) for odd t), v = floor(r_t S / 2^64), idx[t] = the least j
 * with W_0 + ... + W_j > v, scale[t] = 1 / sqrt(T W_idx / S). Bit-exact. */
tucker_status tucker_sample_fibers(const uint64_t* W, int64_t J, int64_t T, uint64_t seed,
                                   int mode, int64_t* idx, double* scale,
                                   const tucker_opts* opts);

/* C' = A_(n) S (Algorithms 4/5): column t of C' (I_n x T, column-major, dt) is
 * scale[t] times fiber idx[t]. idx and scale are device arrays of T entries;
 * every idx[t] must lie in [0, J_n) (tucker_sample_fibers' indices always do):
 * the kernel reads fiber idx[t] without checking it. */
tucker_status tucker_gather_fibers(const void* A, tucker_dtype dt, const int64_t* dims, int N,
                                   int mode, const int64_t* idx, const double* scale, int64_t T,
                                   void* Cp, const tucker_opts* opts);

/* U (I x R, column-major, dt) = the R leading left singular vectors of the
 * sketch C (I x L, column-major, dt), largest-magnitude entry of each column
 * positive (remark after Algorithm 5). CholeskyQR2 (shifted once when the Gram
 * matrix is numerically singular) with the small triangular algebra in
 * double-float (FP32 data) or FP64 (FP64 data), then a one-sided Jacobi SVD of
 * the triangular factor; a final CholeskyQR pass on U keeps it orthonormal
 * where the sketch is numerically rank-deficient. */
tucker_status tucker_leading_factor(const void* C, tucker_dtype dt, int64_t I, int64_t L,
                                    int64_t R, void* U, const tucker_opts* opts);

/* Mode-n product out = A x_n M (Section 2) with M given by M_ptr, a column-major
 * matrix: transpose == 0: M is K x I_n (out has K in mode n);
 *         transpose == 1: M_ptr holds I_n x K and M is its transpose
 *         (out = A x_n M_ptr^T, the truncation B x_n U^T of Algorithm 2).
 * opts->prec FP32 (default): exact FP32 / FP64 FMA. BF16 or TF32: tcgen05 tensor
 * cores with A and M each split into bf16 high and low parts, A_hi M_hi +
 * A_lo M_hi + A_hi M_lo accumulated in FP32 (about 2^-16 relative, unbiased);
 * contiguous fibers only (mode 0), FP32, I_n % 4 == 0, I_n <= 512, K <= 32, A
 * 16-byte aligned, else TUCKER_ERR_UNSUPPORTED. The drivers use this form for
 * the mode-0 product when their prec is BF16 or TF32 (FP32 FMA elsewhere). */
tucker_status tucker_ttm(const void* A, tucker_dtype dt, const int64_t* dims, int N, int mode,
                         const void* M_ptr, int64_t K, int transpose, void* out,
                         const tucker_opts* opts);

/* RE = ||A - G x_1 U_1 ... x_N U_N||_F / ||A||_F (Eq. 8) by explicit
 * reconstruction on the device; *re receives it (host pointer). */
tucker_status tucker_relative_error(const void* A, tucker_dtype dt, const int64_t* dims, int N,
                                    const int32_t* ranks, void* const* U, const void* G,
                                    double* re, const tucker_opts* opts);

/* ---------------------------------------------------------------- steps of a sharded call
 * The tensor partitioned into slabs along its last mode N, one slab per rank
 * (slab-sharded ST-HOSVD): for every mode n < N the sketch is the sum over the
 * slabs of their power-step outputs, and AMM samples the fibers of all slabs
 * together (Algorithm 5, RANDSAMPLE of Section 3.2). A slab's mode-n fibers are
 * consecutive global fibers (mode N is the most significant part of the fiber
 * index), so the global multinomial draws can be resolved slab by slab. These
 * entry points are the steps such a call needs beyond those above; the package's
 * sharded driver combines them with torch.distributed collectives. */

/* W_j = ceil(w_j / wmax * 2^24) for w_j > 0, else 0 (all ones when wmax is 0):
 * the integer weights of RANDSAMPLE (remark after Algorithm 3) with the largest
 * weight wmax taken over every slab. w, W: device arrays of J entries. */
tucker_status tucker_quantize_weights_max(const double* w, int64_t J, double wmax, uint64_t* W,
                                          const tucker_opts* opts);

/* The draws of RANDSAMPLE (Section 3.2) that fall in one slab: this slab holds
 * global fibers fiber_offset .. fiber_offset + J - 1 with weights W (device, J
 * entries) covering the range [S_offset, S_offset + sum W) of the global weight
 * total S_total. Draw t (same Philox word as tucker_sample_fibers) owned by
 * this slab gets its global fiber index in idx[t] and 1/sqrt(T p) in scale[t];
 * draws owned by other slabs get idx[t] = -1 and scale[t] = 0 (device arrays of
 * T entries). Over all slabs the result equals tucker_sample_fibers on the
 * concatenated weights, bit for bit. */
tucker_status tucker_sample_fibers_slab(const uint64_t* W, int64_t J, int64_t T, uint64_t seed, int mode,
                                        uint64_t S_offset, uint64_t S_total, int64_t fiber_offset, int64_t* idx,
                                        double* scale, const tucker_opts* opts);

/* One CholeskyQR pass X = Q F (X, Q: I x L column-major device arrays, I >= L,
 * not aliased): the orthonormalisation between power steps of the factored
 * power scheme (C_n = X_q F_{q-1} ... F_1, remark after Algorithm 1, Strategy
 * A). F: device array of L*L doubles receiving the packed upper triangle (FP64
 * for F64 data, double-float pairs for F32 data) as tucker_leading_factor_chain reads it. */
tucker_status tucker_cholqr(const void* X, tucker_dtype dt, int64_t I, int64_t L, void* Q, double* F,
                            const tucker_opts* opts);

/* U (I x R) = the R leading left singular vectors of C = X F_{nf-1} ... F_0
 * (remark after Algorithm 5), with the factors as written by tucker_cholqr
 * (device, nfactors slots of L*L doubles, F_0 first), sign-fixed as
 * tucker_leading_factor. */
tucker_status tucker_leading_factor_chain(const void* X, tucker_dtype dt, int64_t I, int64_t L, int64_t R,
                                          const double* factors, int nfactors, void* U, const tucker_opts* opts);

/* The factor of Algorithms 4/5 from a gathered sample: U (I x R) = the R
 * leading left singular vectors of (C' C'^T)^q Omega, C' (I x T, column-major
 * device array) the rescaled sampled fibers, Omega the mode's Gaussian
 * (L = min(R + P, I) columns, Philox stream of `mode`), evaluated as the drivers
 * evaluate it (in orthonormalised half steps when T >= L). Paper form only. */
tucker_status tucker_sample_factor(const void* Cp, tucker_dtype dt, int64_t I, int64_t T, int64_t R, int32_t P,
                                   int32_t q, uint64_t seed, int mode, void* U, const tucker_opts* opts);

/* Strategy B of the remark after Algorithm 1: G (I_n x I_n, column-major device
 * array) = A_(n) A_(n)^T in one pass over the tensor on the tensor cores, split
 * bf16 operands with FP32 accumulation (about 2^-16 per product), the partial
 * sums of a fixed set of CTAs added in a fixed order. FP32 data and a
 * tensor-core opts->prec (any; the Gram is always split bf16), I_n <= 128,
 * mode-1 fibers or strides that are multiples of 32, A 16-byte aligned;
 * otherwise TUCKER_ERR_UNSUPPORTED. The drivers take this route in the paper
 * form when q >= 2 and I_n <= 128 (one pass over the tensor instead of q), then
 * C_n = G^q Omega_n in the factored form. */
tucker_status tucker_gram(const void* A, tucker_dtype dt, const int64_t* dims, int N, int mode, void* G,
                          const tucker_opts* opts);

/* Checks the bounded-wait path of the tensor-core kernels on the device (no
 * counterpart in the paper): one CTA takes tensor memory, waits on an mbarrier
 * that nothing completes for `iters` polls (1 .. 2^24), records the timeout in
 * its status word exactly as the kernels do when a wait runs out, frees its
 * tensor memory and returns; nothing is in flight, so nothing is drained.
 * Returns TUCKER_ERR_TIMEOUT when that path works (the stream and the context
 * stay usable), TUCKER_ERR_INVALID_ARG for iters out of range. */
tucker_status tucker_check_wait_timeout(int32_t iters, const tucker_opts* opts);

/* ---------------------------------------------------------------- allocation-free variant
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory while they run (memory reserved once at start,
 * or hosts where cudaMalloc/cudaFree would stall other work).
 *
 * tucker_power_step_noalloc computes what tucker_power_step computes with
 * opts->prec TUCKER_SK_FP32 (X_out = A_(n) (A_(n)^T X_in) in exact FP32 or FP64
 * FMA arithmetic, same arguments and layouts) but takes its partial sums from a
 * fixed block of TUCKER_NOALLOC_SCRATCH_BYTES of device memory that belongs to
 * the library (held on every GPU that loads it until the process exits) and
 * calls no allocator. Only that arithmetic is served: another opts->prec gives
 * TUCKER_ERR_UNSUPPORTED; invalid options give TUCKER_ERR_INVALID_ARG as for
 * tucker_power_step. The first call on a device looks up the block's address
 * there (again after the device's context was recreated, e.g. by
 * cudaDeviceReset) and should come before any stream capture. Calls share the
 * block, so calls whose GPU work overlaps race; order them. Returns
 * TUCKER_ERR_UNSUPPORTED when one I_n x L partial (I_n * L * element size
 * bytes) exceeds the block, and otherwise the statuses of tucker_power_step;
 * it synchronises opts->stream before returning. */
#define TUCKER_NOALLOC_SCRATCH_BYTES (8u << 20)
tucker_status tucker_power_step_noalloc(const void* A, tucker_dtype dt, const int64_t* dims, int N,
                                        int mode, const void* X_in, int64_t L, void* X_out,
                                        const tucker_opts* opts);

/* ---------------------------------------------------------------- serving
 * Not part of the paper's method: a request loop for many decompositions of
 * different orders, sizes and ranks arriving over time. A server owns one
 * worker thread and max_inflight CUDA streams on the current device. Submitted
 * requests wait in FIFO order and are admitted when a stream is free and their
 * device memory (workspace, plus staging for host inputs and outputs) fits in
 * what the budget has left; each admitted request runs as a TUCKER_FLAG_ASYNC
 * decomposition on its own stream, so the work of admitted requests overlaps
 * on the device, and a request that arrives while others run is admitted as
 * soon as a stream and memory free up. Results do not depend on what else
 * runs: every kernel reduces in a fixed order. How far the streams overlap depends on CUDA's hardware work queues:
 * CUDA_DEVICE_MAX_CONNECTIONS (8 when unset, read
 * when the process creates its CUDA context) should be at least max_inflight,
 * or requests sharing a queue wait on one another. */
typedef struct tucker_server tucker_server;

typedef struct {
    uint32_t struct_size;   /* sizeof(tucker_server_opts) */
    int32_t max_inflight;   /* requests on the device at once (streams), 1 .. 256 */
    size_t budget_bytes;    /* device memory admitted requests may hold together */
    int32_t form;           /* tucker_form of every request */
    int32_t prec;           /* tucker_sketch_prec of every request */
    int32_t tick_max;       /* 0 or 1: every request on its own stream. 2 .. 256 (ticks: up to this
                               many consecutive requests at the head of the queue that the work
                               list takes, each of at most tick_elems elements, as one work-list
                               batch on one stream) returns TUCKER_ERR_UNSUPPORTED: the work-list
                               path is not run (see the batches section) */
    int64_t tick_elems;     /* the size limit of a tick's requests, elements (> 0 with ticks) */
} tucker_server_opts;

typedef struct {
    uint32_t struct_size;   /* sizeof(tucker_request) */
    int32_t which;          /* 0 = randomized T-HOSVD (Alg. 1/4), 1 = ST-HOSVD (Alg. 2/5) */
    tucker_dtype dt;
    const void* A;          /* host or device; must stay valid and unchanged until completion */
    const int64_t* dims;    /* N extents (copied at submission) */
    int32_t N;
    const int32_t* ranks;   /* N ranks (copied) */
    int32_t P, q;
    int64_t c;
    tucker_prob prob;
    uint64_t seed;
    void* const* U;         /* N host or device outputs (pointers copied), written by completion */
    void* G;                /* host or device core output */
} tucker_request;

typedef struct {
    uint64_t submitted, completed, failed;
    double p50_ms, p99_ms, mean_ms, max_ms; /* submission -> completion latency of completed requests */
    double throughput;      /* completed / (last completion - first submission), per second */
    size_t peak_bytes;      /* largest device memory held by admitted requests together */
    int32_t peak_inflight;  /* largest number of requests on the device together */
    uint64_t ticks;         /* work-list ticks launched */
    uint64_t tick_requests; /* requests admitted in them */
} tucker_server_stats;

/* Creates a server on the calling thread's current device. */
tucker_status tucker_server_create(const tucker_server_opts* opts, tucker_server** out);

/* Queues a request and returns at once with its ticket (1, 2, ...). Argument
 * errors are reported here; TUCKER_ERR_BUDGET when the request alone needs more
 * device memory than the budget. Any host thread may submit. */
tucker_status tucker_server_submit(tucker_server* srv, const tucker_request* req, uint64_t* ticket);

/* Waits up to timeout_ms (< 0: without limit, 0: poll) for a request. Returns
 * TUCKER_OK with the request's own status in *result once it has completed
 * (outputs written), TUCKER_ERR_TIMEOUT while it has not. */
tucker_status tucker_server_wait(tucker_server* srv, uint64_t ticket, int64_t timeout_ms,
                                 tucker_status* result);

tucker_status tucker_server_stats_get(tucker_server* srv, tucker_server_stats* out);

/* Waits for every submitted request, then releases the server. */
tucker_status tucker_server_destroy(tucker_server* srv);

/* ---------------------------------------------------------------- batches
 * Not part of the paper's method: many independent decompositions (Algorithms
 * 1, 2, 4, 5 with any shapes and parameters each) launched together as one CUDA
 * graph. The requests use the tucker_request layout with DEVICE buffers only.
 * The first call with a given signature - n, every request's fields and buffer
 * addresses, opts->form, opts->prec, the workspace pointer and size - captures
 * the requests' asynchronous launch sequences, each on its own stream, into one
 * graph; a later call with the same signature replays that graph with one
 * launch (the 16 most recently used graphs are kept). The graph runs after the
 * work already on opts->stream and before what is enqueued there next. Each
 * request's results are bitwise those of the same request run alone. The
 * requests overlap as far as CUDA's hardware work queues allow: with more than
 * 8 requests, set CUDA_DEVICE_MAX_CONNECTIONS (up to 32) before the process
 * creates its CUDA context.
 *
 * TUCKER_FLAG_WORKLIST: tucker_batch_run returns TUCKER_ERR_UNSUPPORTED
 * before any launch. The work-list path below is built and planned
 * (tucker_batch_describe, tucker_batch_workspace_size) but not run: in some
 * runs of a heterogeneous 32-request batch replayed back to back it raised an
 * illegal-address fault whose cause has not been found, so it is kept off the
 * device. As designed:
 * with TUCKER_FLAG_WORKLIST in opts->flags the graph holds a work list instead
 * of the requests' own launch sequences (many small tensors in few launches):
 * every stage of every request - Gaussian test matrix, power-step partials and
 * their fixed-order sum, mode products, status reset - becomes items, the
 * blocks its own kernel would run, and one persistent kernel launch per phase
 * claims the items of all requests (per mode: the truncation by U_{n-1} of
 * ST-HOSVD, the status reset and Omega_n; then per power step its partials and
 * their sums; last the cores, T-HOSVD's chain a phase per position). The items
 * of a phase are independent: what they read was written by an earlier phase,
 * so no CTA waits for another. The CholeskyQR passes and extractions of all
 * requests run as one grouped launch per step. The requests are dealt to up to
 * eight lanes (streams of the graph), so that one lane's orthonormalisations
 * overlap another's streaming phases. Each request's results are bitwise those
 * of the request run alone (with autotuning off, which can pick other FP32
 * power-step tiles). The work list takes Algorithms 1 and 2 in the paper form
 * with TUCKER_SK_FP32, no sampling (c = 0, alpha = 0), one element type across
 * the batch, every extent I_n <= 256 and every rank R_n <= 32; other batches
 * return TUCKER_ERR_UNSUPPORTED (from tucker_batch_workspace_size too, which
 * with the flag includes the work list's descriptor area). Not part of the
 * paper's method. */

/* Device workspace bytes (256-byte aligned per request) a batch needs; opts
 * may be NULL (paper form, FP32). */
tucker_status tucker_batch_workspace_size(int n, const tucker_request* reqs, const tucker_opts* opts,
                                          size_t* bytes);

/* Runs n >= 1 requests. opts is required: opts->workspace must be device
 * memory of tucker_batch_workspace_size() bytes; opts->stream orders the batch;
 * rel_error and sample_idx are ignored. Without TUCKER_FLAG_ASYNC the call
 * synchronises opts->stream and returns the first failing request's device
 * status (TUCKER_ERR_TIMEOUT before TUCKER_ERR_NUMERICAL); with it, it returns
 * after enqueueing, and request k's status word is the first 4 bytes of its
 * workspace slice. Argument errors of any request return before any launch. */
tucker_status tucker_batch_run(int n, const tucker_request* reqs, const tucker_opts* opts);

/* Host only (no device work, no pointer checks): the work list a batch with
 * TUCKER_FLAG_WORKLIST in opts->flags would run, as text in buf (len bytes,
 * NUL-terminated; TUCKER_ERR_INVALID_ARG when it does not fit): one line per
 * phase ("step s lane l: items=... init=... gaussian=... power=... sum=...
 * product=... smem=... heavy=..." counting tasks per stage) or grouped
 * orthonormalisation ("cholqr lane l: jobs=..." / "extract lane l: jobs=..."),
 * lane by lane, then "lanes=... tasks=... items=... area=...". Requests are
 * dealt to lanes (request k to lane k mod lanes; one lane per four requests, at
 * most eight), each a sequence on its own stream of the graph. The
 * planner checks that every task whose output another reads runs in an earlier
 * phase of the same lane, and that every extent an item touches lies inside the
 * buffer it targets (TUCKER_ERR_INVALID_ARG otherwise); unsupported batches return
 * TUCKER_ERR_UNSUPPORTED. */
tucker_status tucker_batch_describe(int n, const tucker_request* reqs, const tucker_opts* opts, char* buf,
                                    size_t len);

/* ---------------------------------------------------------------- autotuning
 * Not part of the paper's method. When enabled, the first synchronous call
 * (never an asynchronous one, never under stream capture) that meets a new
 * shape class of a tunable kernel times each candidate configuration on that
 * call's own data and stream (one warm-up and one timed launch each) and keeps
 * the fastest; every later call of the class, synchronous or not, uses it.
 * Classes and candidates:
 *   mode-n product (I_n, K_out, L_f, J_n): register-staged tiles, TMA-fed tiles
 *     with 2 or 3 stages - all three give bitwise the same result;
 *   FP32 power step (I_n, L_n, +-L_f, J_n): fiber-tile x column-group shapes
 *     32x32, 32x16, 16x16, 32x8, 16x8 within the planned partial storage -
 *     these differ in summation order, so results can change in the last bits.
 * Choices are kept for the process. */
tucker_status tucker_autotune_enable(int on);
/* Number of shape classes tuned so far. */
int64_t tucker_autotune_count(void);
/* Class k (0 <= k < count): one line naming the class, its choice and the
 * candidates' times; valid until the next call on this thread. */
const char* tucker_autotune_entry(int64_t k);

/* ---------------------------------------------------------------- measurement
 * Not part of the paper's method: counters for benchmarking the path. */

/* Cumulative number of kernel launches this library has made in the process. */
int64_t tucker_launch_count(void);

/* Kernel classes timed by the profiler. */
typedef enum {
    TUCKER_KERNEL_POWER = 0,   /* fused power step / range sketch on FP32/FP64 FMA (one pass over the unfolding) */
    TUCKER_KERNEL_TTM = 1,     /* mode-n product */
    TUCKER_KERNEL_GATHER = 2,  /* AMM rescaled gather */
    TUCKER_KERNEL_NORMS = 3,   /* squared fiber norms */
    TUCKER_KERNEL_EXTRACT = 4, /* a mode's whole orthonormalisation + extraction sequence */
    TUCKER_KERNEL_SAMPLE = 5,  /* a mode's weights, scan and draws */
    TUCKER_KERNEL_POWER_BF16 = 6, /* fused power step on the tensor cores, split-bf16 operands */
    TUCKER_KERNEL_POWER_TF32 = 7, /* fused power step on the tensor cores, tf32 operands */
    TUCKER_KERNEL_TTM_BF16 = 8,   /* mode-n product on the tensor cores, split-bf16 operands */
    TUCKER_KERNEL_POWER_BF16X1 = 9 /* fused power step on the tensor cores, single-pass bf16 operands */
} tucker_kernel_class;

/* on != 0: clear the accumulators and bracket every launch of the classes
 * above with CUDA events on its stream; on == 0: stop. */
tucker_status tucker_profile_enable(int on);

/* Totals since the last enable for one class: launches, summed event time
 * (ms), algorithmic bytes (the operands' size: each tensor element read once,
 * each output written once) and flops (2 per multiply-add). Synchronises on
 * the recorded events. Any output pointer may be NULL. */
tucker_status tucker_profile_read(int kernel_class, int64_t* launches, double* total_ms, double* bytes,
                                  double* flops);

#ifdef __cplusplus
}
#endif
#endif /* TUCKER_H */
