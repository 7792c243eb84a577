// Orthonormalisation of the sketch and extraction of the leading left singular
// vectors (remark after Algorithm 5: Q_n = U(:, 1:mu_n) from the SVD of C_n).
//
// C (I x L) = Q M with Q orthonormal and M = R_k ... R_1 upper triangular is
// formed by CholeskyQR2 (Gram in FP64 from exact FP32 products, Cholesky in
// FP64); when the first Gram matrix is numerically singular its Cholesky is
// shifted (shifted CholeskyQR, Fukaya et al. 2020) and a third pass runs. The
// leading left singular vectors of C are then Q times those of the small M,
// found with a one-sided (Hestenes) Jacobi SVD.
#include <float.h>

#include <algorithm>

#include "internal.h"

namespace tk {
namespace {

constexpr int kT = kThreads;
constexpr int kSvdThreads = 1024;

// pass 0: first pass; pass 1: second pass; pass 2: runs only if a shift was needed.
__device__ __forceinline__ bool pass_skipped(const int* flag, int pass) {
    return pass == 2 && !(*flag & kStatShifted);
}

// ---------------------------------------------------------------- Gram + Cholesky
// Each CTA accumulates the Gram matrix of its block of rows (packed upper
// triangle); the last CTA to finish (an atomic ticket, no waiting) sums the
// partials in block order, which makes the result independent of scheduling,
// and factors G = R^T R in FP64 (R upper, row-major R[a * L + b]). A pivot
// below 1e-15 of its diagonal entry restarts the factorisation once with
// G + s I, s = 11 (I L + L (L + 1)) 2^-53 tr(G), and flags the shift.
template <typename T> struct GramAcc;
template <> struct GramAcc<float> {
    Pair s{0.f, 0.f};
    __device__ void add(float a, float b) { pair_add_prod(s, a, b); }
    __device__ double value() const { return pair_value(s); }
};
template <> struct GramAcc<double> {
    double s = 0.0;
    __device__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ double value() const { return s; }
};

__device__ __forceinline__ int packed_index(int a, int b, int L) { return a * L - (a * (a - 1)) / 2 + (b - a); }

template <typename T>
__global__ void __launch_bounds__(kT) gram_chol_kernel(const T* __restrict__ X, int64_t I, int L, int rows_per_block,
                                                       double* __restrict__ partial, unsigned* ticket,
                                                       double* __restrict__ R, int* flag, int* status, int pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    if (pass_skipped(flag, pass)) {
        if (blockIdx.x == 0)
            for (int p = tid; p < L * L; p += kT) R[p] = (p / L == p % L) ? 1.0 : 0.0;
        return;
    }
    const int np = L * (L + 1) / 2;
    {
        T* xs = reinterpret_cast<T*>(smem_raw);   // [rows][L]
        const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
        const int nr = (int)max((int64_t)0, min((int64_t)rows_per_block, I - r0));
        for (int e = tid; e < nr * L; e += kT) {
            const int r = e % nr, c = e / nr;
            xs[r * L + c] = X[(int64_t)c * I + r0 + r];
        }
        __syncthreads();
        double* out = partial + (int64_t)blockIdx.x * np;
        for (int a = 0; a < L; ++a) {
            for (int b = a + tid; b < L; b += kT) {
                GramAcc<T> acc;
                for (int r = 0; r < nr; ++r) acc.add(xs[r * L + a], xs[r * L + b]);
                out[packed_index(a, b, L)] = acc.value();
            }
        }
    }
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();

    double* G = reinterpret_cast<double*>(smem_raw);   // [L][L]
    double* W = G + L * L;                               // [L][L]
    __shared__ int bad;
    __shared__ double inv_piv;
    const int nparts = gridDim.x;
    for (int p = tid; p < np; p += kT) {
        double acc = 0.0;
#pragma unroll 8
        for (int b = 0; b < nparts; ++b) acc += __ldcg(partial + (int64_t)b * np + p);
        // unpack (a, b) from the packed index
        int a = 0, rem = p;
        while (rem >= L - a) { rem -= L - a; ++a; }
        const int bb = a + rem;
        G[a * L + bb] = acc;
        G[bb * L + a] = acc;
    }
    if (tid == 0) *ticket = 0;                           // ready for the next pass
    __syncthreads();
    double shift = 0.0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        for (int p = tid; p < L * L; p += kT) W[p] = G[p] + ((p / L == p % L) ? shift : 0.0);
        if (tid == 0) bad = 0;
        __syncthreads();
        for (int k = 0; k < L; ++k) {
            if (tid == 0) {
                const double d = W[k * L + k];
                const double ref = G[k * L + k] + shift;
                if (!(d > 1e-15 * ref) || !isfinite(d)) {
                    bad = 1;
                } else {
                    const double pv = sqrt(d);
                    W[k * L + k] = pv;
                    inv_piv = 1.0 / pv;
                }
            }
            __syncthreads();
            if (bad) break;
            for (int j = k + 1 + tid; j < L; j += kT) W[k * L + j] *= inv_piv;
            __syncthreads();
            const int m = L - k - 1;
            for (int p = tid; p < m * m; p += kT) {
                const int i = k + 1 + p / m, j = k + 1 + p % m;
                if (j >= i) W[i * L + j] -= W[k * L + i] * W[k * L + j];
            }
            __syncthreads();
        }
        if (!bad) break;
        if (attempt == 0) {
            __shared__ double tr;
            if (tid == 0) {
                double t = 0.0;
                for (int k = 0; k < L; ++k) t += G[k * L + k];
                tr = t > 0.0 ? t : 1.0;
                *flag |= kStatShifted;
            }
            __syncthreads();
            shift = 11.0 * ((double)I * L + (double)L * (L + 1)) * 1.1102230246251565e-16 * tr;
            __syncthreads();
        }
    }
    if (bad && tid == 0) set_status(status, kStatNumerical);
    for (int p = tid; p < L * L; p += kT) {
        const int a = p / L, b = p % L;
        R[p] = (b >= a && !bad) ? W[p] : (a == b ? 1.0 : 0.0);
    }
}

// ---------------------------------------------------------------- Q = X R^{-1}
// One warp per row: forward substitution q_l = (x_l - sum_{m<l} q_m R[m][l]) / R[l][l] in FP64.
template <typename T>
__global__ void __launch_bounds__(kT) apply_rinv_kernel(const T* __restrict__ X, int64_t I, int L,
                                                        const double* __restrict__ R, T* __restrict__ Q,
                                                        const int* flag, int pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const bool copy = pass_skipped(flag, pass);
    double* Rs = reinterpret_cast<double*>(smem_raw);    // [L][L]
    double* qs = Rs + L * L;                               // [warps][L]
    if (!copy)
        for (int p = threadIdx.x; p < L * L; p += kT) Rs[p] = R[p];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* q = qs + warp * L;
    for (int64_t i = (int64_t)blockIdx.x * (kT / 32) + warp; i < I; i += (int64_t)gridDim.x * (kT / 32)) {
        if (copy) {
            for (int l = lane; l < L; l += 32) Q[(int64_t)l * I + i] = X[(int64_t)l * I + i];
            continue;
        }
        for (int l = 0; l < L; ++l) {
            double s = 0.0;
            for (int m = lane; m < l; m += 32) s = fma(q[m], Rs[m * L + l], s);
            s = warp_sum(s);
            if (lane == 0) q[l] = ((double)X[(int64_t)l * I + i] - s) / Rs[l * L + l];
            __syncwarp();
        }
        for (int l = lane; l < L; l += 32) Q[(int64_t)l * I + i] = (T)q[l];
        __syncwarp();
    }
}

// ---------------------------------------------------------------- small SVD
// M = F_{n-1} ... F_0 (each F upper triangular FP64, row-major), formed in T
// after scaling every factor by a power of two; then one-sided Jacobi on the
// columns of M (M V = U S); the R columns of largest norm, normalised, are the
// leading left singular vectors. Output UM (L x R, column-major).
template <typename T>
__global__ void __launch_bounds__(kSvdThreads) small_svd_kernel(const double* __restrict__ factors, int nf, int L,
                                                                int R, T* __restrict__ UM, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Lp = L + (L & 1);                           // even number of columns (phantom zero column)
    T* M = reinterpret_cast<T*>(smem_raw);                 // column-major [Lp][L]: column c at M + c * L
    T* Tm = M + Lp * L;                                    // product scratch [L][L]
    T* Fs = Tm + Lp * L;                                   // current factor, row-major [L][L]
    T* nrm = Fs + L * L;                                   // [Lp]
    int* perm = reinterpret_cast<int*>(nrm + Lp);          // [Lp]
    __shared__ unsigned long long fmax_bits;
    __shared__ int rotated;
    __shared__ T fro2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kSvdThreads / 32;

    for (int f = 0; f < nf; ++f) {
        const double* F = factors + (int64_t)f * L * L;
        if (tid == 0) fmax_bits = 0ull;
        __syncthreads();
        double mx = 0.0;
        for (int p = tid; p < L * L; p += kSvdThreads) mx = fmax(mx, fabs(F[p]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomicMax(&fmax_bits, (unsigned long long)__double_as_longlong(mx));
        __syncthreads();
        const double fm = __longlong_as_double((long long)fmax_bits);
        const double sc = fm > 0.0 ? exp2(-floor(log2(fm))) : 1.0;   // a power of two: exact
        for (int p = tid; p < L * L; p += kSvdThreads) Fs[p] = (T)(F[p] * sc);
        __syncthreads();
        if (f == 0) {
            for (int p = tid; p < Lp * L; p += kSvdThreads) {
                const int c = p / L, a = p % L;
                M[p] = (c < L && c >= a) ? Fs[a * L + c] : T(0);
            }
        } else {
            for (int p = tid; p < L * L; p += kSvdThreads) {
                const int c = p / L, a = p % L;
                T acc = T(0);
                for (int b = a; b < L; ++b) acc = fma(Fs[a * L + b], M[c * L + b], acc);
                Tm[p] = acc;
            }
            __syncthreads();
            for (int p = tid; p < L * L; p += kSvdThreads) M[p] = Tm[p];
        }
        __syncthreads();
    }
    // squared Frobenius norm: a pair whose coupling is below eps^2 of it is at the
    // rounding level of the whole matrix and is left alone (rounding would otherwise
    // keep near-zero columns rotating without end)
    if (tid == 0) fro2 = T(0);
    __syncthreads();
    {
        T s2 = T(0);
        for (int p = tid; p < L * L; p += kSvdThreads) s2 = fma(M[p], M[p], s2);
        s2 = warp_sum(s2);
        if (lane == 0) atomicAdd(&fro2, s2);
    }
    __syncthreads();
    const T eps = sizeof(T) == 4 ? (T)FLT_EPSILON : (T)DBL_EPSILON;
    const T tol = eps * T(2);
    const T tiny = eps * eps * fro2;
    const int m = Lp - 1;
    for (int sweep = 0; sweep < 30; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int rnd = 0; rnd < m; ++rnd) {
            for (int pi = warp; pi < Lp / 2; pi += nwarps) {
                int p, q;
                if (pi == 0) { p = rnd; q = m; }
                else { p = (rnd + pi) % m; q = (rnd - pi + m) % m; }
                if (p >= L || q >= L) continue;
                T* cp = M + p * L;
                T* cq = M + q * L;
                T al = 0, be = 0, ga = 0;
                for (int r = lane; r < L; r += 32) {
                    const T x = cp[r], y = cq[r];
                    al = fma(x, x, al); be = fma(y, y, be); ga = fma(x, y, ga);
                }
                al = warp_sum(al); be = warp_sum(be); ga = warp_sum(ga);
                if (fabs(ga) > tiny && fabs(ga) > tol * sqrt(al * be)) {
                    const T zeta = (be - al) / (T(2) * ga);
                    const T t = (zeta >= 0 ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
                    const T c = T(1) / sqrt(T(1) + t * t), s = c * t;
                    for (int r = lane; r < L; r += 32) {
                        const T x = cp[r], y = cq[r];
                        cp[r] = c * x - s * y;
                        cq[r] = s * x + c * y;
                    }
                    if (lane == 0) rotated = 1;
                }
            }
            __syncthreads();
        }
        if (!rotated) break;
        __syncthreads();
    }
    // column norms, order by decreasing norm (ties: lower index first)
    for (int c = warp; c < L; c += nwarps) {
        T s = 0;
        for (int r = lane; r < L; r += 32) s = fma(M[c * L + r], M[c * L + r], s);
        s = warp_sum(s);
        if (lane == 0) nrm[c] = sqrt(s);
    }
    __syncthreads();
    for (int c = tid; c < L; c += kSvdThreads) {
        int rank = 0;
        for (int d = 0; d < L; ++d) rank += (nrm[d] > nrm[c]) || (nrm[d] == nrm[c] && d < c);
        perm[rank] = c;
    }
    __syncthreads();
    for (int p = tid; p < L * R; p += kSvdThreads) {
        const int r = p / L, a = p % L;
        const int c = perm[r];
        const T n = nrm[c];
        UM[p] = n > T(0) ? M[c * L + a] / n : T(0);
    }
    if (tid == 0 && R > 0 && !(nrm[perm[R - 1]] > T(0))) set_status(status, kStatNumerical);
}

// ---------------------------------------------------------------- U = Q UM, sign rule
template <typename T>
__global__ void __launch_bounds__(kT) form_u_kernel(const T* __restrict__ Q, int64_t I, int L,
                                                    const T* __restrict__ UM, T* __restrict__ U) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* um = reinterpret_cast<T*>(smem_raw);   // [L]
    T* col = um + L;                          // [I]
    __shared__ T best_v[kT / 32];
    __shared__ int64_t best_i[kT / 32];
    __shared__ T sgn;
    const int r = blockIdx.x;
    for (int c = threadIdx.x; c < L; c += kT) um[c] = UM[(int64_t)r * L + c];
    __syncthreads();
    T bv = T(-1);
    int64_t bi = 0;
    for (int64_t i = threadIdx.x; i < I; i += kT) {
        T s = 0;
        for (int c = 0; c < L; ++c) s = fma(Q[(int64_t)c * I + i], um[c], s);
        col[i] = s;
        const T a = fabs(s);
        if (a > bv) { bv = a; bi = i; }     // first (lowest) index wins ties within a thread
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if ((threadIdx.x & 31) == 0) { best_v[threadIdx.x >> 5] = bv; best_i[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        T v = best_v[0];
        int64_t k = best_i[0];
        for (int w = 1; w < kT / 32; ++w)
            if (best_v[w] > v || (best_v[w] == v && best_i[w] < k)) { v = best_v[w]; k = best_i[w]; }
        sgn = col[k] < T(0) ? T(-1) : T(1);
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < I; i += kT) U[(int64_t)r * I + i] = sgn * col[i];
}

}  // namespace

OrthPlan orth_plan(int64_t I, int L, int num_sms) {
    OrthPlan p{};
    p.I = I;
    p.L = L;
    // enough CTAs to spread the FP64-grade Gram work, few enough that the last
    // CTA's reduction of the packed partials stays small (<= 512 KB)
    const int64_t np = (int64_t)L * (L + 1) / 2;
    int64_t cap = (512 * 1024) / (np * 8);
    if (cap < 1) cap = 1;
    if (cap > num_sms) cap = num_sms;
    int64_t blocks = (I + 7) / 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    p.gram_blocks = (int)blocks;
    return p;
}

static int gram_rows(const OrthPlan& p) { return (int)((p.I + p.gram_blocks - 1) / p.gram_blocks); }

size_t orth_scratch_bytes(const OrthPlan& p, int elem_size) {
    const size_t np = (size_t)p.L * (p.L + 1) / 2;
    const size_t LL = (size_t)p.L * p.L;
    return sizeof(double) * np * (size_t)p.gram_blocks + 256 + (size_t)elem_size * LL + 512;
}

struct OrthScratch {
    double* partial;
    int* flag;
    unsigned* ticket;
    void* um;
};
static OrthScratch carve(const OrthPlan& p, void* scratch) {
    OrthScratch s;
    char* b = reinterpret_cast<char*>(scratch);
    const size_t np = (size_t)p.L * (p.L + 1) / 2;
    s.partial = reinterpret_cast<double*>(b);
    b += ((sizeof(double) * np * (size_t)p.gram_blocks) + 255) & ~size_t(255);
    s.flag = reinterpret_cast<int*>(b);
    s.ticket = reinterpret_cast<unsigned*>(b + 64);
    b += 256;
    s.um = b;
    return s;
}

template <typename T>
cudaError_t launch_cholqr(const T* X, T* Q, T* Qtmp, const OrthPlan& p, double* factors, int slot, void* scratch,
                          int* status, cudaStream_t s) {
    OrthScratch sc = carve(p, scratch);
    const int L = p.L;
    const size_t LL = (size_t)L * L;
    const int rows = gram_rows(p);
    const size_t gsm = std::max(sizeof(T) * (size_t)rows * L, sizeof(double) * 2 * LL);
    const size_t asm_ = sizeof(double) * (LL + (size_t)(kT / 32) * L);
    if (asm_ > 220 * 1024 || gsm > 220 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(gram_chol_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
    cudaFuncSetAttribute(apply_rinv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asm_);
    cudaMemsetAsync(sc.flag, 0, 128, s);                 // shift flag and ticket
    int64_t ablocks = (p.I + kT / 32 - 1) / (kT / 32);
    if (ablocks > 1024) ablocks = 1024;
    // pass 0: X -> Q ; pass 1: Q -> Qtmp ; pass 2 (only after a shift): Qtmp -> Q, else copy
    const T* src[3] = {X, Q, Qtmp};
    T* dst[3] = {Q, Qtmp, Q};
    for (int pass = 0; pass < 3; ++pass) {
        double* R = factors + (size_t)(3 * slot + pass) * LL;
        gram_chol_kernel<T><<<p.gram_blocks, kT, gsm, s>>>(src[pass], p.I, L, rows, sc.partial, sc.ticket, R,
                                                           sc.flag, status, pass);
        note_launch();
        apply_rinv_kernel<T><<<(unsigned)ablocks, kT, asm_, s>>>(src[pass], p.I, L, R, dst[pass], sc.flag, pass);
        note_launch();
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_extract(const T* Q, const OrthPlan& p, const double* factors, int nfactors, int R, T* U,
                           void* scratch, int* status, cudaStream_t s) {
    OrthScratch sc = carve(p, scratch);
    const int L = p.L;
    const int Lp = L + (L & 1);
    const size_t ssm = sizeof(T) * (2 * (size_t)Lp * L + (size_t)L * L + Lp) + sizeof(int) * Lp + 64;
    if (ssm > 220 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(small_svd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm);
    T* um = reinterpret_cast<T*>(sc.um);
    small_svd_kernel<T><<<1, kSvdThreads, ssm, s>>>(factors, nfactors, L, R, um, status);
    note_launch();
    const size_t fsm = sizeof(T) * ((size_t)L + (size_t)p.I) + 64;
    if (fsm > 220 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(form_u_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
    form_u_kernel<T><<<R, kT, fsm, s>>>(Q, p.I, L, um, U);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t launch_cholqr<float>(const float*, float*, float*, const OrthPlan&, double*, int, void*, int*,
                                          cudaStream_t);
template cudaError_t launch_cholqr<double>(const double*, double*, double*, const OrthPlan&, double*, int, void*,
                                           int*, cudaStream_t);
template cudaError_t launch_extract<float>(const float*, const OrthPlan&, const double*, int, int, float*, void*,
                                           int*, cudaStream_t);
template cudaError_t launch_extract<double>(const double*, const OrthPlan&, const double*, int, int, double*,
                                            void*, int*, cudaStream_t);

}  // namespace tk
