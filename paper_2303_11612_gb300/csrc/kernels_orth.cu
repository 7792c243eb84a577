// Orthonormalisation of the sketch and extraction of the leading left singular
// vectors (remark after Algorithm 5: Q_n = U(:, 1:mu_n) from the SVD of C_n).
//
// The sketch is held as C = X F, where X (I x L) is the last power-step output
// and F = F_k ... F_1 collects the triangular factors of the earlier steps
// (each earlier step orthonormalised its output X_j = Q_j F_j and multiplied Q_j,
// which leaves C unchanged). Extraction:
//   1. One CholeskyQR pass X = Q1 R1: Gram X^T X from exact products summed in
//      paired precision, reduced across CTAs in a fixed order; Cholesky
//      (shifted once on a numerically singular pivot, Fukaya et al. 2020);
//      Q1 = X R1^-1 with a row-oriented triangular inverse.
//   2. A second Gram/Cholesky Q1^T Q1 = R2^T R2, so Q = Q1 R2^-1 is orthonormal
//      and C = Q M with M = R2 R1 F (L x L, upper triangular).
//   3. QR with column pivoting of M^T, M^T P = Q_h R, so M = P R^T Q_h^T, then
//      one-sided (Hestenes) Jacobi on the columns of B = R^T with paired-precision
//      dot products: B V = U_B S, U_B = the rotated columns, normalised, and
//      U_M = P U_B; columns at rounding level are re-orthogonalised (classical
//      Gram-Schmidt, twice), so they keep the sketch's own weak directions.
//      U = Q U_M = Q1 W with W = R2^-1 U_M (back-substitution); Q is never formed.
//   4. U = Q1 W in paired precision.
//   5. A final pass keeps U orthonormal where the sketch is numerically
//      rank-deficient (CholeskyQR cannot orthonormalise those directions): if
//      U^T U is not within 8 eps of I, one CholeskyQR pass on U itself, which
//      leaves the span of every leading set of columns unchanged; columns that
//      collapse are rebuilt from unit vectors by Gram-Schmidt. Then each
//      column's largest-magnitude entry is made positive.
// Intermediate power steps need only Q1 and R1: step 1 alone.
//
// Small matrices (Gram, Cholesky factors, their products and inverses) are
// packed upper triangles, row-major, in the scalar S = SmallScalar<T>: a
// double-float pair for FP32 data (the FP64 pipe of this GPU is narrow, and
// these steps form long dependent chains in one CTA), FP64 for FP64 data.
// Their entries must stay within about 1e-30 .. 1e30 for the pair form.
#include <float.h>

#include <algorithm>

#include "df.cuh"
#include "internal.h"

namespace tk {
namespace {

constexpr int kT = kThreads;
// threads of the kernels whose last CTA runs the serial small-matrix algebra
// (Cholesky, triangular inverse, Jacobi, final pass): their steps are chains of
// barriers, so each step is spread over as many threads as a CTA has
constexpr int kST = 1024;
// the extraction kernel holds two columns' entries per Jacobi lane: 512 threads
// leave it 128 registers and still give every pair of a round (L <= 128) its group
constexpr int kXT = 512;
constexpr int kGramRows = 64;            // fewest rows per Gram CTA (few partials to reduce)
constexpr int kBsCols = 4;               // columns per warp in the extraction's back-substitution
constexpr int kBsRows = 4;               // rows per lane there: L <= 32 kBsRows

__host__ __device__ __forceinline__ int packed_index(int a, int b, int L) {
    return a * L - (a * (a - 1)) / 2 + (b - a);
}
__host__ __device__ __forceinline__ size_t packed_size(int L) { return (size_t)L * (L + 1) / 2; }

// Unit roundoff of the Gram matrix: paired-FP32 sums for FP32 data, FP64 sums otherwise.
template <typename T> __device__ __forceinline__ double gram_unit() { return sizeof(T) == 4 ? 0x1p-44 : 0x1p-53; }

template <typename S, typename T> __device__ __forceinline__ S to_s(T x) {
    if constexpr (sizeof(T) == 4) return Sc<S>::from_float((float)x);
    else return Sc<S>::from_double((double)x);
}

// Broadcast of a small-matrix scalar from lane src of the warp.
__device__ __forceinline__ df shfl_s(df v, int src) {
    return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}
__device__ __forceinline__ double shfl_s(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Load that bypasses L1 (data written by other CTAs of the same launch).
__device__ __forceinline__ df ld_cg(const df* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }

template <typename T> struct GramAcc;
template <> struct GramAcc<float> {
    Pair s{0.f, 0.f};
    __device__ void add(float a, float b) { pair_add_prod(s, a, b); }
    __device__ df value() const { return two_sum(s.hi, s.lo); }
};
template <> struct GramAcc<double> {
    double s = 0.0;
    __device__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ double value() const { return s; }
};

// Gram partial of block bid's rows (packed upper triangle) -> partial[bid].
// Rows of X staged in shared memory per chunk of the Gram partial sums.
constexpr int kGramChunk = 64;

template <typename T, typename S>
__device__ void gram_partial(const T* __restrict__ X, int64_t I, int L, int rows, S* __restrict__ partial,
                             unsigned char* smem, int64_t bid) {
    T* xs = reinterpret_cast<T*>(smem);   // [kGramChunk][L]
    const int64_t r0 = bid * rows;
    const int nr = (int)max((int64_t)0, min((int64_t)rows, I - r0));
    const int np = (int)packed_size(L);
    S* out = partial + bid * np;
    // chunks of kGramChunk rows; each entry's chunk sums are added in chunk order
    // by the thread that owns the entry
    for (int c0 = 0; c0 < nr || c0 == 0; c0 += kGramChunk) {
        const int cn = min(kGramChunk, nr - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < cn * L; e += blockDim.x) {
            const int r = e % cn, c = e / cn;
            xs[r * L + c] = X[(int64_t)c * I + r0 + c0 + r];
        }
        __syncthreads();
        for (int p = threadIdx.x; p < np; p += blockDim.x) {
            int a = 0, rem = p;
            while (rem >= L - a) { rem -= L - a; ++a; }
            const int b = a + rem;
            GramAcc<T> acc;
            for (int r = 0; r < cn; ++r) acc.add(xs[r * L + a], xs[r * L + b]);
            out[p] = c0 == 0 ? acc.value() : out[p] + acc.value();
        }
        if (cn <= 0) break;
    }
}

// True in exactly one CTA: the last to finish its partial (an atomic ticket, no waiting).
__device__ bool last_cta(unsigned* ticket, unsigned nblk) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == nblk - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Entry number e of the trailing triangle, counted from the bottom row up:
// row i = L - 1 - r holds numbers T(r) .. T(r + 1) - 1, T(r) = r (r + 1) / 2,
// and number T(r) + c is column j = i + c. Rows k + 1 .. L - 1 are then the
// first T(L - 1 - k) numbers, for every k.
__device__ __forceinline__ void trailing_entry(int e, int L, int& i, int& j) {
    int r = (int)((sqrtf((float)(8 * e + 1)) - 1.f) * 0.5f);
    if ((r + 1) * (r + 2) / 2 <= e) ++r;
    if (r * (r + 1) / 2 > e) --r;
    i = L - 1 - r;
    j = i + (e - r * (r + 1) / 2);
}

// Sum the partials in block order into G and factor G = R^T R (all packed;
// R in W, 1/R_kk in dinv). A pivot below 8u of its diagonal entry restarts once
// with G + s I, s = 11 (I L + L (L + 1)) u tr(G), u the Gram's unit roundoff.
// Returns false if that also fails (then R = I).
//
// Right-looking, one barrier per column: in the phase of column k every
// thread updates its entries of the trailing rows from the unscaled row k
// (W_ij -= W_ki W_kj / d_k; at most a few entries a thread, numbered as in
// trailing_entry), the thread that updates W_{k+1,k+1} takes the next pivot at
// once (its threshold formed alongside the update), and row k - 1 is scaled by
// 1/R_{k-1,k-1} alongside. The entries' (i, j) are decoded once into `tab`
// ((L - 1) L / 2 ints of shared memory): their numbering does not depend on k.
template <typename T, typename S>
__device__ bool reduce_cholesky(const S* __restrict__ partial, int nparts, int L, int64_t I, S* G, S* W, S* dinv,
                                int* tab, unsigned* ticket, int* status) {
    using F = Sc<S>;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int np = (int)packed_size(L);
    const double u = gram_unit<T>();
    __shared__ int bad;
    __shared__ S inv2[2];
    __shared__ double tr;
    for (int p = tid; p < np; p += nt) {
        S acc = ld_cg(partial + p);
        for (int b = 1; b < nparts; ++b) acc = acc + ld_cg(partial + (int64_t)b * np + p);
        G[p] = acc;
    }
    for (int e = tid; e < (L - 1) * L / 2; e += nt) {
        int i, j;
        trailing_entry(e, L, i, j);
        tab[e] = (i << 16) | j;
    }
    if (tid == 0) *ticket = 0;                           // ready for the next use
    __syncthreads();
    const S thr = F::from_double(8.0 * u);
    S shift = F::zero();
    // pivot k from the updated W_kk = d against lim = (G_kk + shift) 8u;
    // sets bad when numerically singular
    auto pivot = [&](int k, S d, S lim) {
        if (!F::gt(d, lim) || !F::finite(d)) {
            bad = 1;
        } else {
            const S y = F::rsqrt(d);
            W[packed_index(k, k, L)] = d * y;
            dinv[k] = y;
            inv2[k & 1] = y * y;
        }
    };
    for (int attempt = 0; attempt < 2; ++attempt) {
        for (int p = tid; p < np; p += nt) W[p] = G[p];
        __syncthreads();
        for (int k = tid; k < L; k += nt) W[packed_index(k, k, L)] = G[packed_index(k, k, L)] + shift;
        if (tid == 0) bad = 0;
        __syncthreads();
        if (tid == 0) pivot(0, W[0], (G[0] + shift) * thr);
        __syncthreads();
        for (int k = 0; k < L && !bad; ++k) {
            if (k > 0) {                                  // scale row k - 1
                const S y = dinv[k - 1];
                S* row = W + packed_index(k - 1, k - 1, L);
                for (int j = 1 + tid; j < L - k + 1; j += nt) row[j] = row[j] * y;
            }
            const S y2 = inv2[k & 1];
            const S* rk = W + packed_index(k, k, L);      // rk[j - k] = W_kj
            const int ne = (L - 1 - k) * (L - k) / 2;     // entries of rows k + 1 .. L - 1
            for (int e = tid; e < ne; e += nt) {
                const int ij = tab[e];
                const int i = ij >> 16, j = ij & 0xffff;
                const bool piv = j == k + 1;              // then i == k + 1 as well
                S lim = F::zero();
                if (piv) lim = (G[packed_index(k + 1, k + 1, L)] + shift) * thr;
                S* w = W + packed_index(i, j, L);
                const S v = *w - (rk[i - k] * y2) * rk[j - k];
                *w = v;
                if (piv) pivot(k + 1, v, lim);
            }
            __syncthreads();
        }
        if (!bad) break;
        if (attempt == 0) {
            if (tid == 0) {
                double t = 0.0;
                for (int k = 0; k < L; ++k) t += F::to_double(G[packed_index(k, k, L)]);
                tr = t > 0.0 ? t : 1.0;
            }
            __syncthreads();
            shift = F::from_double(11.0 * ((double)I * L + (double)L * (L + 1)) * u * tr);
            __syncthreads();
        }
    }
    const int failed = bad;
    __syncthreads();
    if (failed) {
        for (int p = tid; p < np; p += nt) W[p] = F::zero();
        __syncthreads();
        for (int k = tid; k < L; k += nt) {
            W[packed_index(k, k, L)] = F::one();
            dinv[k] = F::one();
        }
        if (tid == 0) set_status(status, kStatNumerical);
    }
    __syncthreads();
    return !failed;
}

// Inverse of the packed upper-triangular R (1/R_kk in dinv) into Ri (packed),
// with Acc a packed scratch of the same size. Row i of R^-1 solves x R = e_i,
// x_ij = (delta_ij - sum_{k<j} x_ik R_kj) / R_jj, so the computed inverse has a
// small residual R^-1 R - I: X R^-1 R stays close to X, which is what Q R = X
// needs. The columns are solved in order, right-looking: once column j is
// known, every pair (row i <= j, column k > j) adds x_ij R_jk to its running
// sum Acc_ik, so a column costs one dependent step and one barrier for all
// rows together (each thread recomputes the x_ij its pairs need).
template <typename S>
__device__ void upper_inverse(const S* R, const S* dinv, int L, S* Acc, S* Ri) {
    using F = Sc<S>;
    const int np = (int)packed_size(L);
    for (int p = threadIdx.x; p < np; p += blockDim.x) Acc[p] = F::zero();
    __syncthreads();
    for (int j = 0; j < L; ++j) {
        const int rows = j + 1, cols = L - 1 - j;
        const int n = rows * (cols > 0 ? cols : 1);
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const int i = e % rows, c = e / rows;
            const int ij = packed_index(i, j, L);
            const S x = ((i == j ? F::one() : F::zero()) - Acc[ij]) * dinv[j];
            if (c == 0) Ri[ij] = x;
            if (cols > 0) {
                const int ik = packed_index(i, j + 1 + c, L);
                Acc[ik] = F::fma(x, R[packed_index(j, j + 1 + c, L)], Acc[ik]);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- one CholeskyQR pass
// R and R^-1 (packed, scalar S) of X^T X = R^T R.
template <typename T>
__device__ __forceinline__ void gram_chol_body(const T* __restrict__ X, int64_t I, int L, int rows,
                                               typename SmallScalar<T>::type* __restrict__ partial, unsigned* ticket,
                                               typename SmallScalar<T>::type* __restrict__ R,
                                               typename SmallScalar<T>::type* __restrict__ Rinv, int* status,
                                               int bid, int nblk,
                                               typename SmallScalar<T>::type* __restrict__ stage = nullptr) {
    using S = typename SmallScalar<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    gram_partial<T, S>(X, I, L, rows, partial, smem_raw, bid);
    if (!last_cta(ticket, nblk)) return;
    const int np = (int)packed_size(L);
    S* G = reinterpret_cast<S*>(smem_raw);
    S* W = G + np;
    S* RT = W + np;
    S* dinv = RT + np;
    reduce_cholesky<T, S>(partial, nblk, L, I, G, W, dinv, reinterpret_cast<int*>(RT), ticket, status);
    if (stage) {
        // R^-1 by tri_inverse_kernel: rows on warps of their own CTAs
        for (int p = threadIdx.x; p < np; p += blockDim.x) R[p] = W[p];
        for (int k = threadIdx.x; k < L; k += blockDim.x) stage[k] = dinv[k];
        return;
    }
    upper_inverse<S>(W, dinv, L, RT, G);
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        R[p] = W[p];
        Rinv[p] = G[p];
    }
}

// Q = X R^-1, one thread per entry of Q, in paired precision from X (exact)
// and the double-float R^-1 (FP64 for T = double).
template <typename T> struct ApplyAcc;
template <> struct ApplyAcc<float> {
    Pair s{0.f, 0.f};
    __device__ void add(float x, df w) {
        pair_add_prod(s, x, w.hi);
        pair_add_prod(s, x, w.lo);
    }
    __device__ float value() const { return s.hi + s.lo; }
};
template <> struct ApplyAcc<double> {
    double s = 0.0;
    __device__ void add(double x, double w) { s = fma(x, w, s); }
    __device__ double value() const { return s; }
};

template <typename T>
__device__ __forceinline__ void apply_rinv_body(const T* __restrict__ X, int64_t I, int L,
                                                const typename SmallScalar<T>::type* __restrict__ Rinv,
                                                T* __restrict__ Q, int bid, int nblk) {
    using S = typename SmallScalar<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* Ri = reinterpret_cast<S*>(smem_raw);    // packed
    const int np = (int)packed_size(L);
    for (int p = threadIdx.x; p < np; p += kT) Ri[p] = Rinv[p];
    __syncthreads();
    const int64_t n = I * L;
    for (int64_t e = (int64_t)bid * kT + threadIdx.x; e < n; e += (int64_t)nblk * kT) {
        const int l = (int)(e / I);
        const int64_t i = e - (int64_t)l * I;
        ApplyAcc<T> acc;
        for (int m = 0; m <= l; ++m) acc.add(X[(int64_t)m * I + i], Ri[packed_index(m, l, L)]);
        Q[e] = (T)acc.value();
    }
}

// ---------------------------------------------------------------- fused extraction
template <typename T> struct DotAcc;
template <> struct DotAcc<float> {
    Pair s{0.f, 0.f};
    __device__ void add(float a, float b) { pair_add_prod(s, a, b); }
    __device__ void reduce() { s = warp_sum_pair(s); }
    __device__ float value() const { return s.hi + s.lo; }
};
template <> struct DotAcc<double> {
    double s = 0.0;
    __device__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ void reduce() { s = warp_sum(s); }
    __device__ double value() const { return s; }
};

// Pair dot products over a group of GS lanes (GS = 8, 16 or 32).
template <int GS>
__device__ __forceinline__ Pair group_sum_pair(Pair s) {
#pragma unroll
    for (int o = GS / 2; o > 0; o >>= 1) {
        Pair t;
        t.hi = __shfl_xor_sync(0xffffffffu, s.hi, o);
        t.lo = __shfl_xor_sync(0xffffffffu, s.lo, o);
        pair_add(s, t);
    }
    return s;
}
template <int GS, typename V>
__device__ __forceinline__ V group_sum(V s) {
#pragma unroll
    for (int o = GS / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Two FP32 values in one 64-bit register and the packed FP32 pipe's
// operations on both halves at once (each half rounded as the scalar
// operation rounds it): the even and odd entries' chains below run as one.
using f2 = unsigned long long;
__device__ __forceinline__ f2 pk2(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void up2(f2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// sum over e of x[e] y[e] in paired precision, the even and odd entries in two
// chains (packed), combined: the per-lane part of a paired dot product
template <int NE>
__device__ __forceinline__ Pair paired_dot2(const float (&x)[NE], const float (&y)[NE]) {
    static_assert(NE % 2 == 0, "entries in pairs");
    f2 H = 0ull, Lo = 0ull;
#pragma unroll
    for (int e = 0; e < NE; e += 2) {
        const f2 X = pk2(x[e], x[e + 1]), Y = pk2(y[e], y[e + 1]);
        const f2 P = mul2(X, Y);
        const f2 PE = fma2(X, Y, sub2(0ull, P));
        const f2 Tt = add2(H, P);
        const f2 Z = sub2(Tt, H);
        const f2 E = add2(sub2(H, sub2(Tt, Z)), sub2(P, Z));
        H = Tt;
        Lo = add2(Lo, add2(E, PE));
    }
    Pair ga, gb;
    up2(H, ga.hi, gb.hi);
    up2(Lo, ga.lo, gb.lo);
    pair_add(ga, gb);
    return ga;
}

// Dot product of a group of 8 lanes' NE entries each (rows gl + 8 e), paired
// precision for FP32 data; every lane of the group gets the sum.
template <typename T, int NE>
__device__ __forceinline__ T group8_dot(const T (&x)[NE], const T (&y)[NE]) {
    if constexpr (sizeof(T) == 4) {
        Pair a = paired_dot2<NE>(x, y);
        a = group_sum_pair<8>(a);
        return a.hi + a.lo;
    } else {
        T a = T(0);
#pragma unroll
        for (int e = 0; e < NE; ++e) a = fma(x[e], y[e], a);
        return group_sum<8>(a);
    }
}

// Householder QR with column pivoting of the L x L matrix A (column-major in
// shared memory, column p at A + p L): A(:, cmap) = Q R, with Q not formed.
// The strict upper triangle of R stays in A (R_ij, i < j, at A[cmap[j] L + i]),
// its diagonal goes to rdiag and the column order to cmap + (L & 1) Lp.
// Step k takes the remaining column of largest norm (lowest index on ties) and
// the reflector H = I - beta v v^T with H x = alpha e_k, alpha = -sign(x_k) |x|,
// beta = 1 / (alpha (alpha - x_k)) (no cancellation in either). One barrier per
// step: every 8-lane group forms the reflector from the pivot column itself
// (|x|^2 is the pivot's remaining norm, kept from the previous step in paired
// precision), then updates its columns (rows k..) and their remaining norms
// below row k; the norms and the order are double-buffered, since other warps
// still read the previous step's while a group writes.
template <typename T, int NE>
__device__ void pivoted_qr(T* A, int L, int Lp, T* qnrm, T* rdiag, int* cmap) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = (int)blockDim.x >> 5;
    const int gl = lane & 7, gw = lane >> 3;
    const int ngroups = nwarps * 4;
    for (int p = warp; p < L; p += nwarps) {
        DotAcc<T> s2;
        for (int r = lane; r < L; r += 32) s2.add(A[p * L + r], A[p * L + r]);
        s2.reduce();
        if (lane == 0) qnrm[p] = (T)s2.value();
    }
    for (int j = tid; j < L; j += blockDim.x) cmap[j] = j;
    __syncthreads();
    for (int k = 0; k < L; ++k) {
        const int* cur = cmap + (k & 1) * Lp;
        int* nxt = cmap + ((k + 1) & 1) * Lp;
        const T* nin = qnrm + (k & 1) * Lp;
        T* nout = qnrm + ((k + 1) & 1) * Lp;
        T bv = T(-1);
        int bj = L;
        for (int j = k + lane; j < L; j += 32) {
            const T v = nin[cur[j]];
            if (v > bv) { bv = v; bj = j; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (ov > bv || (ov == bv && oj < bj)) { bv = ov; bj = oj; }
        }
        const int piv = bj < L ? bj : k;
        const int pk = cur[k], pc = cur[piv];
        if (warp == 0)
            for (int j = lane; j < L; j += 32) nxt[j] = j == k ? pc : (j == piv ? pk : cur[j]);
        const T n2 = nin[pc];
        const T xk = A[pc * L + k];
        T v[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const int r = gl + 8 * e;
            v[e] = (r >= k && r < L) ? A[pc * L + r] : T(0);
        }
        const bool any = n2 > T(0);
        const T alpha = any ? -copysign(sqrt(n2), xk) : T(0);
        const T beta = any ? T(1) / (alpha * (alpha - xk)) : T(0);
#pragma unroll
        for (int e = 0; e < NE; ++e)
            if (gl + 8 * e == k) v[e] -= alpha;
        if (tid == 0) rdiag[k] = alpha;
        // the loop bound is uniform across a warp (the group sums shuffle over all 32 lanes)
        for (int base = k + 1 + warp * 4; base < L; base += ngroups) {
            const int j = base + gw;
            const bool live = j < L;
            const int p = live ? (j == piv ? pk : cur[j]) : 0;
            T y[NE];
#pragma unroll
            for (int e = 0; e < NE; ++e) {
                const int r = gl + 8 * e;
                y[e] = (live && r >= k && r < L) ? A[p * L + r] : T(0);
            }
            const T d = beta * group8_dot<T, NE>(v, y);
#pragma unroll
            for (int e = 0; e < NE; ++e) {
                const int r = gl + 8 * e;
                if (live && r >= k && r < L) {
                    const T w = fma(-d, v[e], y[e]);
                    A[p * L + r] = w;
                    y[e] = r > k ? w : T(0);
                } else {
                    y[e] = T(0);
                }
            }
            const T m2 = group8_dot<T, NE>(y, y);
            if (live && gl == 0) nout[p] = m2;
        }
        __syncthreads();
    }
}

// Rotation (c, s) that zeroes the coupling g of columns with squared norms a, b
// (t = tan of the angle). Any c, s with s / c = t form a scaled rotation, which
// keeps the pair's orthogonality, so the FP32 form uses the fast approximate
// reciprocal and square roots: their rounding only perturbs the angle.
__device__ __forceinline__ void rotation(float a, float b, float g, float& c, float& s) {
    const float zeta = __fdividef(b - a, 2.f * g);
    const float az = fabsf(zeta);
    float t;
    if (az > 1e18f) {
        t = __fdividef(0.5f, zeta);
    } else {
        const float h = fmaf(zeta, zeta, 1.f);
        t = __fdividef(copysignf(1.f, zeta), az + h * rsqrtf(h));
    }
    c = rsqrtf(fmaf(t, t, 1.f));
    s = c * t;
}
__device__ __forceinline__ void rotation(double a, double b, double g, double& c, double& s) {
    const double zeta = (b - a) / (2.0 * g);
    const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    c = 1.0 / sqrt(1.0 + t * t);
    s = c * t;
}

// Squared norms a, b and coupling g of the column pair x, y held by a group of
// GS lanes (NE entries each): a, b are plain sums (they only set the angle and
// the threshold); g, which cancels, is summed in paired precision.
template <typename T, int GS, int NE>
__device__ __forceinline__ void pair_sums(const T (&x)[NE], const T (&y)[NE], T& a, T& b, T& g) {
    // two independent chains per sum (even and odd entries), combined in a
    // fixed order: the sums are the dependent chains of a round
    if constexpr (sizeof(T) == 4 && NE % 2 == 0) {
        // both chains at once on the packed pipe: the same operations, in the same
        // order, as the scalar form below (pair_add_prod per entry)
        f2 A = 0ull, Bs = 0ull;
#pragma unroll
        for (int e = 0; e < NE; e += 2) {
            const f2 X = pk2(x[e], x[e + 1]), Y = pk2(y[e], y[e + 1]);
            A = fma2(X, X, A);
            Bs = fma2(Y, Y, Bs);
        }
        float a0, a1, b0, b1;
        up2(A, a0, a1);
        up2(Bs, b0, b1);
        a = a0 + a1;
        b = b0 + b1;
        Pair ga = paired_dot2<NE>(x, y);
#pragma unroll
        for (int o = GS / 2; o > 0; o >>= 1) {
            const float ta = __shfl_xor_sync(0xffffffffu, a, o);
            const float tb = __shfl_xor_sync(0xffffffffu, b, o);
            Pair t;
            t.hi = __shfl_xor_sync(0xffffffffu, ga.hi, o);
            t.lo = __shfl_xor_sync(0xffffffffu, ga.lo, o);
            a += ta;
            b += tb;
            pair_add(ga, t);
        }
        g = ga.hi + ga.lo;
        return;
    }
    T a2 = T(0), b2 = T(0);
    a = T(0);
    b = T(0);
#pragma unroll
    for (int e = 0; e < NE; e += 2) {
        a = fma(x[e], x[e], a);
        b = fma(y[e], y[e], b);
        if (e + 1 < NE) {
            a2 = fma(x[e + 1], x[e + 1], a2);
            b2 = fma(y[e + 1], y[e + 1], b2);
        }
    }
    a += a2;
    b += b2;
    if constexpr (sizeof(T) == 4) {
        Pair ga{0.f, 0.f}, gb{0.f, 0.f};
#pragma unroll
        for (int e = 0; e < NE; e += 2) {
            pair_add_prod(ga, x[e], y[e]);
            if (e + 1 < NE) pair_add_prod(gb, x[e + 1], y[e + 1]);
        }
        pair_add(ga, gb);
#pragma unroll
        for (int o = GS / 2; o > 0; o >>= 1) {
            const float ta = __shfl_xor_sync(0xffffffffu, a, o);
            const float tb = __shfl_xor_sync(0xffffffffu, b, o);
            Pair t;
            t.hi = __shfl_xor_sync(0xffffffffu, ga.hi, o);
            t.lo = __shfl_xor_sync(0xffffffffu, ga.lo, o);
            a += ta;
            b += tb;
            pair_add(ga, t);
        }
        g = ga.hi + ga.lo;
    } else {
        double ga = 0.0;
#pragma unroll
        for (int e = 0; e < NE; ++e) ga = fma(x[e], y[e], ga);
        a = group_sum<GS>(a); b = group_sum<GS>(b); g = group_sum<GS>(ga);
    }
}

// One cyclic sweep of one-sided Jacobi on the columns of Mc (column-major,
// column c at Mc + c * L, L <= NE * GS); pairs handled by groups of GS lanes,
// each lane holding up to NE entries of both columns in registers. Returns the
// number of rotations; *mxc2 receives the largest squared cosine g^2 / (a b)
// among the rotated pairs (as the bits of a nonnegative float).
template <typename T, int GS, int NE>
__device__ int jacobi_sweep(T* Mc, int L, int Lp, T tol, T tiny, int* nrot, unsigned* mxc2) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kGroupsPerWarp = 32 / GS;
    const int groups = ((int)blockDim.x >> 5) * kGroupsPerWarp, gl = lane % GS;
    const int m = Lp - 1;
    if (tid == 0) { *nrot = 0; *mxc2 = 0u; }
    __syncthreads();
    int mine = 0;
    float c2max = 0.f;
    for (int rnd = 0; rnd < m; ++rnd) {
        // the loop bound is uniform across a warp, so all 32 lanes reach every
        // shuffle below; groups without a pair take part with zeros
        for (int base = warp * kGroupsPerWarp; base < Lp / 2; base += groups) {
            const int pi = base + lane / GS;
            int p = L, q = L;
            if (pi < Lp / 2) {
                if (pi == 0) {
                    p = rnd; q = m;
                } else {
                    p = rnd + pi; if (p >= m) p -= m;
                    q = rnd - pi; if (q < 0) q += m;
                }
            }
            const bool live = p < L && q < L;
            T* cp = Mc + (live ? p : 0) * L;
            T* cq = Mc + (live ? q : 0) * L;
            T x[NE], y[NE];
#pragma unroll
            for (int e = 0; e < NE; ++e) {
                const int r = gl + e * GS;
                const bool in = live && r < L;
                x[e] = in ? cp[r] : T(0);
                y[e] = in ? cq[r] : T(0);
            }
            T a, b, g;
            pair_sums<T, GS, NE>(x, y, a, b, g);
            if (live && fabs(g) > tiny && g * g > tol * tol * a * b) {
                T c, s;
                rotation(a, b, g, c, s);
                if constexpr (sizeof(T) == 4 && NE % 2 == 0) {
                    // the squared cosine only steers the test of all pairs: an approximate quotient
                    c2max = fmaxf(c2max, __fdividef(g * g, a * b));
                    const f2 C2 = pk2(c, c), S2 = pk2(s, s);
#pragma unroll
                    for (int e = 0; e < NE; e += 2) {
                        const f2 X = pk2(x[e], x[e + 1]), Y = pk2(y[e], y[e + 1]);
                        float u0, u1, v0, v1;
                        up2(fma2(C2, X, sub2(0ull, mul2(S2, Y))), u0, u1);
                        up2(fma2(S2, X, mul2(C2, Y)), v0, v1);
                        const int r = gl + e * GS;
                        if (r < L) { cp[r] = u0; cq[r] = v0; }
                        if (r + GS < L) { cp[r + GS] = u1; cq[r + GS] = v1; }
                    }
                } else {
                    c2max = fmaxf(c2max, (float)((g / a) * (g / b)));
#pragma unroll
                    for (int e = 0; e < NE; ++e) {
                        const int r = gl + e * GS;
                        if (r < L) {
                            cp[r] = c * x[e] - s * y[e];
                            cq[r] = s * x[e] + c * y[e];
                        }
                    }
                }
                mine += gl == 0;
            }
        }
        __syncthreads();
    }
    if (mine) atomicAdd(nrot, mine);
    if (c2max > 0.f) atomicMax(mxc2, __float_as_uint(c2max));
    __syncthreads();
    const int n = *nrot;
    __syncthreads();
    return n;
}

// True when some pair of the L columns would still rotate (the test of
// jacobi_sweep on every pair at once, columns unchanged): what a sweep that
// rotates nothing establishes, at the cost of one round's arithmetic per
// L / 2 pairs and a single barrier.
template <typename T, int GS, int NE>
__device__ bool jacobi_pending(const T* Mc, int L, T tol, T tiny, int* flag) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kGroupsPerWarp = 32 / GS;
    const int groups = ((int)blockDim.x >> 5) * kGroupsPerWarp, gl = lane % GS;
    const int npairs = L * (L - 1) / 2;
    if (tid == 0) *flag = 0;
    __syncthreads();
    bool mine = false;
    for (int base = warp * kGroupsPerWarp; base < npairs; base += groups) {
        const int pi = base + lane / GS;
        const bool live = pi < npairs;
        // pair number pi -> (p, q), p < q: row p holds L - 1 - p pairs
        int p = 0, rem = live ? pi : 0;
        while (rem >= L - 1 - p) { rem -= L - 1 - p; ++p; }
        const int q = p + 1 + rem;
        const T* cp = Mc + p * L;
        const T* cq = Mc + q * L;
        T x[NE], y[NE];
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const int r = gl + e * GS;
            const bool in = live && r < L;
            x[e] = in ? cp[r] : T(0);
            y[e] = in ? cq[r] : T(0);
        }
        T a, b, g;
        pair_sums<T, GS, NE>(x, y, a, b, g);
        if (live && fabs(g) > tiny && g * g > tol * tol * a * b) mine = true;
    }
    if (mine) *flag = 1;
    __syncthreads();
    const bool any = *flag != 0;
    __syncthreads();
    return any;
}

// Shared-memory layout of the extraction's last CTA (byte offsets).
struct XLayout {
    size_t rf, g, h, dinv, sig, inrm, dots, perm, qnrm, rdiag, cmap, total;
};
__host__ __device__ inline size_t up16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline size_t zmax(size_t a, size_t b) { return a > b ? a : b; }
__host__ __device__ inline XLayout xlayout(int L, int R, int elem) {
    const int Lp = L + (L & 1);
    const size_t np = packed_size(L);
    XLayout x;
    x.rf = 0;                                                       // packed R2
    x.g = up16(8 * np);                                             // packed P / M, later B = R^T
    x.h = x.g + up16(zmax(8 * np, (size_t)elem * Lp * L));          // packed products, M^T, later U_M
    x.dinv = x.h + up16(zmax(8 * np, (size_t)elem * Lp * L));
    x.sig = x.dinv + up16((size_t)8 * L);
    x.inrm = x.sig + up16((size_t)elem * Lp);
    x.dots = x.inrm + up16((size_t)elem * Lp);
    x.perm = x.dots + up16((size_t)elem * R);
    x.qnrm = x.perm + up16(sizeof(int) * Lp);                      // [2][Lp] pivoting norms
    x.rdiag = x.qnrm + up16((size_t)elem * 2 * Lp);                 // [Lp] diagonal of R
    x.cmap = x.rdiag + up16((size_t)elem * Lp);                     // [2][Lp] pivot order
    x.total = x.cmap + up16(sizeof(int) * 2 * Lp);
    return x;
}

// Grid of Gram CTAs over Q1 (kXT threads each). The last CTA: Cholesky
// Entries (scalars S) from a back-substitution stage to its U_M (T, [R][L]).
__host__ __device__ inline size_t bs_um_offset(int L) { return ((size_t)packed_size(L) + (size_t)L + 1) & ~size_t(1); }

// W(:, c0 .. c0 + kBsCols - 1) = R2^-1 U_M(:, ...) by one warp: lane q keeps
// u_k - sum_{l' > l} R2_kl' w_l' for the rows k = q + 32 m (m < kBsRows, so
// L <= 128); row l is finished by its lane, broadcast, and subtracted from
// every row above it, so each row costs one dependent step, with the group's
// columns in flight together.
template <typename T>
__device__ __forceinline__ void backsub_group(const T* __restrict__ UM, const typename SmallScalar<T>::type* Rf,
                                              const typename SmallScalar<T>::type* dinv, int L, int R,
                                              typename SmallScalar<T>::type* __restrict__ Wout, int c0, int lane) {
    using S = typename SmallScalar<T>::type;
    using F = Sc<S>;
    S acc[kBsCols][kBsRows];
#pragma unroll
    for (int c = 0; c < kBsCols; ++c)
#pragma unroll
        for (int m = 0; m < kBsRows; ++m) {
            const int k = lane + 32 * m;
            acc[c][m] = (c0 + c < R && k < L) ? to_s<S>(UM[(size_t)(c0 + c) * L + k]) : F::zero();
        }
    for (int l = L - 1; l >= 0; --l) {
        const int src = l & 31, ml = l >> 5;
        const S d = dinv[l];
        S rkl[kBsRows];                                      // R2_kl for this lane's rows above l
#pragma unroll
        for (int m = 0; m < kBsRows; ++m) {
            const int k = lane + 32 * m;
            rkl[m] = (32 * m < l && k < l) ? Rf[packed_index(k, l, L)] : F::zero();
        }
#pragma unroll
        for (int c = 0; c < kBsCols; ++c) {
            S v = acc[c][0];
#pragma unroll
            for (int m = 1; m < kBsRows; ++m)
                if (ml == m) v = acc[c][m];
            const S w = shfl_s(v * d, src);
            if (lane == src && c0 + c < R) Wout[(size_t)(c0 + c) * L + l] = w;
#pragma unroll
            for (int m = 0; m < kBsRows; ++m) {
                if (32 * m >= l) break;                        // the same for the whole warp
                if (lane + 32 * m < l) acc[c][m] = F::fma(-rkl[m], w, acc[c][m]);
            }
        }
    }
}

// Q1^T Q1 = R2^T R2, M = R2 P with P = prev[nprev-1] ... prev[0] (packed
// factors fstride apart; prev[nprev-1] is R1), pivoted QR of M^T, Jacobi on
// R^T, U_M (rounding-level columns re-orthogonalised) and W = R2^-1 U_M for the
// R leading columns
// (scalar S, L x R, column-major). A column with no direction left gets W = 0
// (the final pass completes it).
template <typename T>
__device__ __forceinline__ void extract_body(const T* __restrict__ X, int64_t I, int L, int rows,
                                             typename SmallScalar<T>::type* __restrict__ partial, unsigned* ticket,
                                             const typename SmallScalar<T>::type* __restrict__ prev, size_t fstride,
                                             int nprev, int R, typename SmallScalar<T>::type* __restrict__ Wout,
                                             int* status, int bid, int nblk,
                                             typename SmallScalar<T>::type* __restrict__ stage = nullptr) {
    using S = typename SmallScalar<T>::type;
    using F = Sc<S>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    gram_partial<T, S>(X, I, L, rows, partial, smem_raw, bid);
    if (!last_cta(ticket, nblk)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kXT / 32;
    const int Lp = L + (L & 1);
    const int np = (int)packed_size(L);
    const XLayout lay = xlayout(L, R, sizeof(T));
    S* Rf = reinterpret_cast<S*>(smem_raw + lay.rf);
    S* G = reinterpret_cast<S*>(smem_raw + lay.g);
    S* H = reinterpret_cast<S*>(smem_raw + lay.h);
    S* dinv = reinterpret_cast<S*>(smem_raw + lay.dinv);   // [L] 1 / R2_kk
    T* sig = reinterpret_cast<T*>(smem_raw + lay.sig);     // [Lp] column norms of the rotated M
    T* inrm = reinterpret_cast<T*>(smem_raw + lay.inrm);   // [Lp] their reciprocals
    T* dots = reinterpret_cast<T*>(smem_raw + lay.dots);   // [R] Gram-Schmidt coefficients
    int* perm = reinterpret_cast<int*>(smem_raw + lay.perm);
    T* qnrm = reinterpret_cast<T*>(smem_raw + lay.qnrm);
    T* rdiag = reinterpret_cast<T*>(smem_raw + lay.rdiag);
    int* cmap = reinterpret_cast<int*>(smem_raw + lay.cmap);
    T* Mt = reinterpret_cast<T*>(H);                       // M^T column-major [Lp][L], once M is in G
    __shared__ int nrot;
    __shared__ int graded;
    __shared__ T fro2;
    __shared__ T nrm2;
    __shared__ unsigned long long mx_bits;

    reduce_cholesky<T, S>(partial, nblk, L, I, G, Rf, dinv, reinterpret_cast<int*>(H), ticket, status);

    // M = R2 prev[nprev-1] ... prev[0]: products of packed upper triangles, one
    // thread per output entry, alternating between H and G so the last lands in G
    const S* src = prev;
    for (int f = 1; f <= nprev; ++f) {
        const S* Fm = f < nprev ? prev + (size_t)f * fstride : Rf;
        S* dst = ((nprev - f) & 1) ? H : G;
        for (int p = tid; p < L * L; p += kXT) {
            const int a = p / L, c = p % L;
            if (c < a) continue;
            S acc0 = F::zero(), acc1 = F::zero();
            // (a, b) and (b, c) for b = a, a + 1, ...: packed(b + 1, c) = packed(b, c) + L - b - 1
            int ia = packed_index(a, a, L), ib = packed_index(a, c, L);
            int b = a;
            for (; b + 1 <= c; b += 2) {
                const int ib1 = ib + L - b - 1;
                acc0 = F::fma(Fm[ia], src[ib], acc0);
                acc1 = F::fma(Fm[ia + 1], src[ib1], acc1);
                ia += 2;
                ib = ib1 + L - b - 2;
            }
            if (b == c) acc0 = F::fma(Fm[ia], src[ib], acc0);
            dst[packed_index(a, c, L)] = acc0 + acc1;
        }
        __syncthreads();
        src = dst;
    }
    // M^T scaled by a power of two (largest entry in [1, 2)) and stored in T
    if (tid == 0) { mx_bits = 0ull; fro2 = T(0); }
    __syncthreads();
    {
        double mxl = 0.0;
        for (int p = tid; p < np; p += kXT) mxl = fmax(mxl, fabs(F::to_double(G[p])));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mxl = fmax(mxl, __shfl_xor_sync(0xffffffffu, mxl, o));
        if (lane == 0) atomicMax(&mx_bits, (unsigned long long)__double_as_longlong(mxl));
    }
    __syncthreads();
    const double mxv = __longlong_as_double((long long)mx_bits);
    int ex = 0;
    if (mxv > 0.0) frexp(mxv, &ex);
    {
        T s2 = T(0);
        for (int p = tid; p < Lp * L; p += kXT) {
            const int c = p / L, a = p % L;
            const T v = (c < L && c <= a) ? (T)ldexp(F::to_double(G[packed_index(c, a, L)]), 1 - ex) : T(0);
            Mt[p] = v;
            s2 += v * v;
        }
        s2 = warp_sum(s2);
        if (lane == 0) atomicAdd(&fro2, s2);
    }
    __syncthreads();
    // Preconditioning (Drmac and Veselic, 2008): M^T(:, cmap) = Q R by QR with
    // column pivoting, so M = P R^T Q^T and the left singular vectors of M are
    // those of B = R^T with rows permuted (row j of B is row cmap[j] of M's).
    // The pivoted R is row-graded, B column-graded, and one-sided Jacobi on B's
    // columns needs about half the sweeps it takes on M's. The reflectors are
    // columnwise backward stable: each row of M is perturbed relative to its
    // own norm, as rounding M to T already does.
    if (L <= 32) pivoted_qr<T, 4>(Mt, L, Lp, qnrm, rdiag, cmap);
    else if (L <= 64) pivoted_qr<T, 8>(Mt, L, Lp, qnrm, rdiag, cmap);
    else if (L <= 80) pivoted_qr<T, 10>(Mt, L, Lp, qnrm, rdiag, cmap);
    else if (L <= 96) pivoted_qr<T, 12>(Mt, L, Lp, qnrm, rdiag, cmap);
    else pivoted_qr<T, 16>(Mt, L, Lp, qnrm, rdiag, cmap);
    // A sketch that is numerically rank-deficient in T (its smallest pivot below
    // 2^-20 of the largest, e.g. the Hilbert tensor's) keeps the unconditioned
    // Jacobi on M's columns: there every column has the norm of M's leading rows,
    // the rounding a rotation leaves lies along the strong directions, and the
    // re-orthogonalisation below removes it from the weak columns, which gives
    // better factors on such sketches than the graded B (measured). Otherwise B.
    if (tid == 0) graded = !(fabs(rdiag[L - 1]) >= T(0x1p-20) * fabs(rdiag[0]));
    __syncthreads();
    int* fmap = cmap + (L & 1) * Lp;
    T* Bc = graded ? Mt : reinterpret_cast<T*>(G);         // the matrix the Jacobi rotates, [Lp][L]
    T* UM = graded ? reinterpret_cast<T*>(G) : Mt;         // U_M, column-major [R][L], once Bc is final
    if (graded) {
        for (int p = tid; p < Lp * L; p += kXT) {
            const int c = p / L, a = p % L;
            Bc[p] = (c < L && a <= c) ? (T)ldexp(F::to_double(G[packed_index(a, c, L)]), 1 - ex) : T(0);
        }
        for (int j = tid; j < L; j += kXT) fmap[j] = j;
    } else {
        for (int p = tid; p < Lp * L; p += kXT) {
            const int c = p / L, a = p % L;
            T v = T(0);
            if (c < L) v = a == c ? rdiag[c] : (a > c ? Mt[fmap[a] * L + c] : T(0));
            Bc[p] = v;
        }
    }
    __syncthreads();
    // rotate while a pair's cosine exceeds 4 eps, g^2 > tol^2 a b. B's columns
    // are graded and carry rounding relative to their own norms (the reflectors
    // are columnwise stable), so for B the test is relative to the pair alone
    // (tiny only keeps underflowed couplings out; B's pivots lie within 2^20 of
    // each other and the largest entry of M is in [1, 2), so tol^2 a b stays
    // above the smallest normal); M's columns carry rounding of the whole
    // matrix, so there a coupling must also exceed eps^2 ||M||_F^2. The stored columns carry rounding
    // of their own, so the sweep count is capped. Once a sweep's largest rotated cosine is below 1e-3
    // (Jacobi converges quadratically from there), all pairs are tested at once
    // before another sweep is spent: when none would rotate, that sweep would
    // have rotated nothing.
    const T eps = sizeof(T) == 4 ? (T)FLT_EPSILON : (T)DBL_EPSILON;
    const T tol = T(4) * eps;
    const T tiny = graded ? eps * eps * fro2 : (sizeof(T) == 4 ? (T)FLT_MIN : (T)DBL_MIN);
    __shared__ unsigned mxc2;
    for (int sweep = 0; sweep < 20; ++sweep) {
        int n;
        bool pending;
        // groups of 8 lanes, one pair each, every pair of a round in flight at once;
        // each lane holds NE >= L / 8 entries of both columns (a round is bound by
        // instruction issue, so lanes do not repeat the reductions needlessly)
#define TK_JACOBI(NE)                                                                  \
        n = jacobi_sweep<T, 8, NE>(Bc, L, Lp, tol, tiny, &nrot, &mxc2);                \
        pending = n > 0 && (__uint_as_float(mxc2) >= 1e-6f ||                          \
                            jacobi_pending<T, 8, NE>(Bc, L, tol, tiny, &nrot));
        if (L <= 32) { TK_JACOBI(4) }
        else if (L <= 64) { TK_JACOBI(8) }
        else if (L <= 80) { TK_JACOBI(10) }
        else if (L <= 96) { TK_JACOBI(12) }
        else { TK_JACOBI(16) }                                                      // L <= 128
#undef TK_JACOBI
        if (!pending) break;
    }
    // singular values (column norms), decreasing order, lower index first on ties
    for (int c = warp; c < L; c += nwarps) {
        DotAcc<T> s;
        for (int r = lane; r < L; r += 32) s.add(Bc[c * L + r], Bc[c * L + r]);
        s.reduce();
        if (lane == 0) {
            const T sg = sqrt((T)s.value());
            sig[c] = sg;
            inrm[c] = sg > T(0) ? T(1) / sg : T(0);
        }
    }
    __syncthreads();
    // (a total order: a NaN norm ranks below every number, so perm is a
    // permutation whatever the data and every index taken from it stays in range)
    for (int c = tid; c < L; c += kXT) {
        const T sc = sig[c] == sig[c] ? sig[c] : T(-1);
        int rank = 0;
        for (int d = 0; d < L; ++d) {
            const T sd = sig[d] == sig[d] ? sig[d] : T(-1);
            rank += (sd > sc) || (sd == sc && d < c);
        }
        perm[rank] = c;
    }
    __syncthreads();
    const T weak = T(64) * eps * sig[perm[0]];
    // U_M: B's rotated columns in decreasing order, normalised, rows in M's order
    for (int p = tid; p < L * R; p += kXT) {
        const int r = p / L, j = p % L;
        const int c = perm[r];
        UM[(size_t)r * L + fmap[j]] = Bc[c * L + j] * inrm[c];
    }
    __syncthreads();
    // rounding-level columns: classical Gram-Schmidt against every earlier
    // column, twice (coefficients one warp each, then one update per entry)
    for (int r = 0; r < R; ++r) {
        if (!(sig[perm[r]] <= weak)) continue;
        T* u = UM + (size_t)r * L;
        for (int pass = 0; pass < 2; ++pass) {
            for (int j = warp; j < r; j += nwarps) {
                const T* v = UM + (size_t)j * L;
                DotAcc<T> s;
                for (int a = lane; a < L; a += 32) s.add(v[a], u[a]);
                s.reduce();
                if (lane == 0) dots[j] = (T)s.value();
            }
            __syncthreads();
            for (int a = tid; a < L; a += kXT) {
                T acc = u[a];
                for (int j = 0; j < r; ++j) acc -= dots[j] * UM[(size_t)j * L + a];
                u[a] = acc;
            }
            __syncthreads();
        }
        if (warp == 0) {
            DotAcc<T> s;
            for (int a = lane; a < L; a += 32) s.add(u[a], u[a]);
            s.reduce();
            if (lane == 0) nrm2 = (T)s.value();
        }
        __syncthreads();
        const T n2 = nrm2;
        const bool ok = n2 > T(1e-6);                  // else the sketch has no direction left here
        const T f = ok ? T(1) / sqrt(n2) : T(0);
        for (int a = tid; a < L; a += kXT) u[a] *= f;
        __syncthreads();
    }
    // W(:, r) = R2^-1 U_M(:, r) (backsub_group): with a stage, R2, 1/R2_kk and U_M
    // go to global memory and backsub_kernel runs the column groups on CTAs of
    // their own (the steps are serial and issue-bound on one SM); else here, one
    // warp per group
    if (stage) {
        const int np = (int)packed_size(L);
        for (int p = tid; p < np; p += kXT) stage[p] = Rf[p];
        for (int k = tid; k < L; k += kXT) stage[np + k] = dinv[k];
        T* um = reinterpret_cast<T*>(stage + bs_um_offset(L));
        for (int e = tid; e < L * R; e += kXT) um[e] = UM[e];
        return;
    }
    for (int c0 = warp * kBsCols; c0 < R; c0 += nwarps * kBsCols) backsub_group<T>(UM, Rf, dinv, L, R, Wout, c0, lane);
}

// U(:, r) = X W(:, r) in paired precision, one thread per entry of U.
template <typename T>
__device__ __forceinline__ void form_u_body(const T* __restrict__ X, int64_t I, int L, int R,
                                            const typename SmallScalar<T>::type* __restrict__ W, T* __restrict__ U,
                                            int bid, int nblk) {
    const int64_t n = I * R;
    for (int64_t e = (int64_t)bid * kT + threadIdx.x; e < n; e += (int64_t)nblk * kT) {
        const int r = (int)(e / I);
        const int64_t i = e - (int64_t)r * I;
        const auto* w = W + (int64_t)r * L;
        DotAcc<T> s;
        for (int c = 0; c < L; ++c) {
            const T x = X[(int64_t)c * I + i];
            if constexpr (sizeof(T) == 4) {
                s.add(x, w[c].hi);
                s.add(x, w[c].lo);
            } else {
                s.add(x, w[c]);
            }
        }
        U[e] = (T)s.value();
    }
}

constexpr int kFRows = 64;               // rows of U staged per step of the final Gram

struct FLayout {
    size_t g, w, rt, dinv, valid, idx, lev, xs, total;
};
__host__ __device__ inline FLayout flayout(int R, int elem, int64_t I) {
    const size_t np = packed_size(R);
    FLayout f;
    f.g = 0;                                              // packed Gram (as Pair sums), then R^-1
    f.w = up16(8 * np);                                   // packed Cholesky factor; with rt: coefficients
    f.rt = f.w + up16(8 * np);                            // transposed factor
    f.dinv = f.rt + up16(8 * np);
    f.valid = f.dinv + up16((size_t)8 * R);
    f.idx = f.valid + up16(sizeof(int) * (size_t)R);      // [2][R]: dropped columns, candidate rows
    f.lev = f.idx + up16(sizeof(int) * 2 * (size_t)R);    // [I] row leverages
    f.xs = f.lev + up16((size_t)elem * (size_t)I);
    f.total = f.xs + up16((size_t)elem * kFRows * R);
    return f;
}

// Final pass over U (I x R, column-major), one CTA:
//   1. Gram U^T U in paired precision. If it is within 8 eps of I, U is kept.
//   2. Otherwise Cholesky U^T U = R_U^T R_U, dropping every column whose
//      remaining squared norm is below 1/4 of its own (it lies mostly in the
//      span of the earlier columns, or is zero), and U <- U R_U^-1 in place:
//      column r mixes with earlier columns only, so the span of the first k
//      columns is unchanged for every k. This restores orthonormality where
//      the sketch was numerically rank-deficient and CholeskyQR could not.
//   3. Dropped columns, all at once: the m dropped columns (in order) take the
//      unit vectors e_k of the first m rows k whose leverage
//      ||U_valid(k, :)||^2 leaves a long residual, 1 - leverage_k >
//      (I - d) / (2 I) for d valid columns (the leverages average d / I, so
//      enough rows qualify), projected out of the valid columns twice
//      (e_k - U_v U_v(k, :)^T, then once more by inner products); steps 1-2
//      then run once more over all R columns to orthonormalise them.
//   4. Sign rule: each column's largest-magnitude entry positive (lowest row on ties).
//   5. Any column still dropped (not expected): the first unit vector e_k (k
//      increasing) that keeps a long residual after two Gram-Schmidt passes
//      against every valid column. The squared residuals of e_0 .. e_{I-1}
//      average (I - d) / I for d valid columns, so accepting one above half
//      that average always succeeds.
// With staged set, U is copied into shared memory after the layout's other
// regions (the host checks that it fits), worked on there and copied back at
// the end, which keeps the loops over U off the global-memory latency.
// Partial Grams of U's rows by a grid of CTAs; the last one sums them in block
// order and records in *ok whether U^T U is within 8 eps of I, in which case
// the final pass keeps U and only applies the sign rule.
template <typename T>
__device__ __forceinline__ void ugram_check_body(const T* __restrict__ U, int64_t I, int R, int rows,
                                                 typename SmallScalar<T>::type* __restrict__ partial, unsigned* ticket,
                                                 int* ok, int bid, int nblk) {
    using S = typename SmallScalar<T>::type;
    using F = Sc<S>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    gram_partial<T, S>(U, I, R, rows, partial, smem_raw, bid);
    if (!last_cta(ticket, nblk)) return;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    const int np = (int)packed_size(R);
    const double eps = sizeof(T) == 4 ? (double)FLT_EPSILON : DBL_EPSILON;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        S acc = ld_cg(partial + p);
        for (int b = 1; b < nblk; ++b) acc = acc + ld_cg(partial + (int64_t)b * np + p);
        int a = 0, rem = p;
        while (rem >= R - a) { rem -= R - a; ++a; }
        const double dev = fabs(F::to_double(acc) - (rem == 0 ? 1.0 : 0.0));
        if (!(dev <= 8.0 * eps)) bad = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *ok = !bad;
        *ticket = 0;                                     // ready for the next use
    }
}

template <typename T>
__device__ __forceinline__ void finish_body(T* __restrict__ Ug, int64_t I, int R, int staged,
                                            const int* __restrict__ pre_ok) {
    using S = typename SmallScalar<T>::type;
    using F = Sc<S>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FLayout lay = flayout(R, sizeof(T), I);
    Pair* GP = reinterpret_cast<Pair*>(smem_raw + lay.g);
    S* Ri = reinterpret_cast<S*>(smem_raw + lay.g);
    S* W = reinterpret_cast<S*>(smem_raw + lay.w);
    S* RT = reinterpret_cast<S*>(smem_raw + lay.rt);
    S* dinv = reinterpret_cast<S*>(smem_raw + lay.dinv);
    int* valid = reinterpret_cast<int*>(smem_raw + lay.valid);
    T* xs = reinterpret_cast<T*>(smem_raw + lay.xs);     // [kFRows][R]
    int* drop = reinterpret_cast<int*>(smem_raw + lay.idx);   // [R] dropped columns, in order
    int* cand = drop + R;                                      // [R] their candidate rows
    T* lev = reinterpret_cast<T*>(smem_raw + lay.lev);    // [I]
    T* coef = reinterpret_cast<T*>(smem_raw + lay.w);     // [R][R] projection coefficients (W and RT)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kST / 32;
    const int np = (int)packed_size(R);
    T* U = staged ? reinterpret_cast<T*>(smem_raw + lay.total) : Ug;
    if (staged)
        for (int64_t e = tid; e < I * R; e += kST) U[e] = Ug[e];
    __shared__ int offdiag, ndrop;
    __shared__ double red[kST / 32];
    __shared__ double bcast;
    __shared__ T bvs[kST / 32];
    __shared__ int64_t bis[kST / 32];

    const double eps = sizeof(T) == 4 ? (double)FLT_EPSILON : DBL_EPSILON;
    // U^T U already checked within 8 eps of I by the grid of ugram_check_kernel:
    // nothing to repair, only the sign rule
    const bool checked_ok = *pre_ok != 0;
    if (checked_ok) {
        for (int k = tid; k < R; k += kST) valid[k] = 1;
        __syncthreads();
    }
    for (int pass = 0; pass < 2 && !checked_ok; ++pass) {
    // 1. Gram (FP32 data: Pair sums; FP64 data: the Pair slots hold one double)
    double* GD = reinterpret_cast<double*>(smem_raw + lay.g);
    __syncthreads();
    for (int p = tid; p < np; p += kST) {
        if constexpr (sizeof(T) == 4) GP[p] = Pair{0.f, 0.f};
        else GD[p] = 0.0;
    }
    if (tid == 0) offdiag = 0;
    for (int64_t r0 = 0; r0 < I; r0 += kFRows) {
        const int nr = (int)min((int64_t)kFRows, I - r0);
        __syncthreads();
        for (int e = tid; e < nr * R; e += kST) {
            const int r = e % nr, c = e / nr;
            xs[r * R + c] = U[(int64_t)c * I + r0 + r];
        }
        __syncthreads();
        for (int p = tid; p < np; p += kST) {
            int a = 0, rem = p;
            while (rem >= R - a) { rem -= R - a; ++a; }
            const int b = a + rem;
            // two interleaved chains (even and odd rows), combined in a fixed order
            if constexpr (sizeof(T) == 4) {
                Pair acc = GP[p], acc2{0.f, 0.f};
                int r = 0;
                for (; r + 1 < nr; r += 2) {
                    pair_add_prod(acc, xs[r * R + a], xs[r * R + b]);
                    pair_add_prod(acc2, xs[(r + 1) * R + a], xs[(r + 1) * R + b]);
                }
                if (r < nr) pair_add_prod(acc, xs[r * R + a], xs[r * R + b]);
                pair_add(acc, acc2);
                GP[p] = acc;
            } else {
                double acc = GD[p], acc2 = 0.0;
                int r = 0;
                for (; r + 1 < nr; r += 2) {
                    acc = fma(xs[r * R + a], xs[r * R + b], acc);
                    acc2 = fma(xs[(r + 1) * R + a], xs[(r + 1) * R + b], acc2);
                }
                if (r < nr) acc = fma(xs[r * R + a], xs[r * R + b], acc);
                GD[p] = acc + acc2;
            }
        }
    }
    __syncthreads();
    for (int p = tid; p < np; p += kST) {
        int a = 0, rem = p;
        while (rem >= R - a) { rem -= R - a; ++a; }
        S g;
        if constexpr (sizeof(T) == 4) g = two_sum(GP[p].hi, GP[p].lo);
        else g = GD[p];
        W[p] = g;
        const double dev = fabs(F::to_double(g) - (rem == 0 ? 1.0 : 0.0));
        if (!(dev <= 8.0 * eps)) offdiag = 1;
    }
    for (int k = tid; k < R; k += kST) valid[k] = 1;
    __syncthreads();
    if (!offdiag) break;
    {
        // 2. Cholesky with column dropping (G kept in RT for the reference norms)
        for (int p = tid; p < np; p += kST) RT[p] = W[p];
        __syncthreads();
        for (int k = 0; k < R; ++k) {
            if (tid == 0) {
                const int kk = packed_index(k, k, R);
                const S d = W[kk];
                const bool keep = F::gt(d, RT[kk] * F::from_double(0.25)) && F::finite(d);
                valid[k] = keep;
                if (keep) {
                    const S y = F::rsqrt(d);
                    W[kk] = d * y;
                    dinv[k] = y;
                } else {
                    W[kk] = F::one();
                    dinv[k] = F::one();
                }
            }
            __syncthreads();
            const int kk = packed_index(k, k, R);
            if (!valid[k]) {
                for (int j = k + 1 + tid; j < R; j += kST) W[kk + (j - k)] = F::zero();
                __syncthreads();
                continue;
            }
            const S y = dinv[k];
            for (int j = k + 1 + tid; j < R; j += kST) W[kk + (j - k)] = W[kk + (j - k)] * y;
            __syncthreads();
            for (int i = k + 1 + warp; i < R; i += nw) {
                const S cki = W[kk + (i - k)];
                S* ri = W + packed_index(i, i, R);
                for (int j = i + lane; j < R; j += 32) ri[j - i] = ri[j - i] - cki * W[kk + (j - k)];
            }
            __syncthreads();
        }
        upper_inverse<S>(W, dinv, R, RT, Ri);
        // U <- U R_U^-1, one thread per row, columns from the last (in place)
        for (int64_t i = tid; i < I; i += kST) {
            for (int l = R - 1; l >= 0; --l) {
                T v = T(0);
                if (valid[l]) {
                    DotAcc<T> acc;
                    for (int m = 0; m <= l; ++m) {
                        const S w = Ri[packed_index(m, l, R)];
                        const T x = U[(int64_t)m * I + i];
                        if constexpr (sizeof(T) == 4) {
                            acc.add(x, w.hi);
                            acc.add(x, w.lo);
                        } else {
                            acc.add(x, w);
                        }
                    }
                    v = (T)acc.value();
                }
                U[(int64_t)l * I + i] = v;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        int m = 0;
        for (int r = 0; r < R; ++r)
            if (!valid[r]) drop[m++] = r;
        ndrop = m;
    }
    __syncthreads();
    const int m = ndrop;
    if (m == 0 || pass == 1) break;
    // 3. candidates: the first m rows k (increasing) whose unit vector keeps a
    //    long residual, 1 - leverage_k > (I - valid columns) / (2 I)
    for (int64_t i = tid; i < I; i += kST) {
        T a = T(0);
        for (int r = 0; r < R; ++r)
            if (valid[r]) a = fma(U[(int64_t)r * I + i], U[(int64_t)r * I + i], a);
        lev[i] = a;
    }
    __syncthreads();
    if (tid == 0) {
        const T keep = T(0.5) * (T)(I - (R - m)) / (T)I;
        int t = 0;
        for (int64_t k = 0; k < I && t < m; ++k)
            if (T(1) - lev[k] > keep) cand[t++] = (int)k;
        for (int64_t k = 0; k < I && t < m; ++k) {         // any shortfall: the next rows in order
            bool used = false;
            for (int u = 0; u < t; ++u) used |= cand[u] == (int)k;
            if (!used) cand[t++] = (int)k;
        }
    }
    __syncthreads();
    // first projection, from the candidate rows of the valid columns
    for (int64_t e = tid; e < I * m; e += kST) {
        const int t = (int)(e / I);
        const int64_t i = e - (int64_t)t * I;
        const int k = cand[t];
        T v = i == k ? T(1) : T(0);
        for (int r = 0; r < R; ++r)
            if (valid[r]) v -= U[(int64_t)r * I + i] * U[(int64_t)r * I + k];
        U[(int64_t)drop[t] * I + i] = v;
    }
    __syncthreads();
    // second projection by inner products (one warp per pair)
    for (int pr = warp; pr < R * m; pr += nw) {
        const int r = pr / m, t = pr % m;
        T c = T(0);
        if (valid[r]) {
            DotAcc<T> acc;
            for (int64_t i = lane; i < I; i += 32) acc.add(U[(int64_t)r * I + i], U[(int64_t)drop[t] * I + i]);
            acc.reduce();
            c = (T)acc.value();
        }
        if (lane == 0) coef[r * m + t] = c;
    }
    __syncthreads();
    for (int64_t e = tid; e < I * m; e += kST) {
        const int t = (int)(e / I);
        const int64_t i = e - (int64_t)t * I;
        T v = U[(int64_t)drop[t] * I + i];
        for (int r = 0; r < R; ++r)
            if (valid[r]) v -= coef[r * m + t] * U[(int64_t)r * I + i];
        U[(int64_t)drop[t] * I + i] = v;
    }
    __syncthreads();
    }

    // 4. sign rule, one warp per column
    for (int r = warp; r < R; r += nw) {
        if (!valid[r]) continue;
        T bv = T(-1);
        int64_t bi = 0;
        for (int64_t i = lane; i < I; i += 32) {
            const T a = fabs(U[(int64_t)r * I + i]);
            if (a > bv) { bv = a; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (U[(int64_t)r * I + bi] < T(0))
            for (int64_t i = lane; i < I; i += 32) U[(int64_t)r * I + i] = -U[(int64_t)r * I + i];
    }
    __syncthreads();

    // 5. completion of columns still dropped (the residual is formed in U's own column)
    int nvalid = 0;
    for (int r = 0; r < R; ++r) nvalid += valid[r];
    int64_t k = 0;
    for (int r = 0; r < R; ++r) {
        if (valid[r]) continue;
        T* v = U + (int64_t)r * I;
        for (; k < I; ++k) {
            for (int64_t i = tid; i < I; i += kST) v[i] = (i == k) ? T(1) : T(0);
            __syncthreads();
            for (int pass = 0; pass < 2; ++pass) {
                for (int j = 0; j < R; ++j) {
                    if (!valid[j]) continue;
                    double s = 0.0;
                    for (int64_t i = tid; i < I; i += kST) s = fma((double)U[(int64_t)j * I + i], (double)v[i], s);
                    s = warp_sum(s);
                    if (lane == 0) red[warp] = s;
                    __syncthreads();
                    if (tid == 0) {
                        double t = 0.0;
                        for (int w = 0; w < nw; ++w) t += red[w];
                        bcast = t;
                    }
                    __syncthreads();
                    const double d = bcast;
                    for (int64_t i = tid; i < I; i += kST) v[i] = (T)((double)v[i] - d * (double)U[(int64_t)j * I + i]);
                    __syncthreads();
                }
            }
            double s = 0.0;
            T bv = T(-1);
            int64_t bi = 0;
            for (int64_t i = tid; i < I; i += kST) {
                s = fma((double)v[i], (double)v[i], s);
                if (fabs(v[i]) > bv) { bv = fabs(v[i]); bi = i; }
            }
            s = warp_sum(s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            if (lane == 0) { red[warp] = s; bvs[warp] = bv; bis[warp] = bi; }
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                T b = bvs[0];
                int64_t ii = bis[0];
                for (int w = 0; w < nw; ++w) {
                    t += red[w];
                    if (bvs[w] > b || (bvs[w] == b && bis[w] < ii)) { b = bvs[w]; ii = bis[w]; }
                }
                bcast = t > 0.5 * (double)(I - nvalid) / (double)I ? (v[ii] < T(0) ? -1.0 : 1.0) / sqrt(t) : 0.0;
            }
            __syncthreads();
            const double f = bcast;
            if (f != 0.0) {
                for (int64_t i = tid; i < I; i += kST) v[i] = (T)((double)v[i] * f);
                __syncthreads();
                if (tid == 0) valid[r] = 1;
                __syncthreads();
                ++nvalid;
                ++k;
                break;
            }
            __syncthreads();
        }
    }
    if (staged) {
        __syncthreads();
        for (int64_t e = tid; e < I * R; e += kST) Ug[e] = U[e];
    }
}

// ---------------------------------------------------------------- kernels
// One orthonormalisation per launch: the block programs above at blockIdx.x of gridDim.x.
template <typename T>
__global__ void __launch_bounds__(kST) gram_chol_kernel(const T* __restrict__ X, int64_t I, int L, int rows,
                                                       typename SmallScalar<T>::type* __restrict__ partial,
                                                       unsigned* ticket, typename SmallScalar<T>::type* __restrict__ R,
                                                       typename SmallScalar<T>::type* __restrict__ Rinv, int* status,
                                                       typename SmallScalar<T>::type* __restrict__ stage) {
    gram_chol_body<T>(X, I, L, rows, partial, ticket, R, Rinv, status, blockIdx.x, gridDim.x, stage);
}
// R^-1 of the packed upper-triangular R (1/R_kk in dinv), row i on warp i of the
// grid: x_ij = (delta_ij - sum_{k<j} x_ik R_kj) / R_jj, the sum accumulated in
// increasing k by the lane that owns column j, as upper_inverse forms it (the
// same operations in the same order, so the same bits), with x_ij broadcast
// from its lane once final. R and dinv are copied to shared memory first.
template <typename T>
__global__ void __launch_bounds__(128) tri_inverse_kernel(const typename SmallScalar<T>::type* __restrict__ R,
                                                          const typename SmallScalar<T>::type* __restrict__ dinv_g,
                                                          int L, typename SmallScalar<T>::type* __restrict__ Ri) {
    using S = typename SmallScalar<T>::type;
    using F = Sc<S>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* rs = reinterpret_cast<S*>(smem_raw);
    const int np = (int)packed_size(L);
    S* dv = rs + np;
#pragma unroll 4
    for (int p = threadIdx.x; p < np + L; p += 128) {
        if (p < np) rs[p] = R[p];
        else dv[p - np] = dinv_g[p - np];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int i = (int)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (i >= L) return;                                   // a whole warp
    S acc[kBsRows];
#pragma unroll
    for (int m = 0; m < kBsRows; ++m) acc[m] = F::zero();
    for (int j = i; j < L; ++j) {
        const int src = j & 31, mj = j >> 5;
        S a = acc[0];
#pragma unroll
        for (int m = 1; m < kBsRows; ++m)
            if (mj == m) a = acc[m];
        const S x = shfl_s(((i == j ? F::one() : F::zero()) - a) * dv[j], src);
        if (lane == src) Ri[packed_index(i, j, L)] = x;
#pragma unroll
        for (int m = 0; m < kBsRows; ++m) {
            const int k = lane + 32 * m;
            if (k > j && k < L) acc[m] = F::fma(x, rs[packed_index(j, k, L)], acc[m]);
        }
    }
}
template <typename T>
__global__ void __launch_bounds__(kT) apply_rinv_kernel(const T* __restrict__ X, int64_t I, int L,
                                                        const typename SmallScalar<T>::type* __restrict__ Rinv,
                                                        T* __restrict__ Q) {
    apply_rinv_body<T>(X, I, L, Rinv, Q, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void __launch_bounds__(kXT, 1) extract_kernel(const T* __restrict__ X, int64_t I, int L, int rows,
                                                      typename SmallScalar<T>::type* __restrict__ partial,
                                                      unsigned* ticket,
                                                      const typename SmallScalar<T>::type* __restrict__ prev,
                                                      size_t fstride, int nprev, int R,
                                                      typename SmallScalar<T>::type* __restrict__ Wout,
                                                      int* status, typename SmallScalar<T>::type* __restrict__ stage) {
    extract_body<T>(X, I, L, rows, partial, ticket, prev, fstride, nprev, R, Wout, status, blockIdx.x, gridDim.x,
                    stage);
}
// The back-substitution of a staged extraction: column group blockIdx.x on one
// warp, R2 and 1/R2_kk copied to shared memory first.
template <typename T>
__global__ void __launch_bounds__(128) backsub_kernel(const typename SmallScalar<T>::type* __restrict__ stage, int L,
                                                      int R, typename SmallScalar<T>::type* __restrict__ Wout) {
    using S = typename SmallScalar<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* rf = reinterpret_cast<S*>(smem_raw);
    const int np = (int)packed_size(L);
#pragma unroll 4
    for (int p = threadIdx.x; p < np + L; p += 128) rf[p] = stage[p];
    __syncthreads();
    const int c0 = ((int)blockIdx.x * 4 + (int)(threadIdx.x >> 5)) * kBsCols;
    if (c0 >= R) return;                                  // a whole warp
    backsub_group<T>(reinterpret_cast<const T*>(stage + bs_um_offset(L)), rf, rf + np, L, R, Wout, c0,
                     (int)(threadIdx.x & 31));
}
template <typename T>
__global__ void __launch_bounds__(kT) form_u_kernel(const T* __restrict__ X, int64_t I, int L, int R,
                                                    const typename SmallScalar<T>::type* __restrict__ W,
                                                    T* __restrict__ U) {
    form_u_body<T>(X, I, L, R, W, U, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void __launch_bounds__(kST) ugram_check_kernel(const T* __restrict__ U, int64_t I, int R, int rows,
                                                          typename SmallScalar<T>::type* __restrict__ partial,
                                                          unsigned* ticket, int* ok) {
    ugram_check_body<T>(U, I, R, rows, partial, ticket, ok, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void __launch_bounds__(kST) finish_kernel(T* __restrict__ Ug, int64_t I, int R, int staged,
                                                     const int* __restrict__ pre_ok) {
    finish_body<T>(Ug, I, R, staged, pre_ok);
}

// Grouped: the orthonormalisations of a batch's requests side by side, job
// blockIdx.y with its own parameters; CTAs beyond a job's count return at once
// (the Gram programs count their job's CTAs, not the grid's).
__global__ void orth_reset_group_kernel(const OrthJob* __restrict__ jobs) {
    const OrthJob j = jobs[blockIdx.x];
    if (threadIdx.x < 32) j.flag[threadIdx.x] = 0;     // the flag and ticket words (128 bytes)
}
template <typename T>
__global__ void __launch_bounds__(kST) gram_chol_group_kernel(const OrthJob* __restrict__ jobs) {
    using S = typename SmallScalar<T>::type;
    const OrthJob j = jobs[blockIdx.y];
    if ((int)blockIdx.x >= j.nblk) return;
    gram_chol_body<T>((const T*)j.X, j.I, j.L, j.rows, (S*)j.partial, j.ticket, (S*)(j.factor + j.fofs), (S*)j.W,
                      j.status, blockIdx.x, j.nblk);
}
template <typename T>
__global__ void __launch_bounds__(kT) apply_rinv_group_kernel(const OrthJob* __restrict__ jobs) {
    using S = typename SmallScalar<T>::type;
    const OrthJob j = jobs[blockIdx.y];
    apply_rinv_body<T>((const T*)j.X, j.I, j.L, (const S*)j.W, (T*)j.Q, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void __launch_bounds__(kXT, 1) extract_group_kernel(const OrthJob* __restrict__ jobs) {
    using S = typename SmallScalar<T>::type;
    const OrthJob j = jobs[blockIdx.y];
    if ((int)blockIdx.x >= j.nblk) return;
    extract_body<T>((const T*)j.Q, j.I, j.L, j.rows, (S*)j.partial, j.ticket, (const S*)j.factor,
                    (size_t)j.L * j.L, j.nprev + 1, j.R, (S*)j.W, j.status, blockIdx.x, j.nblk);
}
template <typename T>
__global__ void __launch_bounds__(kT) form_u_group_kernel(const OrthJob* __restrict__ jobs) {
    using S = typename SmallScalar<T>::type;
    const OrthJob j = jobs[blockIdx.y];
    form_u_body<T>((const T*)j.Q, j.I, j.L, j.R, (const S*)j.W, (T*)j.U, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void __launch_bounds__(kST) ugram_check_group_kernel(const OrthJob* __restrict__ jobs) {
    using S = typename SmallScalar<T>::type;
    const OrthJob j = jobs[blockIdx.y];
    if ((int)blockIdx.x >= j.nblk) return;
    ugram_check_body<T>((const T*)j.U, j.I, j.R, j.rows, (S*)j.partial, j.ticket, j.flag + 8, blockIdx.x, j.nblk);
}
template <typename T>
__global__ void __launch_bounds__(kST) finish_group_kernel(const OrthJob* __restrict__ jobs) {
    const OrthJob j = jobs[blockIdx.y];
    finish_body<T>((T*)j.U, j.I, j.R, j.staged, j.flag + 8);
}

}  // namespace

OrthPlan orth_plan(int64_t I, int L, int num_sms) {
    OrthPlan p{};
    p.I = I;
    p.L = L;
    // at least kGramRows rows per CTA (few partials for the serial reduction),
    // and the packed partials within 512 KB
    const int64_t np = (int64_t)packed_size(L);
    int64_t cap = (512 * 1024) / (np * 8);
    if (cap < 1) cap = 1;
    if (cap > num_sms) cap = num_sms;
    int64_t blocks = (I + kGramRows - 1) / kGramRows;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    p.gram_blocks = (int)blocks;
    return p;
}

static int gram_rows(const OrthPlan& p) { return (int)((p.I + p.gram_blocks - 1) / p.gram_blocks); }

// Largest dynamic shared memory any orthonormalisation kernel may take.
static constexpr size_t kSmemCap = 220 * 1024;

static size_t gram_stage_bytes(const OrthPlan& p, int elem) {
    return (size_t)elem * (size_t)std::min(gram_rows(p), kGramChunk) * p.L;
}
static size_t gram_chol_smem(const OrthPlan& p, int elem) {
    const size_t np = packed_size(p.L);
    return std::max(gram_stage_bytes(p, elem), 8 * (3 * np + (size_t)p.L));
}
static size_t extract_smem(const OrthPlan& p, int R, int elem) {
    return std::max(xlayout(p.L, R, elem).total, gram_stage_bytes(p, elem));
}
static size_t finish_smem(int R, int elem, int64_t I) { return flayout(R, elem, I).total; }
// The final pass's shared memory with U staged in it, or 0 when that does not fit.
static size_t finish_staged_smem(int R, int elem, int64_t I) {
    const size_t b = flayout(R, elem, I).total + up16((size_t)elem * (size_t)I * (size_t)R);
    return b <= kSmemCap ? b : 0;
}

bool orth_supported(const OrthPlan& p, int R, int elem) {
    return p.L <= 32 * kBsRows && gram_chol_smem(p, elem) <= kSmemCap && extract_smem(p, R, elem) <= kSmemCap &&
           8 * packed_size(p.L) <= kSmemCap && finish_smem(R, elem, p.I) <= kSmemCap;
}

// partials | flag and ticket | W | back-substitution stage (R2, 1/R2_kk, U_M)
size_t orth_scratch_bytes(const OrthPlan& p, int elem_size) {
    const size_t np = packed_size(p.L);
    const size_t LL = (size_t)p.L * p.L;
    return ((8 * np * (size_t)p.gram_blocks + 255) & ~size_t(255)) + 256 + 8 * LL + 512 +
           8 * bs_um_offset(p.L) + (size_t)(elem_size > 8 ? elem_size : 8) * LL;
}

struct OrthScratch {
    void* partial;
    int* flag;
    unsigned* ticket;
    void* W;       // R^-1 of a CholeskyQR pass (packed), then the extraction's W (L x R)
    void* bs;      // the extraction's back-substitution stage
};
static OrthScratch carve(const OrthPlan& p, void* scratch) {
    OrthScratch s;
    char* b = reinterpret_cast<char*>(scratch);
    const size_t np = packed_size(p.L);
    s.partial = b;
    b += (8 * np * (size_t)p.gram_blocks + 255) & ~size_t(255);
    s.flag = reinterpret_cast<int*>(b);
    s.ticket = reinterpret_cast<unsigned*>(b + 64);
    b += 256;
    s.W = b;
    b += 8 * (size_t)p.L * p.L + 512;
    s.bs = b;
    return s;
}

// Whether the serial steps whose rows or columns are independent (the
// triangular inverse, the back-substitution) run on CTAs of their own, which
// shortens a call that runs alone, or inside the one-CTA kernels: a stream
// being captured belongs to a batch graph, where many decompositions run at
// once and the extra launches cost more than the shorter chain saves
// (measured). Both give the same bits.
static bool split_serial(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return cs == cudaStreamCaptureStatusNone;
}

template <typename T>
cudaError_t launch_cholqr(const T* X, T* Q, const OrthPlan& p, double* factor, void* scratch, int* status,
                          cudaStream_t s) {
    using S = typename SmallScalar<T>::type;
    static_assert(sizeof(S) == sizeof(double), "factor slots hold one double per entry");
    OrthScratch sc = carve(p, scratch);
    const int L = p.L;
    const int rows = gram_rows(p);
    const size_t gsm = gram_chol_smem(p, sizeof(T));
    const size_t asm_ = 8 * packed_size(L);
    if (asm_ > kSmemCap || gsm > kSmemCap) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(gram_chol_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
    cudaFuncSetAttribute(apply_rinv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asm_);
    cudaMemsetAsync(sc.flag, 0, 128, s);                 // flag and ticket
    int64_t ablocks = (p.I * L + kT - 1) / kT;
    if (ablocks > 4 * 1024) ablocks = 4 * 1024;
    // R^-1 goes to the W block, which the extraction writes only after this pass
    const bool split = split_serial(s);
    gram_chol_kernel<T><<<p.gram_blocks, kST, gsm, s>>>(X, p.I, L, rows, (S*)sc.partial, sc.ticket, (S*)factor,
                                                        (S*)sc.W, status, split ? (S*)sc.bs : nullptr);
    note_launch();
    if (split) {
        const size_t ism = sizeof(S) * (packed_size(L) + (size_t)L);
        cudaFuncSetAttribute(tri_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism);
        tri_inverse_kernel<T><<<(unsigned)((L + 3) / 4), 128, ism, s>>>((const S*)factor, (const S*)sc.bs, L,
                                                                       (S*)sc.W);
        note_launch();
    }
    apply_rinv_kernel<T><<<(unsigned)ablocks, kT, asm_, s>>>(X, p.I, L, (const S*)sc.W, Q);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_extract(const T* X, T* Q1, const OrthPlan& p, double* factors, int nprev, int R, T* U,
                           void* scratch, int* status, cudaStream_t s) {
    using S = typename SmallScalar<T>::type;
    // X = Q1 R1 (R1 stored after the earlier factors), then C = Q1 (R1 F)
    const size_t slot = (size_t)p.L * p.L;                 // factor slots hold L^2 doubles
    cudaError_t e = launch_cholqr<T>(X, Q1, p, factors + (size_t)nprev * slot, scratch, status, s);
    if (e != cudaSuccess) return e;
    if (!orth_supported(p, R, sizeof(T))) return cudaErrorInvalidValue;
    OrthScratch sc = carve(p, scratch);
    const int L = p.L;
    const int rows = gram_rows(p);
    const size_t xsm = extract_smem(p, R, sizeof(T));
    cudaFuncSetAttribute(extract_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm);
    cudaMemsetAsync(sc.flag, 0, 128, s);
    const bool split = split_serial(s);
    extract_kernel<T><<<p.gram_blocks, kXT, xsm, s>>>(Q1, p.I, L, rows, (S*)sc.partial, sc.ticket,
                                                      (const S*)factors, slot, nprev + 1, R, (S*)sc.W, status,
                                                      split ? (S*)sc.bs : nullptr);
    note_launch();
    if (split) {
        const size_t bsm = sizeof(S) * (packed_size(L) + (size_t)L);
        cudaFuncSetAttribute(backsub_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm);
        backsub_kernel<T><<<(unsigned)((R + 4 * kBsCols - 1) / (4 * kBsCols)), 128, bsm, s>>>((const S*)sc.bs, L,
                                                                                              R, (S*)sc.W);
        note_launch();
    }
    int64_t ublocks = (p.I * R + kT - 1) / kT;
    if (ublocks > 4 * 1024) ublocks = 4 * 1024;
    form_u_kernel<T><<<(unsigned)ublocks, kT, 0, s>>>(Q1, p.I, L, R, (const S*)sc.W, U);
    note_launch();
    // U^T U by a grid of CTAs (the final pass repairs U only when it is not
    // orthonormal to 8 eps, which a one-CTA Gram over I rows would take long to tell)
    int* ok = sc.flag + 8;
    const size_t usm = (size_t)sizeof(T) * (size_t)std::min(rows, kGramChunk) * R;
    cudaFuncSetAttribute(ugram_check_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usm);
    ugram_check_kernel<T><<<p.gram_blocks, kST, usm, s>>>(U, p.I, R, rows, (S*)sc.partial, sc.ticket, ok);
    note_launch();
    const size_t staged = finish_staged_smem(R, sizeof(T), p.I);
    const size_t fsm = staged ? staged : finish_smem(R, sizeof(T), p.I);
    cudaFuncSetAttribute(finish_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
    finish_kernel<T><<<1, kST, fsm, s>>>(U, p.I, R, staged ? 1 : 0, ok);
    note_launch();
    return cudaGetLastError();
}

OrthJob orth_job(const OrthPlan& p, void* scratch) {
    OrthJob j{};
    const OrthScratch sc = carve(p, scratch);
    j.I = p.I;
    j.L = p.L;
    j.rows = gram_rows(p);
    j.nblk = p.gram_blocks;
    j.partial = sc.partial;
    j.flag = sc.flag;
    j.ticket = sc.ticket;
    j.W = sc.W;
    return j;
}

namespace {
int64_t elementwise_blocks(int64_t n) {
    int64_t b = (n + kT - 1) / kT;
    return b > 4 * 1024 ? 4 * 1024 : (b < 1 ? 1 : b);
}
OrthPlan plan_of(const OrthJob& j) {
    OrthPlan p{};
    p.I = j.I;
    p.L = j.L;
    p.gram_blocks = j.nblk;
    return p;
}
// The CholeskyQR pass of every job (the factor at factor + fofs, R^-1 into W, Q = X R^-1).
template <typename T>
cudaError_t cholqr_group(const OrthJob* d, const std::vector<OrthJob>& h, cudaStream_t s) {
    size_t gsm = 0, asm_ = 0;
    int gx = 1;
    int64_t ax = 1;
    for (const OrthJob& j : h) {
        const OrthPlan p = plan_of(j);
        gsm = std::max(gsm, gram_chol_smem(p, sizeof(T)));
        asm_ = std::max(asm_, 8 * packed_size(j.L));
        gx = std::max(gx, j.nblk);
        ax = std::max(ax, elementwise_blocks(j.I * j.L));
    }
    if (gsm > kSmemCap || asm_ > kSmemCap) return cudaErrorInvalidValue;
    const unsigned ny = (unsigned)h.size();
    cudaFuncSetAttribute(gram_chol_group_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    cudaFuncSetAttribute(apply_rinv_group_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    orth_reset_group_kernel<<<ny, 32, 0, s>>>(d);
    note_launch();
    gram_chol_group_kernel<T><<<dim3((unsigned)gx, ny), kST, gsm, s>>>(d);
    note_launch();
    apply_rinv_group_kernel<T><<<dim3((unsigned)ax, ny), kT, asm_, s>>>(d);
    note_launch();
    return cudaGetLastError();
}
}  // namespace

template <typename T>
cudaError_t launch_cholqr_group(const OrthJob* d_jobs, const std::vector<OrthJob>& h_jobs, cudaStream_t s) {
    if (h_jobs.empty()) return cudaSuccess;
    return cholqr_group<T>(d_jobs, h_jobs, s);
}

template <typename T>
cudaError_t launch_extract_group(const OrthJob* d_jobs, const std::vector<OrthJob>& h_jobs, cudaStream_t s) {
    if (h_jobs.empty()) return cudaSuccess;
    for (const OrthJob& j : h_jobs)
        if (!orth_supported(plan_of(j), j.R, sizeof(T)) || j.fofs != (int64_t)j.nprev * j.L * j.L)
            return cudaErrorInvalidValue;
    cudaError_t e = cholqr_group<T>(d_jobs, h_jobs, s);
    if (e != cudaSuccess) return e;
    size_t xsm = 0, usm = 0, fsm = 0;
    int gx = 1;
    int64_t ux = 1;
    for (const OrthJob& j : h_jobs) {
        const OrthPlan p = plan_of(j);
        xsm = std::max(xsm, extract_smem(p, j.R, sizeof(T)));
        usm = std::max(usm, (size_t)sizeof(T) * (size_t)std::min(j.rows, kGramChunk) * j.R);
        const size_t staged = finish_staged_smem(j.R, sizeof(T), j.I);
        if ((staged != 0) != (j.staged != 0)) return cudaErrorInvalidValue;
        fsm = std::max(fsm, staged ? staged : finish_smem(j.R, sizeof(T), j.I));
        gx = std::max(gx, j.nblk);
        ux = std::max(ux, elementwise_blocks(j.I * j.R));
    }
    const unsigned ny = (unsigned)h_jobs.size();
    cudaFuncSetAttribute(extract_group_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    cudaFuncSetAttribute(ugram_check_group_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    cudaFuncSetAttribute(finish_group_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    orth_reset_group_kernel<<<ny, 32, 0, s>>>(d_jobs);
    note_launch();
    extract_group_kernel<T><<<dim3((unsigned)gx, ny), kXT, xsm, s>>>(d_jobs);
    note_launch();
    form_u_group_kernel<T><<<dim3((unsigned)ux, ny), kT, 0, s>>>(d_jobs);
    note_launch();
    ugram_check_group_kernel<T><<<dim3((unsigned)gx, ny), kST, usm, s>>>(d_jobs);
    note_launch();
    finish_group_kernel<T><<<dim3(1, ny), kST, fsm, s>>>(d_jobs);
    note_launch();
    return cudaGetLastError();
}

bool orth_group_staged(const OrthJob& j, int elem_size) { return finish_staged_smem(j.R, elem_size, j.I) != 0; }

template cudaError_t launch_cholqr_group<float>(const OrthJob*, const std::vector<OrthJob>&, cudaStream_t);
template cudaError_t launch_cholqr_group<double>(const OrthJob*, const std::vector<OrthJob>&, cudaStream_t);
template cudaError_t launch_extract_group<float>(const OrthJob*, const std::vector<OrthJob>&, cudaStream_t);
template cudaError_t launch_extract_group<double>(const OrthJob*, const std::vector<OrthJob>&, cudaStream_t);
template cudaError_t launch_cholqr<float>(const float*, float*, const OrthPlan&, double*, void*, int*, cudaStream_t);
template cudaError_t launch_cholqr<double>(const double*, double*, const OrthPlan&, double*, void*, int*,
                                           cudaStream_t);
template cudaError_t launch_extract<float>(const float*, float*, const OrthPlan&, double*, int, int, float*, void*,
                                           int*, cudaStream_t);
template cudaError_t launch_extract<double>(const double*, double*, const OrthPlan&, double*, int, int, double*,
                                            void*, int*, cudaStream_t);

}  // namespace tk
