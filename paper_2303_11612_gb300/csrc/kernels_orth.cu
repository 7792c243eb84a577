// Orthonormalisation of the sketch and extraction of the leading left singular
// vectors (remark after Algorithm 5: Q_n = U(:, 1:mu_n) from the SVD of C_n).
//
// The sketch is held as C = X F, where X (I x L) is the last power-step output
// and F = F_k ... F_1 collects the triangular factors of the earlier steps
// (each earlier step orthonormalised its output X_j = Q_j F_j and multiplied Q_j,
// which leaves C unchanged). Extraction:
//   1. One CholeskyQR pass X = Q1 R1: Gram X^T X from exact FP32 products summed
//      in paired FP32 (about 2^-44), reduced across CTAs in a fixed order; FP64
//      Cholesky (shifted once on a numerically singular pivot, Fukaya et al.
//      2020); Q1 = X R1^-1 by FP64 substitution.
//   2. A second Gram/Cholesky Q1^T Q1 = R2^T R2, so Q = Q1 R2^-1 is orthonormal
//      and C = Q M with M = R2 R1 F (L x L).
//   3. One-sided (Hestenes) Jacobi on the columns of M with paired-precision
//      dot products: M V = U_M S, U_M = the rotated columns, normalised;
//      columns at rounding level are re-orthogonalised (FP64 Gram-Schmidt), so
//      they keep the sketch's own weak directions. U = Q U_M = Q1 W with
//      W = R2^-1 U_M (FP64 back-substitution) -- Q is never formed.
//   4. U = Q1 W in paired precision; each column's largest-magnitude entry
//      made positive. A column that is exactly dependent is completed by
//      Gram-Schmidt of unit vectors against the others.
// Intermediate power steps need only Q1 and R1: step 1 alone.
#include <float.h>

#include <algorithm>

#include "internal.h"

namespace tk {
namespace {

constexpr int kT = kThreads;
constexpr int kXT = 256;                 // threads of the extraction kernel (any SM can host it)
constexpr int kDegenerate = 8;           // flag bit: some factor column needs completion

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

// Gram partial of this CTA's rows (packed upper triangle) -> partial[blockIdx.x].
template <typename T>
__device__ void gram_partial(const T* __restrict__ X, int64_t I, int L, int rows, double* __restrict__ partial,
                             unsigned char* smem) {
    T* xs = reinterpret_cast<T*>(smem);   // [rows][L]
    const int64_t r0 = (int64_t)blockIdx.x * rows;
    const int nr = (int)max((int64_t)0, min((int64_t)rows, I - r0));
    for (int e = threadIdx.x; e < nr * L; e += blockDim.x) {
        const int r = e % nr, c = e / nr;
        xs[r * L + c] = X[(int64_t)c * I + r0 + r];
    }
    __syncthreads();
    double* out = partial + (int64_t)blockIdx.x * (L * (L + 1) / 2);
    for (int a = 0; a < L; ++a) {
        for (int b = a + threadIdx.x; b < L; b += blockDim.x) {
            GramAcc<T> acc;
            for (int r = 0; r < nr; ++r) acc.add(xs[r * L + a], xs[r * L + b]);
            out[packed_index(a, b, L)] = acc.value();
        }
    }
}

// True in exactly one CTA: the last to finish its partial (an atomic ticket, no waiting).
__device__ bool last_cta(unsigned* ticket) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// 1/sqrt(d) for finite d > 0: an FP32 estimate on the mantissa refined by two
// Newton steps in FP64 (GB300's FP64 square root and division are slow chains).
__device__ __forceinline__ double rsqrt_fp64(double d) {
    int e;
    double m = frexp(d, &e);                      // d = m 2^e, m in [0.5, 1)
    if (e & 1) { m *= 2.0; e -= 1; }              // m in [0.5, 2), e even
    double y = (double)rsqrtf((float)m);
    y = y * fma(-0.5 * m * y, y, 1.5);
    y = y * fma(-0.5 * m * y, y, 1.5);
    return ldexp(y, -e / 2);
}

// Sum the partials in block order into G (L x L, shared) and factor G = R^T R
// (R upper, row-major, left in W with zeros below the diagonal; 1/R_kk in dinv).
// A pivot below 1e-15 of its diagonal entry restarts once with G + s I,
// s = 11 (I L + L (L + 1)) 2^-53 tr(G). Returns false if that also fails (R = I).
__device__ bool reduce_cholesky(const double* __restrict__ partial, int nparts, int L, int64_t I, double* G,
                                double* W, double* dinv, unsigned* ticket, int* status) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int np = L * (L + 1) / 2;
    __shared__ int bad;
    __shared__ double inv_piv;
    __shared__ double tr;
    for (int p = tid; p < np; p += nt) {
        double acc = 0.0;
#pragma unroll 8
        for (int b = 0; b < nparts; ++b) acc += __ldcg(partial + (int64_t)b * np + p);
        int a = 0, rem = p;
        while (rem >= L - a) { rem -= L - a; ++a; }
        const int bb = a + rem;
        G[a * L + bb] = acc;
        G[bb * L + a] = acc;
    }
    if (tid == 0) *ticket = 0;                           // ready for the next use
    __syncthreads();
    double shift = 0.0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        for (int p = tid; p < L * L; p += nt) W[p] = G[p] + ((p / L == p % L) ? shift : 0.0);
        if (tid == 0) bad = 0;
        __syncthreads();
        for (int k = 0; k < L; ++k) {
            if (tid == 0) {
                const double d = W[k * L + k];
                const double ref = G[k * L + k] + shift;
                if (!(d > 1e-15 * ref) || !isfinite(d)) {
                    bad = 1;
                } else {
                    const double y = rsqrt_fp64(d);
                    W[k * L + k] = d * y;
                    dinv[k] = y;
                    inv_piv = y;
                }
            }
            __syncthreads();
            if (bad) break;
            for (int j = k + 1 + tid; j < L; j += nt) W[k * L + j] *= inv_piv;
            __syncthreads();
            const int m = L - k - 1;
            for (int p = tid; p < m * m; p += nt) {
                const int i = k + 1 + p / m, j = k + 1 + p % m;
                if (j >= i) W[i * L + j] -= W[k * L + i] * W[k * L + j];
            }
            __syncthreads();
        }
        if (!bad) break;
        if (attempt == 0) {
            if (tid == 0) {
                double t = 0.0;
                for (int k = 0; k < L; ++k) t += G[k * L + k];
                tr = t > 0.0 ? t : 1.0;
            }
            __syncthreads();
            shift = 11.0 * ((double)I * L + (double)L * (L + 1)) * 1.1102230246251565e-16 * tr;
            __syncthreads();
        }
    }
    const int failed = bad;
    __syncthreads();
    for (int p = tid; p < L * L; p += nt) {
        const int a = p / L, b = p % L;
        if (failed) W[p] = (a == b) ? 1.0 : 0.0;
        else if (b < a) W[p] = 0.0;
    }
    if (failed)
        for (int k = tid; k < L; k += nt) dinv[k] = 1.0;
    if (failed && tid == 0) set_status(status, kStatNumerical);
    __syncthreads();
    return !failed;
}

// Inverse of the upper-triangular R (row-major, L x L, 1/R_kk in dinv) into Ri.
// Row i of R^-1 solves y R = e_i by forward substitution (one thread per row),
// so the computed inverse has a small residual R^-1 R - I: X R^-1 R stays close
// to X, which is what Q R = X needs.
__device__ void upper_inverse(const double* R, const double* dinv, int L, double* Ri) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        double* y = Ri + i * L;
        for (int j = 0; j < i; ++j) y[j] = 0.0;
        for (int j = i; j < L; ++j) {
            double acc = (i == j) ? 1.0 : 0.0;
            for (int k = i; k < j; ++k) acc = fma(-y[k], R[k * L + j], acc);
            y[j] = acc * dinv[j];
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- one CholeskyQR pass
// R (row-major, L x L) and R^-1 (same layout) of X^T X = R^T R.
template <typename T>
__global__ void __launch_bounds__(kT) gram_chol_kernel(const T* __restrict__ X, int64_t I, int L, int rows,
                                                       double* __restrict__ partial, unsigned* ticket,
                                                       double* __restrict__ R, double* __restrict__ Rinv,
                                                       int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    gram_partial<T>(X, I, L, rows, partial, smem_raw);
    if (!last_cta(ticket)) return;
    double* G = reinterpret_cast<double*>(smem_raw);
    double* W = G + L * L;
    double* dinv = W + L * L;
    reduce_cholesky(partial, gridDim.x, L, I, G, W, dinv, ticket, status);
    upper_inverse(W, dinv, L, G);
    for (int p = threadIdx.x; p < L * L; p += blockDim.x) {
        R[p] = W[p];
        Rinv[p] = G[p];
    }
}

// Q = X R^-1, one thread per entry of Q, in paired precision from X (exact) and
// R^-1 split into high and low FP32 parts (FP64 for T = double).
template <typename T> struct ApplyAcc;
template <> struct ApplyAcc<float> {
    Pair s{0.f, 0.f};
    __device__ void add(float x, double w) {
        const float hi = (float)w;
        pair_add_prod(s, x, hi);
        pair_add_prod(s, x, (float)(w - (double)hi));
    }
    __device__ float value() const { return (float)pair_value(s); }
};
template <> struct ApplyAcc<double> {
    double s = 0.0;
    __device__ void add(double x, double w) { s = fma(x, w, s); }
    __device__ double value() const { return s; }
};

template <typename T>
__global__ void __launch_bounds__(kT) apply_rinv_kernel(const T* __restrict__ X, int64_t I, int L,
                                                        const double* __restrict__ Rinv, T* __restrict__ Q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* Ri = reinterpret_cast<double*>(smem_raw);    // [L][L]
    for (int p = threadIdx.x; p < L * L; p += kT) Ri[p] = Rinv[p];
    __syncthreads();
    const int64_t n = I * L;
    for (int64_t e = (int64_t)blockIdx.x * kT + threadIdx.x; e < n; e += (int64_t)gridDim.x * kT) {
        const int l = (int)(e / I);
        const int64_t i = e - (int64_t)l * I;
        ApplyAcc<T> acc;
        for (int m = 0; m <= l; ++m) acc.add(X[(int64_t)m * I + i], Ri[m * L + l]);
        Q[e] = (T)acc.value();
    }
}

// ---------------------------------------------------------------- fused extraction
template <typename T> struct DotAcc;
template <> struct DotAcc<float> {
    Pair s{0.f, 0.f};
    __device__ void add(float a, float b) { pair_add_prod(s, a, b); }
    __device__ void reduce() { s = warp_sum_pair(s); }
    __device__ double value() const { return pair_value(s); }
};
template <> struct DotAcc<double> {
    double s = 0.0;
    __device__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ void reduce() { s = warp_sum(s); }
    __device__ double value() const { return s; }
};

constexpr int kMaxPerThread = 12;        // L * L / kXT for L <= 110

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
template <int GS>
__device__ __forceinline__ double group_sum(double s) {
#pragma unroll
    for (int o = GS / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// One cyclic sweep of one-sided Jacobi on the columns of Mc (column-major,
// column c at Mc + c * L); pairs handled by groups of GS lanes. Returns the
// number of rotations.
template <typename T, int GS>
__device__ int jacobi_sweep(T* Mc, int L, int Lp, T tol, T tiny, int* nrot) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kGroupsPerWarp = 32 / GS;
    const int groups = ((int)blockDim.x >> 5) * kGroupsPerWarp, gl = lane % GS;
    const int m = Lp - 1;
    if (tid == 0) *nrot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < m; ++rnd) {
        // the loop bound is uniform across a warp, so all 32 lanes reach every
        // shuffle below; groups without a pair take part with zeros
        for (int base = warp * kGroupsPerWarp; base < Lp / 2; base += groups) {
            const int pi = base + lane / GS;
            int p = L, q = L;
            if (pi < Lp / 2) {
                if (pi == 0) { p = rnd; q = m; }
                else { p = (rnd + pi) % m; q = (rnd - pi + m) % m; }
            }
            const bool live = p < L && q < L;
            T* cp = Mc + (live ? p : 0) * L;
            T* cq = Mc + (live ? q : 0) * L;
            T a, b, g;
            if (sizeof(T) == 4) {
                Pair al{0.f, 0.f}, be{0.f, 0.f}, ga{0.f, 0.f};
                for (int r = gl; r < L && live; r += GS) {
                    const float x = (float)cp[r], y = (float)cq[r];
                    pair_add_prod(al, x, x);
                    pair_add_prod(be, y, y);
                    pair_add_prod(ga, x, y);
                }
                al = group_sum_pair<GS>(al);
                be = group_sum_pair<GS>(be);
                ga = group_sum_pair<GS>(ga);
                a = (T)(al.hi + al.lo); b = (T)(be.hi + be.lo); g = (T)(ga.hi + ga.lo);
            } else {
                double al = 0, be = 0, ga = 0;
                for (int r = gl; r < L && live; r += GS) {
                    const double x = (double)cp[r], y = (double)cq[r];
                    al = fma(x, x, al); be = fma(y, y, be); ga = fma(x, y, ga);
                }
                a = group_sum<GS>(al); b = group_sum<GS>(be); g = group_sum<GS>(ga);
            }
            // all in the working precision (the dot products are accurate to its
            // last bit): FP64 square roots and divisions are long chains on this part
            if (live && fabs(g) > tiny && g * g > tol * tol * a * b) {
                const T zeta = (b - a) / (T(2) * g);
                const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
                const T c = T(1) / sqrt(T(1) + t * t), s = c * t;
                for (int r = gl; r < L; r += GS) {
                    const T x = cp[r], y = cq[r];
                    cp[r] = c * x - s * y;
                    cq[r] = s * x + c * y;
                }
                if (gl == 0) atomicAdd(nrot, 1);
            }
        }
        __syncthreads();
    }
    const int n = *nrot;
    __syncthreads();
    return n;
}

// Grid of Gram CTAs over Q1 (kXT threads each). The last CTA: Cholesky
// Q1^T Q1 = R2^T R2, M = R2 P with P = prev[nprev-1] ... prev[0], Jacobi on M,
// U_M (rounding-level columns re-orthogonalised) and W = R2^-1 U_M for the R
// leading columns (FP64, L x R, column-major). An exactly dependent column gets
// W = 0 and raises the kDegenerate flag.
template <typename T>
__global__ void __launch_bounds__(kXT) extract_kernel(const T* __restrict__ X, int64_t I, int L, int rows,
                                                      double* __restrict__ partial, unsigned* ticket,
                                                      const double* __restrict__ prev, int nprev, int R,
                                                      double* __restrict__ Wout, int* flag, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    gram_partial<T>(X, I, L, rows, partial, smem_raw);
    if (!last_cta(ticket)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kXT / 32;
    const int Lp = L + (L & 1);
    double* G = reinterpret_cast<double*>(smem_raw);     // [L][L]; after the Cholesky: P, then M
    double* Rf = G + L * L;                                // [L][L] Cholesky factor (upper, row-major)
    double* UM = Rf + L * L;                               // column-major [R][L], FP64
    double* wb = UM + (size_t)R * L;                       // [nwarps][L] back-substitution rows
    double* dinv = wb + nwarps * L;                        // [L] 1 / R2_kk
    double* inrm = dinv + L;                               // [Lp] 1 / column norms of the rotated M
    T* Mc = reinterpret_cast<T*>(inrm + Lp);               // column-major [Lp][L]
    T* sig = Mc + Lp * L;                                  // [Lp]
    int* perm = reinterpret_cast<int*>(sig + Lp);          // [Lp]
    __shared__ unsigned long long mx_bits;
    __shared__ int nrot;
    __shared__ double fro2;
    __shared__ double red[kXT / 32];
    __shared__ double bcast;
    __shared__ int deg;

    reduce_cholesky(partial, gridDim.x, L, I, G, Rf, dinv, ticket, status);

    // P = prev[nprev-1] ... prev[0] (upper triangular, FP64) into G, then M = R2 P
    // in place: row a of F P needs only rows >= a of P, so rows are replaced top-down
    for (int p = tid; p < L * L; p += kXT) G[p] = prev[p];
    __syncthreads();
    for (int f = 1; f <= nprev; ++f) {
        const double* F = f < nprev ? prev + (int64_t)f * L * L : Rf;
        for (int a = 0; a < L; ++a) {
            double acc[kMaxPerThread];
            int cnt = 0;
            for (int c = tid; c < L; c += kXT, ++cnt) {
                double s = 0.0;
                for (int b = a; b <= c; ++b) s = fma(F[a * L + b], G[b * L + c], s);
                acc[cnt] = s;
            }
            __syncthreads();
            cnt = 0;
            for (int c = tid; c < L; c += kXT, ++cnt) G[a * L + c] = c >= a ? acc[cnt] : 0.0;
            __syncthreads();
        }
    }
    // M scaled by a power of two (largest entry in [1, 2)) and stored in T
    if (tid == 0) { mx_bits = 0ull; fro2 = 0.0; }
    __syncthreads();
    {
        double mxl = 0.0;
        for (int p = tid; p < L * L; p += kXT) mxl = fmax(mxl, fabs(G[p]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mxl = fmax(mxl, __shfl_xor_sync(0xffffffffu, mxl, o));
        if (lane == 0) atomicMax(&mx_bits, (unsigned long long)__double_as_longlong(mxl));
    }
    __syncthreads();
    const double mxv = __longlong_as_double((long long)mx_bits);
    int ex = 0;
    if (mxv > 0.0) frexp(mxv, &ex);
    {
        double s2 = 0.0;
        for (int p = tid; p < Lp * L; p += kXT) {
            const int c = p / L, a = p % L;
            const T v = c < L ? (T)ldexp(G[a * L + c], 1 - ex) : T(0);
            Mc[p] = v;
            s2 = fma((double)v, (double)v, s2);
        }
        s2 = warp_sum(s2);
        if (lane == 0) atomicAdd(&fro2, s2);
    }
    __syncthreads();
    // rotate while a pair's cosine exceeds 4 eps and its coupling is above the
    // rounding level of the whole matrix; the stored columns carry rounding of
    // their own, so the sweep count is capped
    const T eps = sizeof(T) == 4 ? (T)FLT_EPSILON : (T)DBL_EPSILON;
    const T tol = T(4) * eps;
    const T tiny = eps * eps * (T)fro2;
    for (int sweep = 0; sweep < 20; ++sweep) {
        int n;
        if (L <= 32) n = jacobi_sweep<T, 8>(Mc, L, Lp, tol, tiny, &nrot);
        else if (L <= 64) n = jacobi_sweep<T, 16>(Mc, L, Lp, tol, tiny, &nrot);
        else n = jacobi_sweep<T, 32>(Mc, L, Lp, tol, tiny, &nrot);
        if (n == 0) break;
    }
    // singular values (column norms), decreasing order, lower index first on ties
    for (int c = warp; c < L; c += nwarps) {
        DotAcc<T> s;
        for (int r = lane; r < L; r += 32) s.add(Mc[c * L + r], Mc[c * L + r]);
        s.reduce();
        if (lane == 0) {
            const double ss = s.value();
            const double y = ss > 0.0 ? rsqrt_fp64(ss) : 0.0;
            inrm[c] = y;
            sig[c] = (T)(ss * y);
        }
    }
    __syncthreads();
    for (int c = tid; c < L; c += kXT) {
        int rank = 0;
        for (int d = 0; d < L; ++d) rank += (sig[d] > sig[c]) || (sig[d] == sig[c] && d < c);
        perm[rank] = c;
    }
    __syncthreads();
    const double smax = (double)sig[perm[0]];
    const double weak = 64.0 * (double)eps * smax;
    // U_M: rotated columns in decreasing order, normalised (FP64)
    for (int p = tid; p < L * R; p += kXT) {
        const int r = p / L, a = p % L;
        const int c = perm[r];
        UM[p] = (double)Mc[c * L + a] * inrm[c];
    }
    if (tid == 0) deg = 0;
    __syncthreads();
    // rounding-level columns: two Gram-Schmidt passes against every earlier column
    for (int r = 0; r < R; ++r) {
        if (!((double)sig[perm[r]] <= weak)) continue;
        double* u = UM + (size_t)r * L;
        for (int pass = 0; pass < 2; ++pass) {
            for (int j = 0; j < r; ++j) {
                const double* v = UM + (size_t)j * L;
                double s = 0.0;
                for (int a = tid; a < L; a += kXT) s = fma(v[a], u[a], s);
                s = warp_sum(s);
                if (lane == 0) red[warp] = s;
                __syncthreads();
                if (tid == 0) {
                    double t = 0.0;
                    for (int w = 0; w < nwarps; ++w) t += red[w];
                    bcast = t;
                }
                __syncthreads();
                const double d = bcast;
                for (int a = tid; a < L; a += kXT) u[a] -= d * v[a];
                __syncthreads();
            }
        }
        double s = 0.0;
        for (int a = tid; a < L; a += kXT) s = fma(u[a], u[a], s);
        s = warp_sum(s);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < nwarps; ++w) t += red[w];
            bcast = t;
        }
        __syncthreads();
        const double n2 = bcast;
        const bool ok = n2 > 1e-6;                     // else the sketch has no direction left here
        const double f = ok ? rsqrt_fp64(n2) : 0.0;
        for (int a = tid; a < L; a += kXT) u[a] *= f;
        if (tid == 0 && !ok) deg = 1;
        __syncthreads();
    }
    // W(:, r) = R2^-1 U_M(:, r): back-substitution in FP64, one warp per column
    double* w = wb + warp * L;
    for (int r = warp; r < R; r += nwarps) {
        const double* u = UM + (size_t)r * L;
        for (int l = L - 1; l >= 0; --l) {
            double s = 0.0;
            for (int k = l + 1 + lane; k < L; k += 32) s = fma(Rf[l * L + k], w[k], s);
            s = warp_sum(s);
            if (lane == 0) w[l] = (u[l] - s) * dinv[l];
            __syncwarp();
        }
        for (int l = lane; l < L; l += 32) Wout[(int64_t)r * L + l] = w[l];
        __syncwarp();
    }
    if (tid == 0) *flag = deg ? kDegenerate : 0;
}

// U(:, r) = X W(:, r) in paired precision, then the sign rule. One CTA per column.
template <typename T>
__global__ void __launch_bounds__(kT) form_u_kernel(const T* __restrict__ X, int64_t I, int L,
                                                    const double* __restrict__ W, T* __restrict__ U) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* whi = reinterpret_cast<T*>(smem_raw);  // [L]
    T* wlo = whi + L;                         // [L]
    T* col = wlo + L;                         // [I]
    __shared__ T best_v[kT / 32];
    __shared__ int64_t best_i[kT / 32];
    __shared__ T sgn;
    const int r = blockIdx.x;
    for (int c = threadIdx.x; c < L; c += kT) {
        const double w = W[(int64_t)r * L + c];
        whi[c] = (T)w;
        wlo[c] = (T)(w - (double)whi[c]);
    }
    __syncthreads();
    T bv = T(-1);
    int64_t bi = 0;
    for (int64_t i = threadIdx.x; i < I; i += kT) {
        DotAcc<T> s;
        for (int c = 0; c < L; ++c) {
            const T x = X[(int64_t)c * I + i];
            s.add(x, whi[c]);
            s.add(x, wlo[c]);
        }
        const T v = (T)s.value();
        col[i] = v;
        const T a = fabs(v);
        if (a > bv) { bv = a; bi = i; }
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

// Columns whose singular value is at rounding level: the first unit vector e_k
// (k increasing) that keeps a long residual after two Gram-Schmidt passes
// against every valid column, normalised and sign-fixed. The squared residuals
// of e_0 .. e_{I-1} average (I - d) / I for d valid columns, so accepting one
// above half that average always succeeds. Runs only when flagged.
template <typename T>
__global__ void __launch_bounds__(kT) complete_kernel(int64_t I, int L, int R, const double* __restrict__ W,
                                                      T* __restrict__ U, const int* flag) {
    if (!(*flag & kDegenerate)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* v = reinterpret_cast<double*>(smem_raw);   // [I]
    int* valid = reinterpret_cast<int*>(v + I);        // [R]
    __shared__ double red[kT / 32];
    __shared__ double bcast;
    __shared__ double bv;
    __shared__ int64_t bi;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int r = tid; r < R; r += kT) {
        int nz = 0;
        for (int c = 0; c < L; ++c) nz |= W[(int64_t)r * L + c] != 0.0;
        valid[r] = nz;
    }
    __syncthreads();
    int nvalid = 0;
    for (int r = 0; r < R; ++r) nvalid += valid[r];
    int64_t k = 0;
    for (int r = 0; r < R; ++r) {
        if (valid[r]) continue;
        const double accept = 0.5 * (double)(I - nvalid) / (double)I;
        for (; k < I; ++k) {
            for (int64_t i = tid; i < I; i += kT) v[i] = (i == k) ? 1.0 : 0.0;
            __syncthreads();
            for (int pass = 0; pass < 2; ++pass) {
                for (int j = 0; j < R; ++j) {
                    if (!valid[j]) continue;
                    double s = 0.0;
                    for (int64_t i = tid; i < I; i += kT) s = fma((double)U[(int64_t)j * I + i], v[i], s);
                    s = warp_sum(s);
                    if (lane == 0) red[warp] = s;
                    __syncthreads();
                    if (tid == 0) {
                        double t = 0.0;
                        for (int w = 0; w < kT / 32; ++w) t += red[w];
                        bcast = t;
                    }
                    __syncthreads();
                    const double d = bcast;
                    for (int64_t i = tid; i < I; i += kT) v[i] -= d * (double)U[(int64_t)j * I + i];
                    __syncthreads();
                }
            }
            double s = 0.0;
            for (int64_t i = tid; i < I; i += kT) s = fma(v[i], v[i], s);
            s = warp_sum(s);
            if (lane == 0) red[warp] = s;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < kT / 32; ++w) t += red[w];
                bcast = sqrt(t);
                bv = -1.0;
                bi = 0;
                for (int64_t i = 0; i < I; ++i)
                    if (fabs(v[i]) > bv) { bv = fabs(v[i]); bi = i; }
            }
            __syncthreads();
            const double nrm = bcast;
            if (nrm * nrm > accept) {
                const double f = (v[bi] < 0 ? -1.0 : 1.0) / nrm;
                for (int64_t i = tid; i < I; i += kT) U[(int64_t)r * I + i] = (T)(v[i] * f);
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
}

}  // namespace

OrthPlan orth_plan(int64_t I, int L, int num_sms) {
    OrthPlan p{};
    p.I = I;
    p.L = L;
    // enough CTAs to spread the paired-precision Gram work, few enough that the
    // last CTA's reduction of the packed partials stays small (<= 512 KB)
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
    (void)elem_size;
    const size_t np = (size_t)p.L * (p.L + 1) / 2;
    const size_t LL = (size_t)p.L * p.L;
    return ((sizeof(double) * np * (size_t)p.gram_blocks + 255) & ~size_t(255)) + 256 + sizeof(double) * LL + 512;
}

struct OrthScratch {
    double* partial;
    int* flag;
    unsigned* ticket;
    double* W;
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
    s.W = reinterpret_cast<double*>(b);
    return s;
}

template <typename T>
cudaError_t launch_cholqr(const T* X, T* Q, const OrthPlan& p, double* factor, void* scratch, int* status,
                          cudaStream_t s) {
    OrthScratch sc = carve(p, scratch);
    const int L = p.L;
    const size_t LL = (size_t)L * L;
    const int rows = gram_rows(p);
    const size_t gsm = std::max(sizeof(T) * (size_t)rows * L, sizeof(double) * (2 * LL + L));
    const size_t asm_ = sizeof(double) * LL;
    if (asm_ > 220 * 1024 || gsm > 220 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(gram_chol_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
    cudaFuncSetAttribute(apply_rinv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asm_);
    cudaMemsetAsync(sc.flag, 0, 128, s);                 // flag and ticket
    int64_t ablocks = (p.I * L + kT - 1) / kT;
    if (ablocks > 4 * 1024) ablocks = 4 * 1024;
    // R^-1 goes to the W block, which the extraction writes only after this pass
    gram_chol_kernel<T><<<p.gram_blocks, kT, gsm, s>>>(X, p.I, L, rows, sc.partial, sc.ticket, factor, sc.W, status);
    note_launch();
    apply_rinv_kernel<T><<<(unsigned)ablocks, kT, asm_, s>>>(X, p.I, L, sc.W, Q);
    note_launch();
    return cudaGetLastError();
}

static size_t extract_smem_bytes(int L, int R, int elem, int rows) {
    const int Lp = L + (L & 1);
    const size_t last = sizeof(double) * (2 * (size_t)L * L + (size_t)R * L + (size_t)(kXT / 32) * L + L + Lp) +
                        (size_t)elem * ((size_t)Lp * L + Lp) + sizeof(int) * Lp + 64;
    return std::max(last, (size_t)elem * (size_t)rows * L);
}

template <typename T>
cudaError_t launch_extract(const T* X, T* Q1, const OrthPlan& p, double* factors, int nprev, int R, T* U,
                           void* scratch, int* status, cudaStream_t s) {
    // X = Q1 R1 (R1 stored after the earlier factors), then C = Q1 (R1 F)
    cudaError_t e = launch_cholqr<T>(X, Q1, p, factors + (size_t)nprev * p.L * p.L, scratch, status, s);
    if (e != cudaSuccess) return e;
    OrthScratch sc = carve(p, scratch);
    const int L = p.L;
    const int rows = gram_rows(p);
    const size_t xsm = extract_smem_bytes(L, R, sizeof(T), rows);
    if (xsm > 220 * 1024 || L > kXT * kMaxPerThread) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(extract_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm);
    cudaMemsetAsync(sc.flag, 0, 128, s);
    extract_kernel<T><<<p.gram_blocks, kXT, xsm, s>>>(Q1, p.I, L, rows, sc.partial, sc.ticket, factors, nprev + 1, R,
                                                      sc.W, sc.flag, status);
    note_launch();
    const size_t fsm = sizeof(T) * (2 * (size_t)L + (size_t)p.I) + 64;
    if (fsm > 220 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(form_u_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
    form_u_kernel<T><<<R, kT, fsm, s>>>(Q1, p.I, L, sc.W, U);
    note_launch();
    const size_t csm = sizeof(double) * (size_t)p.I + sizeof(int) * (size_t)R + 64;
    if (csm > 220 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(complete_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);
    complete_kernel<T><<<1, kT, csm, s>>>(p.I, L, R, sc.W, U, sc.flag);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t launch_cholqr<float>(const float*, float*, const OrthPlan&, double*, void*, int*, cudaStream_t);
template cudaError_t launch_cholqr<double>(const double*, double*, const OrthPlan&, double*, void*, int*,
                                           cudaStream_t);
template cudaError_t launch_extract<float>(const float*, float*, const OrthPlan&, double*, int, int, float*, void*,
                                           int*, cudaStream_t);
template cudaError_t launch_extract<double>(const double*, double*, const OrthPlan&, double*, int, int, double*,
                                            void*, int*, cudaStream_t);

}  // namespace tk
