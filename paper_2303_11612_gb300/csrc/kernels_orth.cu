// Orthonormalisation of the sketch and extraction of the leading left singular
// vectors (remark after Algorithm 5: Q_n = U(:, 1:mu_n) from the SVD of C_n).
//
// The sketch is held as C = X F, where X (I x L) is the last power-step output
// and F = F_k ... F_1 collects the triangular factors of the earlier steps
// (each earlier step orthonormalised its output X_j = Q_j F_j and multiplied Q_j,
// which leaves C unchanged). Extraction:
//   1. G = X^T X from exact FP32 products summed in paired FP32 (about 2^-44),
//      reduced across CTAs in a fixed order; FP64 Cholesky G = R^T R (shifted
//      once on a numerically singular pivot, Fukaya et al. 2020). Then
//      C = Q M with Q = X R^-1 orthonormal and M = R F (L x L).
//   2. One-sided (Hestenes) Jacobi on the columns of M with paired-precision
//      dot products: M V = U_M S. The leading left singular vectors of C are
//      Q U_M = C V S^-1, so U = X W with W = F V S^-1 (L x R) -- no triangular
//      solve and no explicit Q.
//   3. U = X W in paired precision; each column's largest-magnitude entry made
//      positive. Columns whose singular value is at rounding level are
//      completed by Gram-Schmidt against the others.
// Intermediate power steps need only Q_j and F_j: one CholeskyQR pass.
#include <float.h>

#include <algorithm>

#include "internal.h"

namespace tk {
namespace {

constexpr int kT = kThreads;
constexpr int kXT = 1024;                // threads of the extraction kernel
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

// Sum the partials in block order into G (L x L, shared) and factor G = R^T R
// (R upper, row-major, left in W with zeros below the diagonal). A pivot below
// 1e-15 of its diagonal entry restarts once with G + s I,
// s = 11 (I L + L (L + 1)) 2^-53 tr(G). Returns false if that also fails.
__device__ bool reduce_cholesky(const double* __restrict__ partial, int nparts, int L, int64_t I, double* G,
                                double* W, unsigned* ticket, int* status) {
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
                    const double pv = sqrt(d);
                    W[k * L + k] = pv;
                    inv_piv = 1.0 / pv;
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
    if (failed && tid == 0) set_status(status, kStatNumerical);
    __syncthreads();
    return !failed;
}

// ---------------------------------------------------------------- one CholeskyQR pass
template <typename T>
__global__ void __launch_bounds__(kT) gram_chol_kernel(const T* __restrict__ X, int64_t I, int L, int rows,
                                                       double* __restrict__ partial, unsigned* ticket,
                                                       double* __restrict__ R, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    gram_partial<T>(X, I, L, rows, partial, smem_raw);
    if (!last_cta(ticket)) return;
    double* G = reinterpret_cast<double*>(smem_raw);
    double* W = G + L * L;
    reduce_cholesky(partial, gridDim.x, L, I, G, W, ticket, status);
    for (int p = threadIdx.x; p < L * L; p += blockDim.x) R[p] = W[p];
}

// Q = X R^-1, one warp per row: forward substitution in FP64.
template <typename T>
__global__ void __launch_bounds__(kT) apply_rinv_kernel(const T* __restrict__ X, int64_t I, int L,
                                                        const double* __restrict__ R, T* __restrict__ Q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* Rs = reinterpret_cast<double*>(smem_raw);    // [L][L]
    double* qs = Rs + L * L;                               // [warps][L]
    for (int p = threadIdx.x; p < L * L; p += kT) Rs[p] = R[p];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* q = qs + warp * L;
    for (int64_t i = (int64_t)blockIdx.x * (kT / 32) + warp; i < I; i += (int64_t)gridDim.x * (kT / 32)) {
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

// Grid of Gram CTAs (kXT threads each). The last CTA: Cholesky of X^T X,
// M = R P with P = prev[nprev-1] ... prev[0], Jacobi on M, and
// W = P V S^-1 for the R leading columns (FP64, L x R, column-major).
// Columns with a singular value at rounding level get W = 0 and raise the
// kDegenerate flag.
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
    double* G = reinterpret_cast<double*>(smem_raw);     // [L][L]; after the Cholesky: P
    double* Rf = G + L * L;                                // [L][L] Cholesky factor (upper, row-major)
    T* Mc = reinterpret_cast<T*>(Rf + L * L);              // column-major [Lp][L]
    T* V = Mc + Lp * L;                                    // column-major [Lp][L]
    T* sig = V + Lp * L;                                   // [Lp]
    int* perm = reinterpret_cast<int*>(sig + Lp);          // [Lp]
    __shared__ unsigned long long mx_bits;
    __shared__ int nrot;
    __shared__ double fro2;

    reduce_cholesky(partial, gridDim.x, L, I, G, Rf, ticket, status);

    // P = prev[nprev-1] ... prev[0] (upper triangular, FP64) into G
    if (nprev > 0) {
        for (int p = tid; p < L * L; p += kXT) G[p] = prev[p];
        __syncthreads();
        for (int f = 1; f < nprev; ++f) {
            const double* F = prev + (int64_t)f * L * L;
            double acc[kMaxPerThread];
            int cnt = 0;
            for (int p = tid; p < L * L; p += kXT, ++cnt) {
                const int a = p / L, c = p % L;
                double s = 0.0;
                for (int b = a; b <= c; ++b) s = fma(F[a * L + b], G[b * L + c], s);
                acc[cnt] = s;
            }
            __syncthreads();
            cnt = 0;
            for (int p = tid; p < L * L; p += kXT, ++cnt) G[p] = acc[cnt];
            __syncthreads();
        }
    }
    // M = R P (or R), stored in T after scaling by a power of two
    if (tid == 0) mx_bits = 0ull;
    __syncthreads();
    {
        double mxl = 0.0;
        for (int p = tid; p < L * L; p += kXT) {
            const int a = p % L, c = p / L;               // row a, column c
            double s = 0.0;
            if (nprev > 0) {
                for (int b = a; b <= c; ++b) s = fma(Rf[a * L + b], G[b * L + c], s);
            } else if (c >= a) {
                s = Rf[a * L + c];
            }
            mxl = fmax(mxl, fabs(s));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mxl = fmax(mxl, __shfl_xor_sync(0xffffffffu, mxl, o));
        if (lane == 0) atomicMax(&mx_bits, (unsigned long long)__double_as_longlong(mxl));
    }
    __syncthreads();
    const double mxv = __longlong_as_double((long long)mx_bits);
    const double sc = mxv > 0.0 ? exp2(-floor(log2(mxv))) : 1.0;      // exact power of two
    for (int p = tid; p < Lp * L; p += kXT) {
        const int c = p / L, a = p % L;
        double s = 0.0;
        if (c < L) {
            if (nprev > 0) {
                for (int b = a; b <= c; ++b) s = fma(Rf[a * L + b], G[b * L + c], s);
            } else if (c >= a) {
                s = Rf[a * L + c];
            }
        }
        Mc[p] = (T)(s * sc);
        V[p] = (T)((c == a) ? 1.0 : 0.0);
    }
    if (tid == 0) fro2 = 0.0;
    __syncthreads();
    {
        double s2 = 0.0;
        for (int p = tid; p < L * L; p += kXT) s2 = fma((double)Mc[p], (double)Mc[p], s2);
        s2 = warp_sum(s2);
        if (lane == 0) atomicAdd(&fro2, s2);
    }
    __syncthreads();
    const double eps = sizeof(T) == 4 ? (double)FLT_EPSILON : DBL_EPSILON;
    const double tol = 2.0 * eps;
    const double tiny = eps * eps * fro2;
    const int m = Lp - 1;
    for (int sweep = 0; sweep < 30; ++sweep) {
        if (tid == 0) nrot = 0;
        __syncthreads();
        for (int rnd = 0; rnd < m; ++rnd) {
            for (int pi = warp; pi < Lp / 2; pi += nwarps) {
                int p, q;
                if (pi == 0) { p = rnd; q = m; }
                else { p = (rnd + pi) % m; q = (rnd - pi + m) % m; }
                if (p >= L || q >= L) continue;
                T* cp = Mc + p * L;
                T* cq = Mc + q * L;
                DotAcc<T> al, be, ga;
                for (int r = lane; r < L; r += 32) {
                    const T x = cp[r], y = cq[r];
                    al.add(x, x);
                    be.add(y, y);
                    ga.add(x, y);
                }
                al.reduce();
                be.reduce();
                ga.reduce();
                const double a = al.value(), b = be.value(), g = ga.value();
                if (fabs(g) > tiny && fabs(g) > tol * sqrt(a * b)) {
                    const double zeta = (b - a) / (2.0 * g);
                    const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double cs = 1.0 / sqrt(1.0 + t * t);
                    const T c = (T)cs, s = (T)(cs * t);
                    T* vp = V + p * L;
                    T* vq = V + q * L;
                    for (int r = lane; r < L; r += 32) {
                        const T x = cp[r], y = cq[r];
                        cp[r] = c * x - s * y;
                        cq[r] = s * x + c * y;
                        const T u = vp[r], w = vq[r];
                        vp[r] = c * u - s * w;
                        vq[r] = s * u + c * w;
                    }
                    if (lane == 0) atomicAdd(&nrot, 1);
                }
            }
            __syncthreads();
        }
        if (nrot == 0) break;
        __syncthreads();
    }
    // singular values (column norms), decreasing order, lower index first on ties
    for (int c = warp; c < L; c += nwarps) {
        DotAcc<T> s;
        for (int r = lane; r < L; r += 32) s.add(Mc[c * L + r], Mc[c * L + r]);
        s.reduce();
        if (lane == 0) sig[c] = (T)sqrt(s.value());
    }
    __syncthreads();
    for (int c = tid; c < L; c += kXT) {
        int rank = 0;
        for (int d = 0; d < L; ++d) rank += (sig[d] > sig[c]) || (sig[d] == sig[c] && d < c);
        perm[rank] = c;
    }
    __syncthreads();
    const double smax = (double)sig[perm[0]];
    const double floor_rel = 64.0 * eps;
    // W(:, r) = P V(:, c) / (sigma_c / sc), c = perm[r]
    for (int p = tid; p < L * R; p += kXT) {
        const int r = p / L, a = p % L;
        const int c = perm[r];
        const double sg = (double)sig[c];
        double w = 0.0;
        if (sg > floor_rel * smax && sg > 0.0) {
            double s = 0.0;
            if (nprev > 0) {
                for (int b = a; b < L; ++b) s = fma(G[a * L + b], (double)V[c * L + b], s);
            } else {
                s = (double)V[c * L + a];
            }
            w = s * sc / sg;
        }
        Wout[(int64_t)r * L + a] = w;
    }
    if (tid == 0) {
        int deg = 0;
        for (int r = 0; r < R; ++r) {
            const double sg = (double)sig[perm[r]];
            deg |= !(sg > floor_rel * smax && sg > 0.0);
        }
        *flag = deg ? kDegenerate : 0;
    }
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
    const size_t gsm = std::max(sizeof(T) * (size_t)rows * L, sizeof(double) * 2 * LL);
    const size_t asm_ = sizeof(double) * (LL + (size_t)(kT / 32) * L);
    if (asm_ > 220 * 1024 || gsm > 220 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(gram_chol_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
    cudaFuncSetAttribute(apply_rinv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asm_);
    cudaMemsetAsync(sc.flag, 0, 128, s);                 // flag and ticket
    int64_t ablocks = (p.I + kT / 32 - 1) / (kT / 32);
    if (ablocks > 1024) ablocks = 1024;
    gram_chol_kernel<T><<<p.gram_blocks, kT, gsm, s>>>(X, p.I, L, rows, sc.partial, sc.ticket, factor, status);
    note_launch();
    apply_rinv_kernel<T><<<(unsigned)ablocks, kT, asm_, s>>>(X, p.I, L, factor, Q);
    note_launch();
    return cudaGetLastError();
}

static size_t extract_smem_bytes(int L, int elem, int rows) {
    const int Lp = L + (L & 1);
    const size_t last = sizeof(double) * 2 * (size_t)L * L + (size_t)elem * (2 * (size_t)Lp * L + Lp) +
                        sizeof(int) * Lp + 64;
    return std::max(last, (size_t)elem * (size_t)rows * L);
}

template <typename T>
cudaError_t launch_extract(const T* X, const OrthPlan& p, const double* prev, int nprev, int R, T* U, void* scratch,
                           int* status, cudaStream_t s) {
    OrthScratch sc = carve(p, scratch);
    const int L = p.L;
    const int rows = gram_rows(p);
    if ((int64_t)L * L > (int64_t)kXT * kMaxPerThread) return cudaErrorInvalidValue;
    const size_t xsm = extract_smem_bytes(L, sizeof(T), rows);
    if (xsm > 220 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(extract_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xsm);
    cudaMemsetAsync(sc.flag, 0, 128, s);
    extract_kernel<T><<<p.gram_blocks, kXT, xsm, s>>>(X, p.I, L, rows, sc.partial, sc.ticket, prev, nprev, R, sc.W,
                                                      sc.flag, status);
    note_launch();
    const size_t fsm = sizeof(T) * (2 * (size_t)L + (size_t)p.I) + 64;
    if (fsm > 220 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(form_u_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
    form_u_kernel<T><<<R, kT, fsm, s>>>(X, p.I, L, sc.W, U);
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
template cudaError_t launch_extract<float>(const float*, const OrthPlan&, const double*, int, int, float*, void*,
                                           int*, cudaStream_t);
template cudaError_t launch_extract<double>(const double*, const OrthPlan&, const double*, int, int, double*, void*,
                                            int*, cudaStream_t);

}  // namespace tk
