// The two halves of a power step on the gathered AMM sample C' (I_n x T,
// column-major, materialised by the gather), for the half-step evaluation of
// C_n = (C' C'^T)^q Omega_n:
//   Y = C'^T X      (T x L)      gemm_tn_kernel
//   X = C' Q_Y      (I_n x L)    gemm_nn_kernel, split over T with partial sums
//                                reduced in a fixed order
// with Y orthonormalised (CholeskyQR, triangular factor kept) between them. A
// stored half step carries the sketch's directions with weights sigma_i, a full
// step sigma_i^2: in FP32 a full step loses every direction with
// sigma_i / sigma_1 below about 2^-12, a half step only those below about 2^-24.
// C' is small (T fibers of I_n values), so these are plain FMA register-tiled
// products in the data's own precision.
#include "internal.h"

namespace tk {
namespace {

constexpr int kHT = 256;
constexpr int kHTile = 64;       // columns t (tn) or rows i (nn) per CTA
constexpr int kHK = 16;          // contraction chunk staged in shared memory (FP64 at L = 128: 25 KB)
constexpr int kHLG = 16;         // thread groups along L: a thread holds L / 16 (rounded up) columns

// Y(t, l) = sum_i M(i, t) X(i, l); thread (tg, lg): t = tg * 4 + 0..3, l = lg + 16 k
template <typename T, int LPT>
__global__ void __launch_bounds__(kHT) gemm_tn_kernel(const T* __restrict__ M, int64_t I, int64_t Tn,
                                                      const T* __restrict__ X, int L, T* __restrict__ Y) {
    __shared__ T Ms[kHK][kHTile + 1];
    __shared__ T Xs[kHK][kHLG * LPT + 1];
    const int tid = threadIdx.x, tg = tid / kHLG, lg = tid % kHLG;
    const int64_t t0 = (int64_t)blockIdx.x * kHTile;
    T acc[4][LPT];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < LPT; ++k) acc[a][k] = T(0);
    for (int64_t i0 = 0; i0 < I; i0 += kHK) {
        __syncthreads();
        for (int e = tid; e < kHK * kHTile; e += kHT) {
            const int ii = e % kHK, tt = e / kHK;
            const int64_t i = i0 + ii, t = t0 + tt;
            Ms[ii][tt] = (i < I && t < Tn) ? M[i + I * t] : T(0);
        }
        for (int e = tid; e < kHK * kHLG * LPT; e += kHT) {
            const int ii = e % kHK, l = e / kHK;
            const int64_t i = i0 + ii;
            Xs[ii][l] = (i < I && l < L) ? X[i + I * l] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int ii = 0; ii < kHK; ++ii) {
            T m[4], x[LPT];
#pragma unroll
            for (int a = 0; a < 4; ++a) m[a] = Ms[ii][tg * 4 + a];
#pragma unroll
            for (int k = 0; k < LPT; ++k) x[k] = Xs[ii][lg + kHLG * k];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int k = 0; k < LPT; ++k) acc[a][k] = fma(m[a], x[k], acc[a][k]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t t = t0 + tg * 4 + a;
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
            const int l = lg + kHLG * k;
            if (t < Tn && l < L) Y[t + Tn * l] = acc[a][k];
        }
    }
}

// partial[s](i, l) = sum_{t in split s} M(i, t) Q(t, l); thread (ig, lg): i = ig * 4 + 0..3
template <typename T, int LPT>
__global__ void __launch_bounds__(kHT) gemm_nn_kernel(const T* __restrict__ M, int64_t I, int64_t Tn,
                                                      const T* __restrict__ Q, int L, T* __restrict__ partial,
                                                      int64_t per_split) {
    __shared__ T Ms[kHK][kHTile + 1];
    __shared__ T Qs[kHK][kHLG * LPT + 1];
    const int tid = threadIdx.x, ig = tid / kHLG, lg = tid % kHLG;
    const int64_t i0 = (int64_t)blockIdx.x * kHTile;
    const int64_t ta = (int64_t)blockIdx.y * per_split;
    const int64_t tb = ta + per_split < Tn ? ta + per_split : Tn;
    T acc[4][LPT];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < LPT; ++k) acc[a][k] = T(0);
    for (int64_t c0 = ta; c0 < tb; c0 += kHK) {
        __syncthreads();
        for (int e = tid; e < kHK * kHTile; e += kHT) {
            const int ii = e % kHTile, tt = e / kHTile;
            const int64_t i = i0 + ii, t = c0 + tt;
            Ms[tt][ii] = (i < I && t < tb) ? M[i + I * t] : T(0);
        }
        for (int e = tid; e < kHK * kHLG * LPT; e += kHT) {
            const int tt = e % kHK, l = e / kHK;
            const int64_t t = c0 + tt;
            Qs[tt][l] = (t < tb && l < L) ? Q[t + Tn * l] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int tt = 0; tt < kHK; ++tt) {
            T m[4], q[LPT];
#pragma unroll
            for (int a = 0; a < 4; ++a) m[a] = Ms[tt][ig * 4 + a];
#pragma unroll
            for (int k = 0; k < LPT; ++k) q[k] = Qs[tt][lg + kHLG * k];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int k = 0; k < LPT; ++k) acc[a][k] = fma(m[a], q[k], acc[a][k]);
        }
    }
    T* out = partial + (int64_t)blockIdx.y * (I * L);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + ig * 4 + a;
#pragma unroll
        for (int k = 0; k < LPT; ++k) {
            const int l = lg + kHLG * k;
            if (i < I && l < L) out[i + I * l] = acc[a][k];
        }
    }
}

// Sign rule on the columns of U (I x R, column-major): each column's
// largest-magnitude entry positive, the lowest row on ties; one warp per column.
template <typename T>
__global__ void __launch_bounds__(kHT) sign_fix_kernel(T* __restrict__ U, int64_t I, int R) {
    const int lane = threadIdx.x & 31;
    const int r = (int)((blockIdx.x * (int64_t)kHT + threadIdx.x) >> 5);
    if (r >= R) return;
    T* u = U + (int64_t)r * I;
    T bv = T(-1);
    int64_t bi = 0;
    for (int64_t i = lane; i < I; i += 32) {
        const T a = fabs(u[i]);
        if (a > bv) { bv = a; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (u[bi] < T(0))
        for (int64_t i = lane; i < I; i += 32) u[i] = -u[i];
}

int half_splits(int64_t I, int64_t Tn, int num_sms) {
    const int64_t rows = (I + kHTile - 1) / kHTile;
    int64_t s = (num_sms + rows - 1) / rows;
    const int64_t most = (Tn + 255) / 256;              // at least 256 fibers per split
    if (s > most) s = most;
    return (int)(s < 1 ? 1 : s);
}

template <typename T, int LPT>
cudaError_t tn_t(const T* M, int64_t I, int64_t Tn, const T* X, int L, T* Y, cudaStream_t s) {
    gemm_tn_kernel<T, LPT><<<(unsigned)((Tn + kHTile - 1) / kHTile), kHT, 0, s>>>(M, I, Tn, X, L, Y);
    note_launch();
    return cudaGetLastError();
}

template <typename T, int LPT>
cudaError_t nn_t(const T* M, int64_t I, int64_t Tn, const T* Q, int L, T* part, int splits, cudaStream_t s) {
    const int64_t per = (Tn + splits - 1) / splits;
    const dim3 grid((unsigned)((I + kHTile - 1) / kHTile), (unsigned)splits);
    gemm_nn_kernel<T, LPT><<<grid, kHT, 0, s>>>(M, I, Tn, Q, L, part, per);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

bool half_supported(int L) { return L >= 1 && L <= kHLG * 8; }

size_t half_partials_bytes(int64_t I, int L, int64_t Tn, int num_sms, int elem_size) {
    return (size_t)half_splits(I, Tn, num_sms) * (size_t)I * (size_t)L * (size_t)elem_size;
}

template <typename T>
cudaError_t launch_gemm_tn(const T* M, int64_t I, int64_t Tn, const T* X, int L, T* Y, cudaStream_t s) {
    switch ((L + kHLG - 1) / kHLG) {           // columns per thread, no more than needed
        case 1: return tn_t<T, 1>(M, I, Tn, X, L, Y, s);
        case 2: return tn_t<T, 2>(M, I, Tn, X, L, Y, s);
        case 3: return tn_t<T, 3>(M, I, Tn, X, L, Y, s);
        case 4: return tn_t<T, 4>(M, I, Tn, X, L, Y, s);
        case 5: return tn_t<T, 5>(M, I, Tn, X, L, Y, s);
        case 6: return tn_t<T, 6>(M, I, Tn, X, L, Y, s);
        case 7: return tn_t<T, 7>(M, I, Tn, X, L, Y, s);
        case 8: return tn_t<T, 8>(M, I, Tn, X, L, Y, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_gemm_nn(const T* M, int64_t I, int64_t Tn, const T* Q, int L, T* X, void* partials, int num_sms,
                           cudaStream_t s) {
    const int lpt = (L + kHLG - 1) / kHLG;
    const int splits = half_splits(I, Tn, num_sms);
    T* part = reinterpret_cast<T*>(partials);
    cudaError_t e;
    switch (lpt) {
        case 1: e = nn_t<T, 1>(M, I, Tn, Q, L, part, splits, s); break;
        case 2: e = nn_t<T, 2>(M, I, Tn, Q, L, part, splits, s); break;
        case 3: e = nn_t<T, 3>(M, I, Tn, Q, L, part, splits, s); break;
        case 4: e = nn_t<T, 4>(M, I, Tn, Q, L, part, splits, s); break;
        case 5: e = nn_t<T, 5>(M, I, Tn, Q, L, part, splits, s); break;
        case 6: e = nn_t<T, 6>(M, I, Tn, Q, L, part, splits, s); break;
        case 7: e = nn_t<T, 7>(M, I, Tn, Q, L, part, splits, s); break;
        case 8: e = nn_t<T, 8>(M, I, Tn, Q, L, part, splits, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return launch_reduce_partials<T>(part, splits, I * (int64_t)L, X, s);
}

template <typename T>
cudaError_t launch_sign_fix(T* U, int64_t I, int R, cudaStream_t s) {
    sign_fix_kernel<T><<<(unsigned)((R * 32 + kHT - 1) / kHT), kHT, 0, s>>>(U, I, R);
    note_launch();
    return cudaGetLastError();
}
template cudaError_t launch_sign_fix<float>(float*, int64_t, int, cudaStream_t);
template cudaError_t launch_sign_fix<double>(double*, int64_t, int, cudaStream_t);

template cudaError_t launch_gemm_tn<float>(const float*, int64_t, int64_t, const float*, int, float*, cudaStream_t);
template cudaError_t launch_gemm_tn<double>(const double*, int64_t, int64_t, const double*, int, double*,
                                            cudaStream_t);
template cudaError_t launch_gemm_nn<float>(const float*, int64_t, int64_t, const float*, int, float*, void*, int,
                                           cudaStream_t);
template cudaError_t launch_gemm_nn<double>(const double*, int64_t, int64_t, const double*, int, double*, void*, int,
                                            cudaStream_t);

}  // namespace tk
