// Mode-n products (Section 2) for the truncation B <- B x_n U_n^T of
// Algorithms 2/5, the core chain G = A x_1 U_1^T ... x_N U_N^T of Algorithms
// 1/4, and the reconstruction used by the relative error (Eq. 8); plus
// deterministic sums of squares.
//
// Each CTA takes JB consecutive mode-n fibers and OB output indices; the fiber
// tile streams through shared memory in chunks of KC input indices while the
// JB x OB block of results stays in registers, so the input is read once per
// output block (one block whenever K_out <= OB).
#include "internal.h"

namespace tk {
namespace {

constexpr int kT = kThreads;
constexpr int JB = 64, KC = 32;

// OB = output block (a multiple of 8 covering K_out, or 64 with several blocks);
// thread (jj = tid % JB, og = tid / JB) owns fiber jj and outputs og*OPT .. +OPT.
template <typename T, int OB>
__global__ void __launch_bounds__(kT) ttm_kernel(const T* __restrict__ A, ModeView v, const T* __restrict__ Mp,
                                                 int64_t K_out, int64_t ld_i, int64_t ld_k, T* __restrict__ out) {
    constexpr int OPT = OB / (kT / JB);
    // the tile buffers (Ts, Ms) are dead once the products are done, so the output
    // staging block Os reuses their storage
    constexpr size_t kTileBytes = sizeof(T) * (JB * (KC + 1) + KC * OB);
    constexpr size_t kOutBytes = sizeof(T) * JB * (OB + 1);
    __shared__ __align__(16) unsigned char smem[kTileBytes > kOutBytes ? kTileBytes : kOutBytes];
    auto Ts = reinterpret_cast<T(*)[KC + 1]>(smem);
    auto Ms = reinterpret_cast<T(*)[OB]>(smem + sizeof(T) * JB * (KC + 1));
    auto Os = reinterpret_cast<T(*)[OB + 1]>(smem);
    __shared__ int64_t bases[JB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t J = v.fibers();
    const int64_t j0 = (int64_t)blockIdx.x * JB;
    const int64_t o0 = (int64_t)blockIdx.y * OB;
    const int I = (int)v.i;
    if (tid < JB) {
        const int64_t j = j0 + tid;
        bases[tid] = j < J ? v.base(j) : -1;
    }
    __syncthreads();
    const int jj = tid % JB, og = tid / JB;
    T acc[OPT];
#pragma unroll
    for (int u = 0; u < OPT; ++u) acc[u] = T(0);
    for (int i0 = 0; i0 < I; i0 += KC) {
        if (v.lf == 1) {
            // contiguous fibers: a warp reads KC consecutive elements of one fiber
            for (int r = warp; r < JB; r += kT / 32) {
                const int64_t b = bases[r];
                const int i = i0 + lane;
                Ts[r][lane] = (b >= 0 && i < I) ? __ldg(A + b + i) : T(0);
            }
        } else {
            // strided fibers: a warp reads one element of 32 neighbouring fibers
            for (int e = tid; e < JB * KC; e += kT) {
                const int r = e % JB, c = e / JB;
                const int64_t b = bases[r];
                const int i = i0 + c;
                Ts[r][c] = (b >= 0 && i < I) ? __ldg(A + b + (int64_t)i * v.lf) : T(0);
            }
        }
        // M chunk: walk the unit-stride index across threads
        if (ld_i == 1) {
            for (int e = tid; e < KC * OB; e += kT) {
                const int kk = e % KC, oo = e / KC;
                const int i = i0 + kk;
                const int64_t o = o0 + oo;
                Ms[kk][oo] = (i < I && o < K_out) ? __ldg(Mp + i + o * ld_k) : T(0);
            }
        } else {
            for (int e = tid; e < KC * OB; e += kT) {
                const int kk = e / OB, oo = e % OB;
                const int i = i0 + kk;
                const int64_t o = o0 + oo;
                Ms[kk][oo] = (i < I && o < K_out) ? __ldg(Mp + (int64_t)i * ld_i + o * ld_k) : T(0);
            }
        }
        __syncthreads();
        const int kc = min(KC, I - i0);
        for (int kk = 0; kk < kc; ++kk) {
            const T t = Ts[jj][kk];
            const T* mr = &Ms[kk][og * OPT];
#pragma unroll
            for (int u = 0; u < OPT; ++u) acc[u] = fma(t, mr[u], acc[u]);
        }
        __syncthreads();
    }
    // (the loop ends with a barrier, so every thread is done reading Ts and Ms)
#pragma unroll
    for (int u = 0; u < OPT; ++u) Os[jj][og * OPT + u] = acc[u];
    __syncthreads();
    if (v.lf == 1) {
        // out[o + j K_out]: consecutive threads -> consecutive o
        for (int e = tid; e < JB * OB; e += kT) {
            const int r = e / OB, oo = e % OB;
            const int64_t j = j0 + r, o = o0 + oo;
            if (j < J && o < K_out) out[j * K_out + o] = Os[r][oo];
        }
    } else {
        // out[l + o Lf + t Lf K_out]: consecutive threads -> consecutive fibers
        for (int e = tid; e < JB * OB; e += kT) {
            const int r = e % JB, oo = e / JB;
            const int64_t j = j0 + r, o = o0 + oo;
            if (j < J && o < K_out) {
                const int64_t t = j / v.lf, l = j - t * v.lf;
                out[l + o * v.lf + t * v.lf * K_out] = Os[r][oo];
            }
        }
    }
}

// sum of squares of (a - b) (b may be null), one partial per block, FP64 out
template <typename T> struct SqAcc;
template <> struct SqAcc<float> {
    Pair s{0.f, 0.f};
    __device__ void add(float x) { pair_add_prod(s, x, x); }
    __device__ void merge(const SqAcc& o) { pair_add(s, o.s); }
    __device__ void warp_reduce() { s = warp_sum_pair(s); }
    __device__ double value() const { return pair_value(s); }
};
template <> struct SqAcc<double> {
    double s = 0.0;
    __device__ void add(double x) { s = fma(x, x, s); }
    __device__ void warp_reduce() { s = warp_sum(s); }
    __device__ double value() const { return s; }
};

constexpr int kSumBlocks = 1024;

template <typename T>
__global__ void __launch_bounds__(kT) sumsq_kernel(const T* __restrict__ a, const T* __restrict__ b, int64_t n,
                                                   double* __restrict__ partial) {
    __shared__ double sh[kT / 32];
    SqAcc<T> acc;
    for (int64_t k = blockIdx.x * (int64_t)kT + threadIdx.x; k < n; k += (int64_t)gridDim.x * kT) {
        const T x = b ? (T)(a[k] - b[k]) : a[k];
        acc.add(x);
    }
    acc.warp_reduce();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc.value();
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kT / 32; ++w) s += sh[w];
        partial[blockIdx.x] = s;
    }
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += partial[k];
        *out = s;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_ttm(const T* A, const ModeView& v, const T* Mp, int64_t K_out, int64_t ld_i, int64_t ld_k, T* out,
                       cudaStream_t s) {
    const int64_t J = v.fibers();
    if (J == 0 || K_out == 0) return cudaSuccess;
    const int OB = K_out <= 8 ? 8 : K_out <= 16 ? 16 : K_out <= 32 ? 32 : 64;
    dim3 grid((unsigned)((J + JB - 1) / JB), (unsigned)((K_out + OB - 1) / OB));
    const double ein = (double)v.i * (double)J, eout = (double)K_out * (double)J;
    ProfScope prof(kKTtm, (ein + eout) * sizeof(T), 2.0 * ein * (double)K_out, s);
    switch (OB) {
        case 8: ttm_kernel<T, 8><<<grid, kT, 0, s>>>(A, v, Mp, K_out, ld_i, ld_k, out); break;
        case 16: ttm_kernel<T, 16><<<grid, kT, 0, s>>>(A, v, Mp, K_out, ld_i, ld_k, out); break;
        case 32: ttm_kernel<T, 32><<<grid, kT, 0, s>>>(A, v, Mp, K_out, ld_i, ld_k, out); break;
        default: ttm_kernel<T, 64><<<grid, kT, 0, s>>>(A, v, Mp, K_out, ld_i, ld_k, out); break;
    }
    note_launch();
    return cudaGetLastError();
}

size_t sumsq_scratch_bytes() { return sizeof(double) * kSumBlocks + 256; }

template <typename T>
cudaError_t launch_sumsq(const T* a, const T* b, int64_t n, double* out, void* scratch, cudaStream_t s) {
    double* partial = reinterpret_cast<double*>(scratch);
    int64_t blocks = (n + kT - 1) / kT;
    if (blocks > kSumBlocks) blocks = kSumBlocks;
    if (blocks < 1) blocks = 1;
    sumsq_kernel<T><<<(unsigned)blocks, kT, 0, s>>>(a, b, n, partial);
    note_launch();
    sum_partials_kernel<<<1, 32, 0, s>>>(partial, (int)blocks, out);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t launch_ttm<float>(const float*, const ModeView&, const float*, int64_t, int64_t, int64_t, float*,
                                       cudaStream_t);
template cudaError_t launch_ttm<double>(const double*, const ModeView&, const double*, int64_t, int64_t, int64_t,
                                        double*, cudaStream_t);
template cudaError_t launch_sumsq<float>(const float*, const float*, int64_t, double*, void*, cudaStream_t);
template cudaError_t launch_sumsq<double>(const double*, const double*, int64_t, double*, void*, cudaStream_t);

}  // namespace tk
