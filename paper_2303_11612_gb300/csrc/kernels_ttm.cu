// Mode-n products (Section 2) for the truncation B <- B x_n U_n^T of
// Algorithms 2/5, the core chain G = A x_1 U_1^T ... x_N U_N^T of Algorithms
// 1/4, and the reconstruction used by the relative error (Eq. 8); plus
// deterministic sums of squares.
//
// Each CTA takes JB = 64 NF consecutive mode-n fibers and OB = 4 OPT output
// indices; the fiber tile streams through shared memory in chunks of KC input
// indices while the JB x OB block of results stays in registers, so the input
// is read once per output block (one block whenever K_out <= 64).
#include "internal.h"

namespace tk {
namespace {

constexpr int kT = kThreads;
constexpr int KC = 32, KP = KC + 4;   // rows padded to 36 elements: 16-byte aligned, conflict-free

// four consecutive T values from 16-byte aligned shared memory
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
    const double2 x = *reinterpret_cast<const double2*>(p), y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

// Thread (lane64 = tid % 64, og = tid / 64) owns fibers lane64 + 64 f (f < NF)
// and outputs og * OPT .. og * OPT + OPT - 1. Both shared tiles keep the input
// index contiguous, so stores are unit-stride and the inner loop reads four
// input indices per 128-bit load; the M rows are the same across a warp
// (broadcast) and each serves 4 NF multiply-adds. The next chunk's global
// loads are issued into registers before the current chunk is multiplied.
template <typename T, int OPT, int NF>
__global__ void __launch_bounds__(kT) ttm_kernel(const T* __restrict__ A, ModeView v, const T* __restrict__ Mp,
                                                 int64_t K_out, int64_t ld_i, int64_t ld_k, T* __restrict__ out) {
    constexpr int JB = 64 * NF, OB = 4 * OPT;
    constexpr int TPT = JB * KC / kT;                    // tile elements loaded per thread and chunk
    constexpr int MPT = (OB * KC + kT - 1) / kT;         // M elements loaded per thread and chunk
    constexpr size_t kTileBytes = sizeof(T) * (JB * KP + OB * KP);
    constexpr size_t kOutBytes = sizeof(T) * JB * (OB + 1);
    __shared__ __align__(16) unsigned char smem[kTileBytes > kOutBytes ? kTileBytes : kOutBytes];
    auto Ts = reinterpret_cast<T(*)[KP]>(smem);                       // [JB][KP]
    auto Ms = reinterpret_cast<T(*)[KP]>(smem + sizeof(T) * JB * KP);  // [OB][KP]
    auto Os = reinterpret_cast<T(*)[OB + 1]>(smem);                   // [JB][OB + 1], after the products
    __shared__ int64_t bases[JB];
    const int tid = threadIdx.x;
    const int64_t J = v.fibers();
    const int64_t j0 = (int64_t)blockIdx.x * JB;
    const int64_t o0 = (int64_t)blockIdx.y * OB;
    const int I = (int)v.i;
    const bool contig = v.lf == 1;
    for (int r = tid; r < JB; r += kT) {
        const int64_t j = j0 + r;
        bases[r] = j < J ? v.base(j) : -1;
    }
    __syncthreads();
    T tr[TPT], mr[MPT];
    // element u of this thread's share of a chunk: (fiber, k) for the tile, (output, k) for M
    auto load_chunk = [&](int i0) {
#pragma unroll
        for (int u = 0; u < TPT; ++u) {
            const int e = tid + u * kT;
            int r, c;
            if (contig) { r = e / KC; c = e % KC; }      // a warp reads KC consecutive elements of a fiber
            else { r = e % JB; c = e / JB; }             // a warp reads one element of 32 neighbouring fibers
            const int64_t b = bases[r];
            const int i = i0 + c;
            tr[u] = (b >= 0 && i < I) ? __ldg(A + b + (int64_t)i * v.lf) : T(0);
        }
#pragma unroll
        for (int u = 0; u < MPT; ++u) {
            const int e = tid + u * kT;
            int kk, oo;
            if (ld_i == 1) { kk = e % KC; oo = e / KC; } // unit stride along the input index
            else { oo = e % OB; kk = e / OB; }
            const int i = i0 + kk;
            const int64_t o = o0 + oo;
            mr[u] = (e < OB * KC && i < I && o < K_out) ? __ldg(Mp + (int64_t)i * ld_i + o * ld_k) : T(0);
        }
    };
    auto store_chunk = [&]() {
#pragma unroll
        for (int u = 0; u < TPT; ++u) {
            const int e = tid + u * kT;
            int r, c;
            if (contig) { r = e / KC; c = e % KC; }
            else { r = e % JB; c = e / JB; }
            Ts[r][c] = tr[u];
        }
#pragma unroll
        for (int u = 0; u < MPT; ++u) {
            const int e = tid + u * kT;
            int kk, oo;
            if (ld_i == 1) { kk = e % KC; oo = e / KC; }
            else { oo = e % OB; kk = e / OB; }
            if (e < OB * KC) Ms[oo][kk] = mr[u];
        }
    };
    const int jl = tid % 64, og = tid / 64;
    T acc[NF][OPT];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int u = 0; u < OPT; ++u) acc[f][u] = T(0);
    load_chunk(0);
    for (int i0 = 0; i0 < I; i0 += KC) {
        store_chunk();
        __syncthreads();
        if (i0 + KC < I) load_chunk(i0 + KC);            // in flight during the products below
#pragma unroll 2
        for (int kk = 0; kk < KC; kk += 4) {
            T t4[NF][4];
#pragma unroll
            for (int f = 0; f < NF; ++f) ld4(&Ts[jl + 64 * f][kk], t4[f]);
#pragma unroll
            for (int u = 0; u < OPT; ++u) {
                T m4[4];
                ld4(&Ms[og * OPT + u][kk], m4);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    acc[f][u] = fma(t4[f][0], m4[0], acc[f][u]);
                    acc[f][u] = fma(t4[f][1], m4[1], acc[f][u]);
                    acc[f][u] = fma(t4[f][2], m4[2], acc[f][u]);
                    acc[f][u] = fma(t4[f][3], m4[3], acc[f][u]);
                }
            }
        }
        __syncthreads();
    }
    // (the loop ends with a barrier, so every thread is done reading Ts and Ms)
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int u = 0; u < OPT; ++u) Os[jl + 64 * f][og * OPT + u] = acc[f][u];
    __syncthreads();
    if (contig) {
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
    // outputs per thread: the smallest instantiated OPT with 4 OPT >= K_out (at most 16)
    static const int kOpts[] = {1, 2, 3, 4, 5, 6, 8, 12, 16};
    int OPT = 16;
    for (int o : kOpts)
        if (4 * o >= K_out) { OPT = o; break; }
    constexpr int NF = sizeof(T) == 4 ? 2 : 1;
    const int OB = 4 * OPT, JBl = 64 * NF;
    dim3 grid((unsigned)((J + JBl - 1) / JBl), (unsigned)((K_out + OB - 1) / OB));
    const double ein = (double)v.i * (double)J, eout = (double)K_out * (double)J;
    ProfScope prof(kKTtm, (ein + eout) * sizeof(T), 2.0 * ein * (double)K_out, s);
    switch (OPT) {
        case 1: ttm_kernel<T, 1, NF><<<grid, kT, 0, s>>>(A, v, Mp, K_out, ld_i, ld_k, out); break;
        case 2: ttm_kernel<T, 2, NF><<<grid, kT, 0, s>>>(A, v, Mp, K_out, ld_i, ld_k, out); break;
        case 3: ttm_kernel<T, 3, NF><<<grid, kT, 0, s>>>(A, v, Mp, K_out, ld_i, ld_k, out); break;
        case 4: ttm_kernel<T, 4, NF><<<grid, kT, 0, s>>>(A, v, Mp, K_out, ld_i, ld_k, out); break;
        case 5: ttm_kernel<T, 5, NF><<<grid, kT, 0, s>>>(A, v, Mp, K_out, ld_i, ld_k, out); break;
        case 6: ttm_kernel<T, 6, NF><<<grid, kT, 0, s>>>(A, v, Mp, K_out, ld_i, ld_k, out); break;
        case 8: ttm_kernel<T, 8, NF><<<grid, kT, 0, s>>>(A, v, Mp, K_out, ld_i, ld_k, out); break;
        case 12: ttm_kernel<T, 12, NF><<<grid, kT, 0, s>>>(A, v, Mp, K_out, ld_i, ld_k, out); break;
        default: ttm_kernel<T, 16, NF><<<grid, kT, 0, s>>>(A, v, Mp, K_out, ld_i, ld_k, out); break;
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
