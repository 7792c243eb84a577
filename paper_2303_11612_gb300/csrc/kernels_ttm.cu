// Mode-n products (Section 2) for the truncation B <- B x_n U_n^T of
// Algorithms 2/5, the core chain G = A x_1 U_1^T ... x_N U_N^T of Algorithms
// 1/4, and the reconstruction used by the relative error (Eq. 8); plus
// deterministic sums of squares.
//
// Each CTA takes JB = 64 NF consecutive mode-n fibers and OB = 4 OPT output
// indices; the fiber tile streams through shared memory in chunks of KC input
// indices while the JB x OB block of results stays in registers, so the input
// is read once per output block (one block whenever K_out <= 64).
#include <algorithm>

#include "blocks.cuh"
#include "internal.h"
#include "tc.cuh"
#include "tma.cuh"

namespace tk {
namespace {

constexpr int kT = kThreads;
// Block (blockIdx.x, blockIdx.y) of the register-staged mode-n product: JB =
// 64 NF fibers by OB = 4 OPT outputs (the block program's layout and order).
template <typename T, int OPT, int NF>
__global__ void __launch_bounds__(kT) ttm_kernel(const T* __restrict__ A, ModeView v, const T* __restrict__ Mp,
                                                 int64_t K_out, int64_t ld_i, int64_t ld_k, T* __restrict__ out) {
    __shared__ __align__(16) unsigned char smem[blk::ttm_block_smem<T, OPT, NF>()];
    blk::ttm_block<T, OPT, NF, true>(A, v, Mp, K_out, ld_i, ld_k, out, blockIdx.x, blockIdx.y, smem);
}

// TMA-fed FP32 mode-n product. Each CTA takes JB = 128 consecutive fibers
// (contiguous fibers: 128 fibers of the mode-1 view; strided fibers: 128
// consecutive l of one slab t, the last tile of a slab partly beyond L_f) and
// OB = 4 OPT outputs. The fiber tile arrives in chunks of 32 input indices
// (16 KB) by cp.async.bulk.tensor into a ring of 2 or 3 shared-memory stages
// (the autotuner picks; 2 by default); the CTA's block of M stays in shared
// memory. Two stages keep a CTA near 66 KB so three fit on an SM: the kernel is
// bound by issue (20 multiply-adds per element at K_out = 20), and occupancy
// beat deeper staging when measured (4 stages: 0.151 ms, 2 stages: 0.137 ms on
// a 400^3 mode-2 product). Contiguous fibers land 128B-swizzled (16-byte chunk
// c of fiber row r at chunk c ^ (r % 8)), so the four-index reads of eight
// neighbouring fibers hit distinct banks; strided fibers land index-major.
// One thread waits (bounded) on each stage's mbarrier and refills the stage
// once every thread has read it; out-of-range indices and fibers load as 0.
constexpr int kTJB = 128, kTKC = 32;
constexpr uint32_t kTStageBytes = kTJB * kTKC * 4;
constexpr int kTWaitIters = 1 << 24;

__host__ __device__ inline int tma_ipad(int I) { return (I + kTKC - 1) / kTKC * kTKC; }

template <int OPT, bool CONTIG, int kTStages>
__global__ void __launch_bounds__(kT, 3) ttm_tma_kernel(const __grid_constant__ CUtensorMap map, ModeView v,
                                                        const float* __restrict__ Mp, int64_t K_out, int64_t ld_i,
                                                        int64_t ld_k, float* __restrict__ out, int64_t tiles_per_t,
                                                        int* status) {
    constexpr int NF = 2, OB = 4 * OPT;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the 128B swizzle is a function of the shared-memory address, so the
    // stages start on a 1024-byte boundary (the launch adds 1 KB of slack)
    unsigned char* smem = smem_raw + ((1024 - (tma::smem_addr(smem_raw) & 1023)) & 1023);
    const int I = (int)v.i;
    const int Ip = tma_ipad(I);
    const int nch = Ip / kTKC;
    float* Ms = reinterpret_cast<float*>(smem + kTStages * kTStageBytes);   // [OB][Ip]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(Ms + (size_t)OB * Ip);     // [kTStages]
    __shared__ int flag;
    const int tid = threadIdx.x;
    const int64_t o0 = (int64_t)blockIdx.y * OB;
    int64_t j0 = 0, t = 0;
    int l0 = 0;
    if (CONTIG) {
        j0 = (int64_t)blockIdx.x * kTJB;
    } else {
        t = blockIdx.x / tiles_per_t;
        l0 = (int)(blockIdx.x - t * tiles_per_t) * kTJB;
    }
    if (tid == 0) {
        for (int s = 0; s < kTStages; ++s) tc::mbar_init(&mbar[s], 1);
        flag = 0;
        tma::fence_barrier_init();
    }
    __syncthreads();
    auto issue = [&](int c) {
        const int s = c % kTStages;
        unsigned char* dst = smem + s * kTStageBytes;
        tma::expect_tx(&mbar[s], kTStageBytes);
        if (CONTIG) tma::load_2d(dst, &map, c * kTKC, (int)j0, &mbar[s]);
        else tma::load_3d(dst, &map, l0, c * kTKC, (int)t, &mbar[s]);
    };
    if (tid == 0)
        for (int c = 0; c < nch && c < kTStages; ++c) issue(c);
    // the CTA's block of M (outputs o0 .. o0 + OB - 1), zero beyond I and K_out
    for (int e = tid; e < OB * Ip; e += kT) {
        const int o = e / Ip, i = e - o * Ip;
        Ms[e] = (i < I && o0 + o < K_out) ? __ldg(Mp + (int64_t)i * ld_i + (o0 + o) * ld_k) : 0.f;
    }
    __syncthreads();
    const int jl = tid % 64, og = tid / 64;
    float acc[NF][OPT];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int u = 0; u < OPT; ++u) acc[f][u] = 0.f;
    int c = 0;
    for (; c < nch; ++c) {
        const int s = c % kTStages;
        if (tid == 0 && !tc::mbar_wait(&mbar[s], (c / kTStages) & 1, kTWaitIters)) {
            flag = 1;
            set_status(status, kStatTimeout);
        }
        __syncthreads();
        if (flag) break;
        const unsigned char* st = smem + s * kTStageBytes;
        const float* mrow = Ms + c * kTKC;
#pragma unroll 2
        for (int kk = 0; kk < kTKC; kk += 4) {
            float t4[NF][4];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const int jj = jl + 64 * f;
                if (CONTIG) {
                    const float4 x = *reinterpret_cast<const float4*>(st + jj * 128 + ((((kk >> 2) ^ (jj & 7))) << 4));
                    t4[f][0] = x.x; t4[f][1] = x.y; t4[f][2] = x.z; t4[f][3] = x.w;
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) t4[f][q] = *reinterpret_cast<const float*>(st + (kk + q) * (kTJB * 4) + jj * 4);
                }
            }
#pragma unroll
            for (int u = 0; u < OPT; ++u) {
                const float4 m = *reinterpret_cast<const float4*>(mrow + (size_t)(og * OPT + u) * Ip + kk);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    acc[f][u] = fmaf(t4[f][0], m.x, acc[f][u]);
                    acc[f][u] = fmaf(t4[f][1], m.y, acc[f][u]);
                    acc[f][u] = fmaf(t4[f][2], m.z, acc[f][u]);
                    acc[f][u] = fmaf(t4[f][3], m.w, acc[f][u]);
                }
            }
        }
        __syncthreads();                                   // every thread is done with stage s
        if (tid == 0 && c + kTStages < nch) issue(c + kTStages);
    }
    if (flag) {
        // stop only once the copies already issued into this CTA's stages have
        // landed (each waited with the same bound)
        if (tid == 0)
            for (int cc = c; cc < nch && cc < c + kTStages; ++cc)
                tc::mbar_wait(&mbar[cc % kTStages], (cc / kTStages) & 1, kTWaitIters);
        __syncthreads();
        return;
    }
    // results through shared memory (the stages are free now) for coalesced stores
    float (*Os)[OB + 1] = reinterpret_cast<float (*)[OB + 1]>(smem);
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int u = 0; u < OPT; ++u) Os[jl + 64 * f][og * OPT + u] = acc[f][u];
    __syncthreads();
    const int64_t J = v.fibers();
    if (CONTIG) {
        for (int e = tid; e < kTJB * OB; e += kT) {
            const int r = e / OB, oo = e % OB;
            const int64_t j = j0 + r, o = o0 + oo;
            if (j < J && o < K_out) out[j * K_out + o] = Os[r][oo];
        }
    } else {
        for (int e = tid; e < kTJB * OB; e += kT) {
            const int r = e % kTJB, oo = e / kTJB;
            const int64_t l = l0 + r, o = o0 + oo;
            if (l < v.lf && o < K_out) out[l + o * v.lf + t * v.lf * K_out] = Os[r][oo];
        }
    }
}

size_t ttm_tma_smem(int I, int OPT, int stages) {
    return 1024 + (size_t)stages * kTStageBytes + (size_t)4 * OPT * tma_ipad(I) * sizeof(float) + 8 * stages;
}

// Encodes the tile map and launches; false when the shape or alignment does not
// suit the TMA path (the caller then runs ttm_kernel).
template <int OPT, int STAGES>
bool launch_ttm_tma_t(const float* A, const ModeView& v, const float* Mp, int64_t K_out, int64_t ld_i, int64_t ld_k,
                      float* out, int* status, cudaStream_t s, cudaError_t* err) {
    const bool contig = v.lf == 1;
    const int64_t J = v.fibers();
    CUtensorMap map;
    bool ok;
    int64_t tiles, tiles_per_t = 1;
    if (contig) {
        const uint64_t dims[2] = {(uint64_t)v.i, (uint64_t)J};
        const uint64_t strides[1] = {(uint64_t)v.i * 4};
        const uint32_t box[2] = {kTKC, kTJB};
        ok = v.i % 4 == 0 && tma::make_map_f32(&map, A, 2, dims, strides, box, true);
        tiles = (J + kTJB - 1) / kTJB;
    } else {
        const uint64_t dims[3] = {(uint64_t)v.lf, (uint64_t)v.i, (uint64_t)v.rt};
        const uint64_t strides[2] = {(uint64_t)v.lf * 4, (uint64_t)v.lf * v.i * 4};
        const uint32_t box[3] = {kTJB, kTKC, 1};
        ok = v.lf % 4 == 0 && tma::make_map_f32(&map, A, 3, dims, strides, box, false);
        tiles_per_t = (v.lf + kTJB - 1) / kTJB;
        tiles = tiles_per_t * v.rt;
    }
    const size_t smem = ttm_tma_smem((int)v.i, OPT, STAGES);
    if (!ok || smem > 200 * 1024 || tiles > 0x7fffffff) return false;
    dim3 grid((unsigned)tiles, (unsigned)((K_out + 4 * OPT - 1) / (4 * OPT)));
    if (contig) {
        auto k = ttm_tma_kernel<OPT, true, STAGES>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, kT, smem, s>>>(map, v, Mp, K_out, ld_i, ld_k, out, tiles_per_t, status);
    } else {
        auto k = ttm_tma_kernel<OPT, false, STAGES>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, kT, smem, s>>>(map, v, Mp, K_out, ld_i, ld_k, out, tiles_per_t, status);
    }
    note_launch();
    *err = cudaGetLastError();
    return true;
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

// Energies of the mode-n slices of Y (viewed as [rt][K][lf], lf fastest):
// e_k = sum of Y^2 over slice k, i.e. ||u_k^T B_(n)||^2 when Y = B x_n U^T.
// Long runs (lf >= kT): block (k, c) reads chunk c of slice k, runs of lf
// consecutive elements. Short runs: Y is the [rt][K lf] matrix and each thread
// sums one column over a chunk of rows (consecutive threads, consecutive
// columns). Partials are reduced in a fixed order: the result is deterministic.
template <typename T>
__global__ void __launch_bounds__(kT) slice_sumsq_runs_kernel(const T* __restrict__ Y, int64_t lf, int64_t K,
                                                              int64_t rt, double* __restrict__ partial) {
    __shared__ double sh[kT / 32];
    const int64_t k = blockIdx.x;
    const int chunks = (int)gridDim.y, c = (int)blockIdx.y;
    const int64_t per = lf * rt;
    double acc = 0.0;
    for (int64_t e = (int64_t)c * kT + threadIdx.x; e < per; e += (int64_t)chunks * kT) {
        const int64_t o = e / lf, i = e - o * lf;
        const double v = (double)Y[(o * K + k) * lf + i];
        acc = fma(v, v, acc);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kT / 32; ++w) t += sh[w];
        partial[k * chunks + c] = t;
    }
}

template <typename T>
__global__ void __launch_bounds__(kT) slice_sumsq_cols_kernel(const T* __restrict__ Y, int64_t W, int64_t rt,
                                                              double* __restrict__ partial) {
    const int64_t m = (int64_t)blockIdx.x * kT + threadIdx.x;
    const int chunks = (int)gridDim.y, c = (int)blockIdx.y;
    if (m >= W) return;
    double acc = 0.0;
    for (int64_t o = c; o < rt; o += chunks) {
        const double v = (double)Y[o * W + m];
        acc = fma(v, v, acc);
    }
    partial[(int64_t)c * W + m] = acc;
}

// e_k from the partials: runs layout [K][chunks], columns layout [chunks][K lf].
__global__ void slice_sum_partials_kernel(const double* __restrict__ partial, int64_t K, int chunks, int64_t lf,
                                          bool cols, double* __restrict__ e) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double t = 0.0;
    if (!cols) {
        for (int c = 0; c < chunks; ++c) t += partial[k * chunks + c];
    } else {
        for (int c = 0; c < chunks; ++c)
            for (int64_t i = 0; i < lf; ++i) t += partial[(int64_t)c * K * lf + k * lf + i];
    }
    e[k] = t;
}

struct SliceSplit {
    bool runs;
    int chunks;
};
SliceSplit slice_split(const ModeView& v, int num_sms) {
    SliceSplit sp;
    sp.runs = v.lf >= kT;
    const int64_t target = 4 * (int64_t)num_sms;
    if (sp.runs) {
        const int64_t c = (target + v.i - 1) / v.i;
        sp.chunks = (int)std::max<int64_t>(1, std::min<int64_t>(c, 256));
    } else {
        const int64_t tiles = (v.i * v.lf + kT - 1) / kT;
        const int64_t c = (target + tiles - 1) / tiles;
        sp.chunks = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(c, 64), std::max<int64_t>(v.rt, 1)));
    }
    return sp;
}

}  // namespace

template <typename T>
cudaError_t launch_ttm(const T* A, const ModeView& v, const T* Mp, int64_t K_out, int64_t ld_i, int64_t ld_k, T* out,
                       cudaStream_t s, int* status) {
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
    auto run_register = [&]() -> cudaError_t {
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
    };
    if constexpr (sizeof(T) == 4) {
        // FP32 with a status word for the bounded waits: the TMA-fed kernel where
        // the shape and alignment allow it (2 stages unless the tuner chose else)
        if (status && (reinterpret_cast<uintptr_t>(A) & 15) == 0) {
            auto run_tma = [&](int stages, cudaError_t* e) -> bool {
#define TK_TMA_CASE(O)                                                                                        \
    case O:                                                                                                   \
        return stages == 3 ? launch_ttm_tma_t<O, 3>(A, v, Mp, K_out, ld_i, ld_k, out, status, s, e)          \
                           : launch_ttm_tma_t<O, 2>(A, v, Mp, K_out, ld_i, ld_k, out, status, s, e);
                switch (OPT) {
                    TK_TMA_CASE(1) TK_TMA_CASE(2) TK_TMA_CASE(3) TK_TMA_CASE(4) TK_TMA_CASE(5)
                    TK_TMA_CASE(6) TK_TMA_CASE(8) TK_TMA_CASE(12)
                    default: TK_TMA_CASE(16)
                }
#undef TK_TMA_CASE
            };
            // candidates: 0 register-staged, 1 TMA 2 stages, 2 TMA 3 stages (same results)
            auto run = [&](int c) -> cudaError_t {
                if (c == 0) return run_register();
                cudaError_t e = cudaSuccess;
                return run_tma(c == 1 ? 2 : 3, &e) ? e : cudaErrorNotSupported;
            };
            const TuneKey key{kTuneTtm, {v.i, K_out, v.lf, J}};
            int choice = tune_get(key);
            if (choice < 0 && tune_active(s))
                choice = tune_pick(s, key, "mode-n product (I, K_out, L_f, J)", {"register", "tma2", "tma3"}, run, 1);
            if (choice < 0) choice = 1;
            const cudaError_t e = run(choice);
            if (e != cudaErrorNotSupported) return e;
            cudaGetLastError();
        }
    }
    return run_register();
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
                                       cudaStream_t, int*);
template cudaError_t launch_ttm<double>(const double*, const ModeView&, const double*, int64_t, int64_t, int64_t,
                                        double*, cudaStream_t, int*);
template cudaError_t launch_sumsq<float>(const float*, const float*, int64_t, double*, void*, cudaStream_t);
template cudaError_t launch_sumsq<double>(const double*, const double*, int64_t, double*, void*, cudaStream_t);

size_t slice_sumsq_scratch_bytes(const ModeView& v, int num_sms) {
    const SliceSplit sp = slice_split(v, num_sms);
    const int64_t n = sp.runs ? v.i * sp.chunks : (int64_t)sp.chunks * v.i * v.lf;
    return sizeof(double) * (size_t)n + 256;
}

template <typename T>
cudaError_t launch_slice_sumsq(const T* Y, const ModeView& v, double* e, void* scratch, int num_sms,
                               cudaStream_t s) {
    if (v.i < 1 || v.fibers() < 1) return cudaSuccess;
    if (v.i > 65535) return cudaErrorInvalidValue;
    const SliceSplit sp = slice_split(v, num_sms);
    double* partial = reinterpret_cast<double*>(scratch);
    if (sp.runs) {
        slice_sumsq_runs_kernel<T><<<dim3((unsigned)v.i, (unsigned)sp.chunks), kT, 0, s>>>(Y, v.lf, v.i, v.rt,
                                                                                          partial);
    } else {
        const int64_t W = v.i * v.lf;
        slice_sumsq_cols_kernel<T><<<dim3((unsigned)((W + kT - 1) / kT), (unsigned)sp.chunks), kT, 0, s>>>(
            Y, W, v.rt, partial);
    }
    note_launch();
    slice_sum_partials_kernel<<<(unsigned)((v.i + 127) / 128), 128, 0, s>>>(partial, v.i, sp.chunks,
                                                                             sp.runs ? 1 : v.lf, !sp.runs, e);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t launch_slice_sumsq<float>(const float*, const ModeView&, double*, void*, int, cudaStream_t);
template cudaError_t launch_slice_sumsq<double>(const double*, const ModeView&, double*, void*, int,
                                                cudaStream_t);

}  // namespace tk
