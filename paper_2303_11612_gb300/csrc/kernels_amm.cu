// Approximate matrix multiplication by fiber sampling (Section 3.2,
// Algorithms 3-5): squared fiber norms, integer sampling weights, their
// inclusive prefix sum, the multinomial draws (inverse CDF, exact integer
// arithmetic) and the rescaled gather C' = A_(n) S.
#include "internal.h"

namespace tk {
namespace {

constexpr int kT = kThreads;
constexpr int kScanItems = 4;                 // elements per thread in the scan
constexpr int kScanBlock = kT * kScanItems;   // elements per scan block

// ---------------------------------------------------------------- fiber norms
template <typename T> struct NormAcc;
template <> struct NormAcc<float> {
    Pair s{0.f, 0.f};
    __device__ void add(float x) { pair_add_prod(s, x, x); }
    __device__ void warp_reduce() { s = warp_sum_pair(s); }
    __device__ double value() const { return pair_value(s); }
};
template <> struct NormAcc<double> {
    double s = 0.0;
    __device__ void add(double x) { s = fma(x, x, s); }
    __device__ void warp_reduce() { s = warp_sum(s); }
    __device__ double value() const { return s; }
};

// Contiguous fibers (mode 1): one warp per fiber; each lane issues its loads in
// predicated batches of 16 (coalesced 128-byte rows) before summing them.
template <typename T>
__global__ void __launch_bounds__(kT) norms_contig_kernel(const T* __restrict__ A, int64_t I, int64_t J,
                                                          double* __restrict__ w) {
    constexpr int kB = 16;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)kT + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kT) >> 5;
    for (int64_t j = warp; j < J; j += nwarps) {
        NormAcc<T> acc;
        const T* f = A + j * I;
        for (int64_t i0 = 0; i0 < I; i0 += 32 * kB) {
            T x[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int64_t i = i0 + lane + 32 * u;
                x[u] = i < I ? __ldg(f + i) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) acc.add(x[u]);
        }
        acc.warp_reduce();
        if (lane == 0) w[j] = acc.value();
    }
}

// Strided fibers: 32 FW consecutive fibers per block (consecutive lanes read
// consecutive addresses: neighbouring fibers differ in the fastest index; FW
// warps side by side read 128 FW contiguous bytes), the fiber's I_n values
// split over the block's kT / (32 FW) warp groups (group w takes
// i = w, w + groups, ...); the per-group sums are combined in group order.
template <typename T> struct NormPart;
template <> struct NormPart<float> {
    static __device__ void merge(NormAcc<float>& a, const NormAcc<float>& b) { pair_add(a.s, b.s); }
};
template <> struct NormPart<double> {
    static __device__ void merge(NormAcc<double>& a, const NormAcc<double>& b) { a.s += b.s; }
};

template <typename T, int FW>
__global__ void __launch_bounds__(kT) norms_strided_kernel(const T* __restrict__ A, ModeView v,
                                                           double* __restrict__ w) {
    constexpr int kG = kT / (32 * FW);          // warp groups along i
    constexpr int kF = 32 * FW;                 // fibers per block
    __shared__ __align__(16) unsigned char part_raw[kG * kF * sizeof(NormAcc<T>)];
    NormAcc<T>(*part)[kF] = reinterpret_cast<NormAcc<T>(*)[kF]>(part_raw);
    const int f = threadIdx.x % kF, grp = threadIdx.x / kF;
    const int64_t J = v.fibers();
    for (int64_t j0 = (int64_t)blockIdx.x * kF; j0 < J; j0 += (int64_t)gridDim.x * kF) {
        const int64_t j = j0 + f;
        NormAcc<T> acc;
        if (j < J) {
            const T* p = A + v.base(j);
            constexpr int kB = 8;
            for (int64_t i0 = grp; i0 < v.i; i0 += (int64_t)kB * kG) {
                T x[kB];
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int64_t i = i0 + (int64_t)u * kG;
                    x[u] = i < v.i ? __ldg(p + i * v.lf) : (T)0;
                }
#pragma unroll
                for (int u = 0; u < kB; ++u) acc.add(x[u]);
            }
        }
        part[grp][f] = acc;
        __syncthreads();
        if (grp == 0 && j < J) {
            NormAcc<T> tot = part[0][f];
            for (int q = 1; q < kG; ++q) NormPart<T>::merge(tot, part[q][f]);
            w[j] = tot.value();
        }
        __syncthreads();
    }
}

// The squared norms of the mode-1 and the mode-2 fibers in one pass (the remark
// after Algorithm 3, for the sampling of both modes in Algorithm 4). The tensor
// is read as I1 x I2 x rest (i1 fastest); slab s of rest is an I1 x I2 matrix
// whose rows (fixed i2) are mode-1 fibers and whose columns (fixed i1) are
// mode-2 fibers. Warp w takes rows i2 = w, w + warps, ...: a row's sum is the
// lanes' partials (lane takes i1 = lane + 32 k, k increasing: the order of
// norms_contig_kernel, so the mode-1 norms are the same) reduced across the
// warp; each lane also adds its elements into its columns' sums over the
// warp's rows, and the warps' column sums are combined in warp order.
template <typename T, int NK>
__global__ void __launch_bounds__(kT) norms12_kernel(const T* __restrict__ A, int64_t I1, int64_t I2, int64_t rest,
                                                     double* __restrict__ w1, double* __restrict__ w2) {
    constexpr int kW = kT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    NormAcc<T>* part = reinterpret_cast<NormAcc<T>*>(smem_raw);    // [kW][I1]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t s = blockIdx.x; s < rest; s += gridDim.x) {
        const T* slab = A + s * I1 * I2;
        NormAcc<T> col[NK];
        for (int64_t i2 = warp; i2 < I2; i2 += kW) {
            const T* row = slab + i2 * I1;
            T x[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const int64_t i = lane + 32 * k;
                x[k] = i < I1 ? __ldg(row + i) : T(0);
            }
            NormAcc<T> r;
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                r.add(x[k]);
                col[k].add(x[k]);
            }
            r.warp_reduce();
            if (lane == 0) w1[i2 + I2 * s] = r.value();
        }
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const int64_t i = lane + 32 * k;
            if (i < I1) part[warp * I1 + i] = col[k];
        }
        __syncthreads();
        for (int64_t i = threadIdx.x; i < I1; i += kT) {
            NormAcc<T> t = part[i];
            for (int q = 1; q < kW; ++q) NormPart<T>::merge(t, part[q * I1 + i]);
            w2[i + I1 * s] = t.value();
        }
        __syncthreads();
    }
}

// All three modes' squared fiber norms of an order-3 tensor from one pass
// (Algorithm 4 samples every mode of the same tensor). CTA (b, c) takes the
// band of rows i_2 = b RB .. b RB + RB - 1 (RB = 8 RR: warp w owns rows
// b RB + w + 8 r, r < RR) of the slabs i_3 of chunk c. Mode 1: a row's sum is
// complete, formed as norms_contig forms it (bitwise equal where that takes a
// warp per fiber). Mode 2: per slab, the band's column sums (each warp's rows
// in order, then the warps in order) go to P2[b] (i_1 + I_1 i_3). Mode 3: each
// entry's sum over the chunk's slabs, in order, kept in shared memory beside
// the band, goes to P3[c] (i_1 + I_1 i_2). norms_merge_kernel then adds the
// bands' and the chunks' partials in order. A warp issues all its rows' loads
// of a slab before summing them.
template <typename T, int NK, int RR>
__global__ void __launch_bounds__(kT) norms123_kernel(const T* __restrict__ A, int64_t I1, int64_t I2, int64_t I3,
                                                      int64_t SC, double* __restrict__ w1, NormAcc<T>* __restrict__ P2,
                                                      NormAcc<T>* __restrict__ P3) {
    constexpr int kW = kT / 32, RB = kW * RR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    NormAcc<T>* part = reinterpret_cast<NormAcc<T>*>(smem_raw);    // [kW][I1]
    NormAcc<T>* m3 = part + kW * I1;                                // [RB][I1]: row warp + kW r at r kW + warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = blockIdx.x, c = blockIdx.y;
    const int64_t s0 = c * SC, s1 = s0 + SC < I3 ? s0 + SC : I3;
    for (int64_t e = threadIdx.x; e < RB * I1; e += kT) m3[e] = NormAcc<T>();
    __syncthreads();
    for (int64_t s = s0; s < s1; ++s) {
        const T* slab = A + s * I1 * I2;
        T x[RR][NK];
#pragma unroll
        for (int r = 0; r < RR; ++r) {
            const int64_t i2 = b * RB + warp + kW * r;
            const T* row = slab + i2 * I1;
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const int64_t i = lane + 32 * k;
                x[r][k] = (i2 < I2 && i < I1) ? __ldg(row + i) : T(0);
            }
        }
        NormAcc<T> col[NK];
#pragma unroll
        for (int r = 0; r < RR; ++r) {
            const int64_t i2 = b * RB + warp + kW * r;
            if (i2 >= I2) break;                                     // the same for the whole warp
            NormAcc<T>* m3r = m3 + (r * kW + warp) * I1;
            NormAcc<T> rs;
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                rs.add(x[r][k]);
                col[k].add(x[r][k]);
                const int64_t i = lane + 32 * k;
                if (i < I1) {
                    NormAcc<T> t = m3r[i];
                    t.add(x[r][k]);
                    m3r[i] = t;
                }
            }
            rs.warp_reduce();
            if (lane == 0) w1[i2 + I2 * s] = rs.value();
        }
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const int64_t i = lane + 32 * k;
            if (i < I1) part[warp * I1 + i] = col[k];
        }
        __syncthreads();
        NormAcc<T>* out2 = P2 + b * (I1 * I3) + I1 * s;
        for (int64_t i = threadIdx.x; i < I1; i += kT) {
            NormAcc<T> t = part[i];
            for (int q = 1; q < kW; ++q) NormPart<T>::merge(t, part[q * I1 + i]);
            out2[i] = t;
        }
        __syncthreads();
    }
    NormAcc<T>* out3 = P3 + c * (I1 * I2);
    for (int64_t e = threadIdx.x; e < RB * I1; e += kT) {
        const int64_t slot = e / I1, i = e - slot * I1;
        const int64_t i2 = b * RB + (slot % kW) + kW * (slot / kW);
        if (i2 < I2) out3[i + I1 * i2] = m3[e];
    }
}

// out[x] = the partials P[p count + x], p = 0 .. parts - 1, added in order.
template <typename T>
__global__ void __launch_bounds__(kT) norms_merge_kernel(const NormAcc<T>* __restrict__ P, int64_t parts,
                                                         int64_t count, double* __restrict__ out) {
    for (int64_t x = blockIdx.x * (int64_t)kT + threadIdx.x; x < count; x += (int64_t)gridDim.x * kT) {
        NormAcc<T> t = P[x];
        for (int64_t p = 1; p < parts; ++p) NormPart<T>::merge(t, P[p * count + x]);
        out[x] = t.value();
    }
}

// ---------------------------------------------------------------- integer weights
__global__ void __launch_bounds__(kT) max_kernel(const double* __restrict__ w, int64_t J,
                                                 unsigned long long* __restrict__ out) {
    double m = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)kT + threadIdx.x; j < J; j += (int64_t)gridDim.x * kT)
        m = fmax(m, w[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void __launch_bounds__(kT) quantize_kernel(const double* __restrict__ w, int64_t J, int uniform,
                                                      const unsigned long long* __restrict__ maxbits,
                                                      uint64_t* __restrict__ W) {
    const double wmax = uniform ? 0.0 : __longlong_as_double((long long)*maxbits);
    for (int64_t j = blockIdx.x * (int64_t)kT + threadIdx.x; j < J; j += (int64_t)gridDim.x * kT) {
        uint64_t q = 1;
        if (!uniform && wmax > 0.0) {
            const double x = w[j];
            q = x > 0.0 ? (uint64_t)ceil((x / wmax) * 16777216.0) : 0;
        }
        W[j] = q;
    }
}

// W_j = ceil(w_j / wmax 2^24) with wmax given (the largest weight over every
// slab of a sharded call); 0 for w_j = 0, all ones if wmax is 0.
__global__ void __launch_bounds__(kT) quantize_value_kernel(const double* __restrict__ w, int64_t J, double wmax,
                                                            uint64_t* __restrict__ W) {
    for (int64_t j = blockIdx.x * (int64_t)kT + threadIdx.x; j < J; j += (int64_t)gridDim.x * kT) {
        uint64_t q = 1;
        if (wmax > 0.0) {
            const double x = w[j];
            q = x > 0.0 ? (uint64_t)ceil((x / wmax) * 16777216.0) : 0;
        }
        W[j] = q;
    }
}

// ---------------------------------------------------------------- inclusive scan
__device__ __forceinline__ uint64_t block_inclusive_scan(uint64_t x, uint64_t* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t s = lane < kT / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kT / 32) sh[lane] = s;
    }
    __syncthreads();
    const uint64_t off = warp ? sh[warp - 1] : 0;
    __syncthreads();
    return x + off;
}

__global__ void __launch_bounds__(kT) scan_block_sums(const uint64_t* __restrict__ W, int64_t J,
                                                      uint64_t* __restrict__ bsum) {
    __shared__ uint64_t sh[kT / 32];
    const int64_t base = blockIdx.x * (int64_t)kScanBlock + threadIdx.x * kScanItems;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < J) s += W[base + k];
    s = block_inclusive_scan(s, sh);
    if (threadIdx.x == kT - 1) bsum[blockIdx.x] = s;
}

// Exclusive scan of the block sums in one block, in chunks of kT.
__global__ void __launch_bounds__(kT) scan_offsets(uint64_t* __restrict__ bsum, int64_t nb) {
    __shared__ uint64_t sh[kT / 32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t c = 0; c < nb; c += kT) {
        const int64_t k = c + threadIdx.x;
        const uint64_t x = k < nb ? bsum[k] : 0;
        const uint64_t inc = block_inclusive_scan(x, sh);
        const uint64_t base = carry;
        if (k < nb) bsum[k] = base + inc - x;
        __syncthreads();
        if (threadIdx.x == kT - 1) carry = base + inc;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kT) scan_final(const uint64_t* __restrict__ W, int64_t J,
                                                 const uint64_t* __restrict__ boff, uint64_t* __restrict__ cdf) {
    __shared__ uint64_t sh[kT / 32];
    const int64_t base = blockIdx.x * (int64_t)kScanBlock + threadIdx.x * kScanItems;
    uint64_t v[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < J ? W[base + k] : 0;
        s += v[k];
    }
    const uint64_t inc = block_inclusive_scan(s, sh);
    uint64_t run = boff[blockIdx.x] + inc - s;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        run += v[k];
        if (base + k < J) cdf[base + k] = run;
    }
}

// ---------------------------------------------------------------- multinomial draws
__global__ void __launch_bounds__(kT) sample_kernel(const uint64_t* __restrict__ cdf, const uint64_t* __restrict__ W,
                                                    int64_t J, int64_t T_, uint64_t seed, uint32_t stream_id,
                                                    int64_t* __restrict__ idx, double* __restrict__ scale) {
    const uint64_t S = cdf[J - 1];
    for (int64_t t = blockIdx.x * (int64_t)kT + threadIdx.x; t < T_; t += (int64_t)gridDim.x * kT) {
        const uint4 x = philox_block(seed, stream_id, (uint64_t)(t >> 1));
        const uint64_t r = (t & 1) ? ((uint64_t)x.w << 32 | x.z) : ((uint64_t)x.y << 32 | x.x);
        const uint64_t v = __umul64hi(r, S);          // floor(r * S / 2^64)
        int64_t lo = 0, hi = J - 1;                   // least j with cdf[j] > v
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cdf[mid] > v) hi = mid; else lo = mid + 1;
        }
        idx[t] = lo;
        const double p = (double)W[lo] / (double)S;
        scale[t] = 1.0 / sqrt((double)T_ * p);
    }
}

// The draws of one slab of a sharded call: the slab's fibers are global fibers
// fiber_offset .. fiber_offset + J - 1 and its weights the CDF range
// [S_offset, S_offset + S_slab) of the whole S_total. Draw t falls in this slab
// when S_offset <= v_t < S_offset + S_slab; then idx[t] is its global index and
// scale[t] its scale, else idx[t] = -1 and scale[t] = 0 (the owning slab sets them).
__global__ void __launch_bounds__(kT) sample_slab_kernel(const uint64_t* __restrict__ cdf,
                                                         const uint64_t* __restrict__ W, int64_t J, int64_t T_,
                                                         uint64_t seed, uint32_t stream_id, uint64_t S_offset,
                                                         uint64_t S_total, int64_t fiber_offset,
                                                         int64_t* __restrict__ idx, double* __restrict__ scale) {
    const uint64_t S_slab = cdf[J - 1];
    for (int64_t t = blockIdx.x * (int64_t)kT + threadIdx.x; t < T_; t += (int64_t)gridDim.x * kT) {
        const uint4 x = philox_block(seed, stream_id, (uint64_t)(t >> 1));
        const uint64_t r = (t & 1) ? ((uint64_t)x.w << 32 | x.z) : ((uint64_t)x.y << 32 | x.x);
        const uint64_t v = __umul64hi(r, S_total);
        if (v < S_offset || v - S_offset >= S_slab) {
            idx[t] = -1;
            scale[t] = 0.0;
            continue;
        }
        const uint64_t u = v - S_offset;
        int64_t lo = 0, hi = J - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cdf[mid] > u) hi = mid; else lo = mid + 1;
        }
        idx[t] = lo + fiber_offset;
        const double p = (double)W[lo] / (double)S_total;
        scale[t] = 1.0 / sqrt((double)T_ * p);
    }
}

// ---------------------------------------------------------------- rescaled gather
template <typename T>
__global__ void __launch_bounds__(kT) gather_kernel(const T* __restrict__ A, ModeView v,
                                                    const int64_t* __restrict__ idx,
                                                    const double* __restrict__ scale, int64_t T_,
                                                    T* __restrict__ Cp) {
    // one warp per sampled fiber; lanes walk the fiber
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)kT + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kT) >> 5;
    for (int64_t t = warp; t < T_; t += nwarps) {
        const T* f = A + v.base(idx[t]);
        const T s = (T)scale[t];
        T* out = Cp + t * v.i;
        for (int64_t i = lane; i < v.i; i += 32) out[i] = s * __ldg(f + i * v.lf);
    }
}

unsigned grid_for(int64_t n, int per_block, int cap) {
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

}  // namespace

template <typename T>
cudaError_t launch_fiber_norms(const T* A, const ModeView& v, double* w, cudaStream_t s) {
    const int64_t J = v.fibers();
    if (J == 0) return cudaSuccess;
    ProfScope prof(kKNorms, (double)v.i * (double)J * sizeof(T), 2.0 * (double)v.i * (double)J, s);
    // a warp per fiber for long contiguous fibers; otherwise a thread per fiber
    // (for short contiguous fibers the block's fibers still cover one contiguous range)
    if (v.lf == 1 && v.i >= 64)
        norms_contig_kernel<T><<<grid_for(J, kT / 32, 8192), kT, 0, s>>>(A, v.i, J, w);
    else if (v.lf >= 128 && J >= 128 * 152)
        norms_strided_kernel<T, 4><<<grid_for(J, 128, 8192), kT, 0, s>>>(A, v, w);
    else
        norms_strided_kernel<T, 1><<<grid_for(J, 32, 8192), kT, 0, s>>>(A, v, w);
    note_launch();
    return cudaGetLastError();
}

bool fiber_norms12_supported(int64_t I1) { return I1 >= 1 && I1 <= 1024; }

template <typename T>
cudaError_t launch_fiber_norms12(const T* A, int64_t I1, int64_t I2, int64_t rest, double* w1, double* w2,
                                 cudaStream_t s) {
    if (!fiber_norms12_supported(I1) || I2 < 1) return cudaErrorInvalidValue;
    if (rest == 0) return cudaSuccess;
    const double elems = (double)I1 * (double)I2 * (double)rest;
    ProfScope prof(kKNorms, elems * sizeof(T), 4.0 * elems, s);
    const size_t smem = (size_t)(kT / 32) * (size_t)I1 * sizeof(NormAcc<T>);
    const int64_t grid = rest < 4 * (int64_t)num_sms() ? rest : 4 * (int64_t)num_sms();
    auto run = [&](auto kernel) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kernel<<<(unsigned)grid, kT, smem, s>>>(A, I1, I2, rest, w1, w2);
    };
    if (I1 <= 128) run(norms12_kernel<T, 4>);
    else if (I1 <= 256) run(norms12_kernel<T, 8>);
    else if (I1 <= 512) run(norms12_kernel<T, 16>);
    else run(norms12_kernel<T, 32>);
    note_launch();
    return cudaGetLastError();
}

namespace {
// Bands of 8 RR rows (RR = 2 up to I_1 = 512, else 1); chunks of slabs so that
// the grid holds about four CTAs per SM.
struct N123Grid {
    int rr;
    int64_t nb, nc, sc;
};
N123Grid n123_grid(int64_t I1, int64_t I2, int64_t I3) {
    N123Grid g;
    g.rr = I1 <= 512 ? 2 : 1;
    g.nb = (I2 + 8 * g.rr - 1) / (8 * g.rr);
    int64_t nc = (4 * (int64_t)num_sms() + g.nb - 1) / g.nb;
    nc = nc < 1 ? 1 : (nc > I3 ? I3 : nc);
    if (nc > 65535) nc = 65535;
    g.sc = (I3 + nc - 1) / nc;
    g.nc = (I3 + g.sc - 1) / g.sc;
    return g;
}
}  // namespace

bool fiber_norms123_supported(int64_t I1) { return I1 >= 1 && I1 <= 1024; }

size_t fiber_norms123_scratch_bytes(int64_t I1, int64_t I2, int64_t I3) {
    if (!fiber_norms123_supported(I1) || I2 < 1 || I3 < 1) return 0;
    const N123Grid g = n123_grid(I1, I2, I3);
    const size_t p2 = ((size_t)g.nb * I1 * I3 * 8 + 255) & ~size_t(255);
    return p2 + (size_t)g.nc * I1 * I2 * 8;           // NormAcc is 8 bytes for both types
}

template <typename T>
cudaError_t launch_fiber_norms123(const T* A, int64_t I1, int64_t I2, int64_t I3, double* w1, double* w2,
                                  double* w3, void* scratch, cudaStream_t s) {
    static_assert(sizeof(NormAcc<T>) == 8, "partials hold 8 bytes per entry");
    if (!fiber_norms123_supported(I1) || I2 < 1 || I3 < 1 || !scratch) return cudaErrorInvalidValue;
    const double elems = (double)I1 * (double)I2 * (double)I3;
    ProfScope prof(kKNorms, elems * sizeof(T), 6.0 * elems, s);
    const N123Grid g = n123_grid(I1, I2, I3);
    NormAcc<T>* P2 = reinterpret_cast<NormAcc<T>*>(scratch);
    NormAcc<T>* P3 = reinterpret_cast<NormAcc<T>*>((char*)scratch + (((size_t)g.nb * I1 * I3 * 8 + 255) & ~size_t(255)));
    const size_t smem = (size_t)(kT / 32) * (1 + g.rr) * (size_t)I1 * sizeof(NormAcc<T>);
    const dim3 grid((unsigned)g.nb, (unsigned)g.nc);
    auto run = [&](auto kernel) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kernel<<<grid, kT, smem, s>>>(A, I1, I2, I3, g.sc, w1, P2, P3);
    };
    if (I1 <= 128) run(norms123_kernel<T, 4, 2>);
    else if (I1 <= 256) run(norms123_kernel<T, 8, 2>);
    else if (I1 <= 512) run(norms123_kernel<T, 16, 2>);
    else run(norms123_kernel<T, 32, 1>);
    note_launch();
    auto merge = [&](const NormAcc<T>* P, int64_t parts, int64_t count, double* out) {
        const int64_t blocks = (count + kT - 1) / kT;
        const int64_t grid1 = blocks < 4 * (int64_t)num_sms() ? blocks : 4 * (int64_t)num_sms();
        norms_merge_kernel<T><<<(unsigned)(grid1 > 0 ? grid1 : 1), kT, 0, s>>>(P, parts, count, out);
        note_launch();
    };
    merge(P2, g.nb, I1 * I3, w2);
    merge(P3, g.nc, I1 * I2, w3);
    return cudaGetLastError();
}

size_t quantize_scratch_bytes(int64_t) { return 256; }

cudaError_t launch_quantize(const double* w, int64_t J, int prob, uint64_t* W, void* scratch, cudaStream_t s) {
    auto* mx = reinterpret_cast<unsigned long long*>(scratch);
    const int uniform = prob == TUCKER_PROB_UNIFORM;
    if (!uniform) {
        cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s);
        max_kernel<<<grid_for(J, kT, 1024), kT, 0, s>>>(w, J, mx);
        note_launch();
    }
    quantize_kernel<<<grid_for(J, kT, 8192), kT, 0, s>>>(w, J, uniform, mx, W);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_quantize_max(const double* w, int64_t J, double wmax, uint64_t* W, cudaStream_t s) {
    if (J == 0) return cudaSuccess;
    quantize_value_kernel<<<grid_for(J, kT, 8192), kT, 0, s>>>(w, J, wmax, W);
    note_launch();
    return cudaGetLastError();
}

size_t sample_scratch_bytes(int64_t J) {
    const int64_t nb = (J + kScanBlock - 1) / kScanBlock;
    return sizeof(uint64_t) * (size_t)J + sizeof(uint64_t) * (size_t)(nb + 1) + 512;
}

cudaError_t launch_sample(const uint64_t* W, int64_t J, int64_t T_, uint64_t seed, uint32_t stream_id,
                          int64_t* idx, double* scale, void* scratch, cudaStream_t s) {
    if (T_ == 0) return cudaSuccess;
    auto* cdf = reinterpret_cast<uint64_t*>(scratch);
    auto* bsum = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(scratch) +
                                             (((sizeof(uint64_t) * (size_t)J) + 255) & ~size_t(255)));
    const int64_t nb = (J + kScanBlock - 1) / kScanBlock;
    scan_block_sums<<<(unsigned)nb, kT, 0, s>>>(W, J, bsum);
    note_launch();
    scan_offsets<<<1, kT, 0, s>>>(bsum, nb);
    note_launch();
    scan_final<<<(unsigned)nb, kT, 0, s>>>(W, J, bsum, cdf);
    note_launch();
    sample_kernel<<<grid_for(T_, kT, 4096), kT, 0, s>>>(cdf, W, J, T_, seed, stream_id, idx, scale);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sample_slab(const uint64_t* W, int64_t J, int64_t T_, uint64_t seed, uint32_t stream_id,
                               uint64_t S_offset, uint64_t S_total, int64_t fiber_offset, int64_t* idx, double* scale,
                               void* scratch, cudaStream_t s) {
    if (T_ == 0 || J == 0) return cudaSuccess;
    auto* cdf = reinterpret_cast<uint64_t*>(scratch);
    auto* bsum = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(scratch) +
                                             (((sizeof(uint64_t) * (size_t)J) + 255) & ~size_t(255)));
    const int64_t nb = (J + kScanBlock - 1) / kScanBlock;
    scan_block_sums<<<(unsigned)nb, kT, 0, s>>>(W, J, bsum);
    note_launch();
    scan_offsets<<<1, kT, 0, s>>>(bsum, nb);
    note_launch();
    scan_final<<<(unsigned)nb, kT, 0, s>>>(W, J, bsum, cdf);
    note_launch();
    sample_slab_kernel<<<grid_for(T_, kT, 4096), kT, 0, s>>>(cdf, W, J, T_, seed, stream_id, S_offset, S_total,
                                                              fiber_offset, idx, scale);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather(const T* A, const ModeView& v, const int64_t* idx, const double* scale, int64_t T_,
                          T* Cp, cudaStream_t s) {
    if (T_ == 0) return cudaSuccess;
    ProfScope prof(kKGather, 2.0 * (double)v.i * (double)T_ * sizeof(T), (double)v.i * (double)T_, s);
    gather_kernel<T><<<grid_for(T_, kT / 32, 8192), kT, 0, s>>>(A, v, idx, scale, T_, Cp);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t launch_fiber_norms123<float>(const float*, int64_t, int64_t, int64_t, double*, double*,
                                                 double*, void*, cudaStream_t);
template cudaError_t launch_fiber_norms123<double>(const double*, int64_t, int64_t, int64_t, double*, double*,
                                                  double*, void*, cudaStream_t);
template cudaError_t launch_fiber_norms12<float>(const float*, int64_t, int64_t, int64_t, double*, double*,
                                                cudaStream_t);
template cudaError_t launch_fiber_norms12<double>(const double*, int64_t, int64_t, int64_t, double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_fiber_norms<float>(const float*, const ModeView&, double*, cudaStream_t);
template cudaError_t launch_fiber_norms<double>(const double*, const ModeView&, double*, cudaStream_t);
template cudaError_t launch_gather<float>(const float*, const ModeView&, const int64_t*, const double*, int64_t,
                                          float*, cudaStream_t);
template cudaError_t launch_gather<double>(const double*, const ModeView&, const int64_t*, const double*, int64_t,
                                           double*, cudaStream_t);

}  // namespace tk
