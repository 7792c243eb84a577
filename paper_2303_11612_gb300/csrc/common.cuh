// Shared device helpers of the randomized Tucker library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tucker.h"

namespace tk {

constexpr int kThreads = 256;

// Device status word bits (OR-ed by kernels, read by the host at the end of a call).
enum : int { kStatNumerical = 1, kStatTimeout = 2, kStatShifted = 4 };

// ------------------------------------------------------------------ mode-n view
// The mode-n unfolding of an I_1 x ... x I_N tensor (i_1 fastest) as a 3-D
// array (Lf, I, Rt): Lf = prod_{m<n} I_m (fastest), I = I_n, Rt = prod_{m>n} I_m.
// Column j of A_(n) is the fiber (l, r) with j = l + r * Lf (Section 2 index map);
// its element i sits at l + i * Lf + r * Lf * I.
struct ModeView {
    int64_t lf;
    int64_t i;
    int64_t rt;
    __host__ __device__ int64_t fibers() const { return lf * rt; }
    __host__ __device__ int64_t base(int64_t j) const {
        if (lf == 1) return j * i;
        int64_t r = j / lf;
        return (j - r * lf) + r * lf * i;
    }
    __host__ __device__ int64_t stride() const { return lf; }
};

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of two 32x32->64 multiplies,
// the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 philox_block(uint64_t seed, uint32_t stream, uint64_t block) {
    return philox(make_uint4((uint32_t)block, (uint32_t)(block >> 32), stream, 0u),
                  (uint32_t)seed, (uint32_t)(seed >> 32));
}

// u = ((x >> 9) + 0.5) 2^-23, exact in FP32 and FP64, strictly inside (0, 1).
__device__ __forceinline__ float u01f(uint32_t x) { return ((float)(x >> 9) + 0.5f) * 1.1920928955078125e-07f; }
__device__ __forceinline__ double u01d(uint32_t x) { return ((double)(x >> 9) + 0.5) * 1.1920928955078125e-07; }

// Gaussian element e of a stream: block e/4, lane e%4, Box-Muller on lane pairs.
template <typename T> __device__ __forceinline__ T gaussian_at(uint64_t seed, uint32_t stream, uint64_t e);
template <> __device__ __forceinline__ float gaussian_at<float>(uint64_t seed, uint32_t stream, uint64_t e) {
    const uint4 x = philox_block(seed, stream, e >> 2);
    const int lane = (int)(e & 3);
    const uint32_t a = lane < 2 ? x.x : x.z, b = lane < 2 ? x.y : x.w;
    const float r = sqrtf(-2.0f * logf(u01f(a)));
    float s, c;
    sincospif(2.0f * u01f(b), &s, &c);
    return r * ((lane & 1) ? s : c);
}
template <> __device__ __forceinline__ double gaussian_at<double>(uint64_t seed, uint32_t stream, uint64_t e) {
    const uint4 x = philox_block(seed, stream, e >> 2);
    const int lane = (int)(e & 3);
    const uint32_t a = lane < 2 ? x.x : x.z, b = lane < 2 ? x.y : x.w;
    const double r = sqrt(-2.0 * log(u01d(a)));
    double s, c;
    sincospi(2.0 * u01d(b), &s, &c);
    return r * ((lane & 1) ? s : c);
}

// ------------------------------------------------------------------ paired-FP32 sums
// Sums of FP32 products carried as an unevaluated pair (hi, lo): the product's
// rounding error comes exactly from an FMA and the addition's from Knuth's
// TwoSum, so the pair holds the sum to about 2^-44 relative while running on
// the FP32 pipes (GB300's FP64 rate is far lower).
struct Pair {
    float hi, lo;
};
__device__ __forceinline__ void pair_add_prod(Pair& s, float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    const float t = s.hi + p;
    const float z = t - s.hi;
    const float e = (s.hi - (t - z)) + (p - z);
    s.hi = t;
    s.lo += e + pe;
}
__device__ __forceinline__ void pair_add(Pair& s, Pair o) {
    const float t = s.hi + o.hi;
    const float z = t - s.hi;
    const float e = (s.hi - (t - z)) + (o.hi - z);
    s.hi = t;
    s.lo += e + o.lo;
}
__device__ __forceinline__ double pair_value(Pair s) { return (double)s.hi + (double)s.lo; }

__device__ __forceinline__ Pair warp_sum_pair(Pair s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Pair t;
        t.hi = __shfl_xor_sync(0xffffffffu, s.hi, o);
        t.lo = __shfl_xor_sync(0xffffffffu, s.lo, o);
        pair_add(s, t);
    }
    return s;
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void set_status(int* st, int bits) {
    if (st) atomicOr(st, bits);
}

}  // namespace tk
