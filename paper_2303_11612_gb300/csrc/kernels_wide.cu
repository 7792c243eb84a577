// Tensor-core kernels for contiguous mode-n fibers (mode 1) at shapes beyond
// the tiles of the fused kernels: extents I_n in the thousands and sketch widths
// or output ranks up to 128 (the 1024 x 1024 x 512 workload's mode 1 has
// I_1 = 1024, L_1 = 80, R_1 = 64). tcgen05 kind::f16 with FP32 accumulation in
// tensor memory; operands are bf16, either the single rounding of each FP32
// value (the single-pass BF16 form) or its split a = a_hi + a_lo with the three
// products hi.hi + lo.hi + hi.lo (about 2^-16 relative, the FP32-class forms).
//
// Two contractions, each a plain streaming pass over the tensor:
//
//   wide_ttm_kernel     D[j, o] = sum_i A_(n)[i, j] M[i, o]     (contracts I_n)
//     Tiles of 128 fibers (M of the product, one fiber per accumulator lane),
//     units of 64 values i. TMA loads a unit as two FP32 boxes (128-byte
//     swizzled); sixteen converter warps round or split it into the K-major
//     swizzled bf16 operand; M^T, prepared once per call as a swizzled bf16
//     image in global memory (image_kernel), streams through a small ring
//     by untiled bulk copies, one unit beside each tensor unit (at I_n = 1024
//     the whole M^T does not fit in shared memory beside the rings). N = K_out
//     padded to 16; the accumulator is double-buffered so a tile's read-back
//     overlaps the next tile's products. Outputs: the mode-n product (FP32,
//     fiber-major: out[j K_out + o], the truncation B x_n U^T of Algorithm 2),
//     or W = A_(n)^T X as the bf16 operand image wide_power2_kernel reads.
//
//   wide_power2_kernel  P[i, l] = sum_j A_(n)[i, j] B[j, l]     (contracts J_n)
//     B = W from the kernel above (second half of a power step of Strategy A,
//     X_out = A_(n) W), or the range form's Gaussian Omega (J_n x L), generated
//     per 64-fiber chunk from the Philox stream inside the kernel, so that it
//     never touches HBM. A CTA owns up to 4 blocks of 128 rows i (its row group)
//     and a strided set of 64-fiber chunks; its accumulators (rows on lanes, L
//     padded to 16 columns per block) stay in tensor memory across its chunks
//     and are written once as its partial; partials are summed in a fixed order
//     afterwards. TMA loads a 128-row x 64-fiber unit as four FP32 boxes; eight
//     converter warps write it in the no-swizzle core-matrix layout with i
//     contiguous (the MN-major A operand), B arrives by bulk copy (or is
//     generated) in the same layout with l contiguous (MN-major B).
//
// A power step is therefore two passes over the tensor (W is written between
// them, 2 x L bytes per fiber per part) instead of the fused single pass of
// kernels_bf16x1.cu / kernels_tc.cu, whose tiles stop at I_n = 512 and L <= 64:
// an I_n x L FP32 accumulator of 1024 x 80 needs 320 KB of tensor memory, more
// than one SM has (256 KB), so here the rows are split over CTAs instead.
//
// Every mbarrier wait is bounded: on a timeout the kernel records kStatTimeout,
// lets the copies and products it issued finish (with the same bound), frees its
// tensor memory and returns.
#include <algorithm>
#include <climits>

#include "internal.h"
#include "tc.cuh"
#include "tma.cuh"

namespace tk {
namespace {

constexpr int kWWaitIters = 1 << 22;
constexpr size_t kWSmemMax = 227 * 1024;

__device__ __forceinline__ bool wait_bar(uint64_t* b, uint32_t parity, volatile int* flag) {
    for (int it = 0; it < kWWaitIters; ++it) {
        if (tc::mbar_try(b, parity)) return true;
        if ((it & 255) == 255 && *flag) return false;
    }
    return false;
}

__device__ __forceinline__ void fail(volatile int* flag, int* status) {
    *flag = 1;
    set_status(status, kStatTimeout);
}

__device__ __forceinline__ void drain(uint64_t* b, uint32_t parity) {
    for (int it = 0; it < kWWaitIters; ++it)
        if (tc::mbar_try(b, parity)) break;
}

__device__ __forceinline__ uint32_t bf2(float a, float b) {
    __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&p);
}

// Eight FP32 values -> bf16 (round to nearest), and for SPLIT the bf16 of the
// remainders x - bf16(x) (exact in FP32).
template <bool SPLIT>
__device__ __forceinline__ void cvt8(const float (&x)[8], uint4& hi, uint4& lo) {
    hi = make_uint4(bf2(x[0], x[1]), bf2(x[2], x[3]), bf2(x[4], x[5]), bf2(x[6], x[7]));
    if (SPLIT) {
        const uint32_t h[4] = {hi.x, hi.y, hi.z, hi.w};
        uint32_t l[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            l[k] = bf2(x[2 * k] - __uint_as_float(h[k] << 16), x[2 * k + 1] - __uint_as_float(h[k] & 0xFFFF0000u));
        lo = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// ------------------------------------------------------------------ M^T image
// K-major swizzled bf16 image of M^T (M(i, o) = Mp[i ld_i + o ld_k]) for the B
// operand of wide_ttm_kernel: unit u (values i = 64 u ..), part p (hi, lo), row o
// at u * ubytes + p * Np * 128 + (o / 8) 1024 + (o % 8) 128, its 16-byte group q
// (values 64 u + 8 q .. + 7) at group position q ^ (o % 8); zero beyond K_out, I.
template <bool SPLIT>
__global__ void image_kernel(const float* __restrict__ Mp, int I, int K_out, int64_t ld_i, int64_t ld_k, int Np,
                             int nu, unsigned char* __restrict__ img) {
    const int parts = SPLIT ? 2 : 1;
    const size_t ubytes = (size_t)parts * Np * 128;
    const int64_t total = (int64_t)nu * Np * 8;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(e / (Np * 8));
        const int rem = (int)(e - (int64_t)u * Np * 8);
        const int o = rem >> 3, q = rem & 7;
        float x[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int i = 64 * u + 8 * q + w;
            x[w] = (o < K_out && i < I) ? __ldg(Mp + (int64_t)i * ld_i + (int64_t)o * ld_k) : 0.f;
        }
        uint4 hi, lo;
        cvt8<SPLIT>(x, hi, lo);
        unsigned char* row = img + (size_t)u * ubytes + (o >> 3) * 1024 + (o & 7) * 128 + ((q ^ (o & 7)) << 4);
        *reinterpret_cast<uint4*>(row) = hi;
        if (SPLIT) *reinterpret_cast<uint4*>(row + (size_t)Np * 128) = lo;
    }
}

// B operand image of wide_power2_kernel from a column-major FP32 matrix Q (Tn x L):
// chunk c of 64 rows t at c Np 128 bytes of each part, element (l, jj = t % 64) at
// (jj / 8) (Np / 8) 128 + (l / 8) 128 + (jj % 8) 16 + (l % 8) 2; zero beyond Tn and L.
template <bool SPLIT>
__global__ void bimage_kernel(const float* __restrict__ Q, int64_t Tn, int L, int Np, int64_t chunks,
                              unsigned char* __restrict__ hi, unsigned char* __restrict__ lo) {
    const int ng = Np / 8;
    const int64_t total = chunks * 64 * ng;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int jj = (int)(e % 64);
        const int64_t rest = e / 64;
        const int lg = (int)(rest % ng);
        const int64_t ch = rest / ng;
        const int64_t t = ch * 64 + jj;
        float x[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int l = 8 * lg + w;
            x[w] = (t < Tn && l < L) ? __ldg(Q + t + Tn * (int64_t)l) : 0.f;
        }
        uint4 h, lw;
        cvt8<SPLIT>(x, h, lw);
        const size_t off = (size_t)ch * Np * 128 + (size_t)(jj >> 3) * ng * 128 + (size_t)lg * 128 + (jj & 7) * 16;
        *reinterpret_cast<uint4*>(hi + off) = h;
        if (SPLIT) *reinterpret_cast<uint4*>(lo + off) = lw;
    }
}

// ------------------------------------------------------------------ wide_ttm_kernel
constexpr int kAJB = 128;                  // fibers per tile
constexpr int kABox = kAJB * 128;          // FP32 box: 32 values i x 128 fibers = 16 KB
constexpr int kAUnit = 2 * kABox;          // FP32 unit: 64 values i
constexpr int kAHalf = kAJB * 128;         // one bf16 part of a unit: 64 values i x 128 fibers
constexpr int kAFMin = 3;                  // FP32 ring stages: as many as shared memory holds, 3 .. 6
constexpr int kAFMax = 6;
constexpr int kACStages = 2;
constexpr int kAUStages = 2;
constexpr int kAConv = 16;                 // converter warps 2 .. 17
constexpr int kAEpi = 4;                   // read-back warps 18 .. 21
constexpr int kAThreads = 64 + 32 * kAConv + 32 * kAEpi;
constexpr int kABars = 2 * kAFMax + 2 * kACStages + 2 * kAUStages + 5;
static_assert(kABars * 8 + 8 <= 256, "barrier area");

struct WideALayout {
    int nu = 0, Np = 0, parts = 1, fst = kAFMin;
    size_t ubytes = 0, c_off = 0, u_off = 0, bar_off = 0, bytes = 0;
    uint32_t tmem_cols = 0;
};

WideALayout wide_a_layout(int I, int K_out, bool split, int max_stages = kAFMax) {
    WideALayout t;
    t.nu = (I + 63) / 64;
    t.Np = (K_out + 15) / 16 * 16;
    t.parts = split ? 2 : 1;
    t.ubytes = (size_t)t.parts * t.Np * 128;
    // the FP32 ring takes what the converted ring, the image ring and the barriers leave
    // (each stage keeps 32 KB of the tensor in flight per SM)
    const size_t rest = (size_t)kACStages * t.parts * kAHalf + (size_t)kAUStages * t.ubytes + 256 + 1024;
    if (rest + (size_t)kAFMin * kAUnit <= kWSmemMax)
        t.fst = (int)std::max<size_t>(kAFMin, std::min<size_t>(std::min(kAFMax, max_stages), (kWSmemMax - rest) / kAUnit));
    t.c_off = (size_t)t.fst * kAUnit;
    t.u_off = t.c_off + (size_t)kACStages * t.parts * kAHalf;
    t.bar_off = t.u_off + (size_t)kAUStages * t.ubytes;
    t.bytes = t.bar_off + 256 + 1024;
    uint32_t c = 32;
    while (c < (uint32_t)(2 * t.Np)) c <<= 1;
    t.tmem_cols = c;
    return t;
}

// OUT 2: out[j + J o] (FP32, column-major J x K_out: the half-step product
// Y = C'^T X of the AMM sketch). OUT 0: out[j K_out + o] (FP32). OUT 1: W image for wide_power2_kernel's B
// operand: 64-fiber chunk c = j / 64 at c * Np * 128 bytes of each part's array,
// element (l, jj = j % 64) at (jj / 8) (Np / 8) 128 + (l / 8) 128 + (jj % 8) 16 +
// (l % 8) 2 (core matrices of 8 fibers x 8 columns, columns contiguous).
// STRIDED: fibers of modes 2..N (stride Lf, a multiple of 32) in the unfolding's
// order j = l + r Lf; a tile is 128 consecutive fibers, four groups of 32 that
// each lie in one slab r; TMA loads a group as 3-D boxes of 32 fibers x 32
// values (fibers contiguous) and the converters transpose them.
template <bool SPLIT, int OUT, bool STRIDED>
__global__ void __launch_bounds__(kAThreads, 1)
    wide_ttm_kernel(const __grid_constant__ CUtensorMap map, int I, int64_t J, const unsigned char* __restrict__ uimg,
                    int K_out, int Np, float* __restrict__ out, unsigned char* __restrict__ w_hi,
                    unsigned char* __restrict__ w_lo, int64_t tiles, int nu, int64_t lf, int* status, int fst) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024 - (tma::smem_addr(smem_raw) & 1023)) & 1023);
    constexpr int parts = SPLIT ? 2 : 1;
    const uint32_t ubytes = (uint32_t)(parts * Np * 128);
    unsigned char* F = smem;
    unsigned char* Cb = smem + (size_t)fst * kAUnit;
    unsigned char* Us = Cb + (size_t)kACStages * parts * kAHalf;
    uint64_t* bar = reinterpret_cast<uint64_t*>(Us + (size_t)kAUStages * ubytes);
    uint64_t* f_full = bar;
    uint64_t* f_empty = f_full + kAFMax;
    uint64_t* c_full = f_empty + kAFMax;
    uint64_t* c_empty = c_full + kACStages;
    uint64_t* u_full = c_empty + kACStages;
    uint64_t* u_empty = u_full + kAUStages;
    uint64_t* d_full = u_empty + kAUStages;
    uint64_t* d_empty = d_full + 2;
    uint64_t* done = d_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nloc = tiles > (int64_t)blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    uint32_t tcols = 32;
    while (tcols < (uint32_t)(2 * Np)) tcols <<= 1;

    if (tid == 0) {
        for (int k = 0; k < kABars; ++k) tc::mbar_init(&bar[k], 1);
        for (int k = 0; k < fst; ++k) tc::mbar_init(&f_empty[k], kAConv);
        for (int k = 0; k < kACStages; ++k) tc::mbar_init(&c_full[k], kAConv);
        for (int k = 0; k < 2; ++k) tc::mbar_init(&d_empty[k], kAEpi);
        *flag = 0;
        tma::fence_barrier_init();
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, tcols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // two producers: lane 0 streams the tensor as far ahead as the FP32 ring
        // allows; lane 1 streams the operand image (from L2) one unit ahead of each
        // product, so the short image ring never holds back the tensor's loads
        if (lane == 0) {
            int64_t g = 0;
            for (int64_t k = 0; k < nloc; ++k) {
                const int j0 = (int)((blockIdx.x + k * gridDim.x) * kAJB);
                bool ok = true;
                for (int u = 0; u < nu; ++u, ++g) {
                    const int fs = (int)(g % fst);
                    if (g >= fst && !wait_bar(&f_empty[fs], (uint32_t)((g / fst - 1) & 1), flag)) {
                        fail(flag, status);
                        ok = false;
                        break;
                    }
                    tma::expect_tx(&f_full[fs], (uint32_t)kAUnit);
                    unsigned char* dst = F + (size_t)fs * kAUnit;
                    // a box wholly beyond I_n (or, strided, beyond the last slab) loads zeros
                    if (STRIDED) {
#pragma unroll
                        for (int gq = 0; gq < 4; ++gq) {
                            const int64_t jg = (int64_t)j0 + 32 * gq;
                            const int r = (int)(jg / lf), l = (int)(jg - (int64_t)r * lf);
                            tma::load_3d(dst + (2 * gq) * 4096, &map, l, 64 * u, r, &f_full[fs]);
                            tma::load_3d(dst + (2 * gq + 1) * 4096, &map, l, 64 * u + 32, r, &f_full[fs]);
                        }
                    } else {
                        tma::load_2d(dst, &map, 64 * u, j0, &f_full[fs]);
                        tma::load_2d(dst + kABox, &map, 64 * u + 32, j0, &f_full[fs]);
                    }
                }
                if (!ok) break;
            }
            if (*flag) {
                // the copies issued so far land before the kernel returns
                const int64_t f0 = g > fst ? g - fst : 0;
                for (int64_t gg = f0; gg < g; ++gg) drain(&f_full[gg % fst], (uint32_t)((gg / fst) & 1));
            }
        } else if (lane == 1) {
            int64_t g = 0;
            for (int64_t k = 0; k < nloc; ++k) {
                bool ok = true;
                for (int u = 0; u < nu; ++u, ++g) {
                    const int us = (int)(g % kAUStages);
                    if (g >= kAUStages && !wait_bar(&u_empty[us], (uint32_t)((g / kAUStages - 1) & 1), flag)) {
                        fail(flag, status);
                        ok = false;
                        break;
                    }
                    tma::expect_tx(&u_full[us], ubytes);
                    tma::bulk_load(Us + (size_t)us * ubytes, uimg + (size_t)u * ubytes, ubytes, &u_full[us]);
                }
                if (!ok) break;
            }
            if (*flag) {
                const int64_t u0 = g > kAUStages ? g - kAUStages : 0;
                for (int64_t gg = u0; gg < g; ++gg) drain(&u_full[gg % kAUStages], (uint32_t)((gg / kAUStages) & 1));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id = tc::idesc_bf16(128, Np, false, false);
            const uint64_t c_desc = tc::desc_sw128(tc::smem_u32(Cb), 16, 1024);
            const uint64_t u_desc = tc::desc_sw128(tc::smem_u32(Us), 16, 1024);
            const uint64_t lo_step = (uint64_t)(kAHalf >> 4), ulo_step = (uint64_t)((Np * 128) >> 4);
            bool ok = true;
            int64_t g = 0;
            for (int64_t k = 0; k < nloc && ok; ++k) {
                const int b = (int)(k & 1);
                if (k >= 2 && !wait_bar(&d_empty[b], (uint32_t)(((k >> 1) - 1) & 1), flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d = tmem + (uint32_t)(b * Np);
                for (int u = 0; u < nu; ++u, ++g) {
                    const int cs = (int)(g % kACStages), us = (int)(g % kAUStages);
                    if (!wait_bar(&c_full[cs], (uint32_t)((g / kACStages) & 1), flag) ||
                        !wait_bar(&u_full[us], (uint32_t)((g / kAUStages) & 1), flag)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint64_t ahi = c_desc + (uint64_t)((cs * parts * kAHalf) >> 4);
                    const uint64_t bhi = u_desc + (uint64_t)((us * ubytes) >> 4);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t s2 = (uint64_t)(ks * 2);
                        tc::mma_bf16(d, ahi + s2, bhi + s2, id, u > 0 || ks > 0);
                        if (SPLIT) {
                            tc::mma_bf16(d, ahi + lo_step + s2, bhi + s2, id, true);
                            tc::mma_bf16(d, ahi + s2, bhi + ulo_step + s2, id, true);
                        }
                    }
                    tc::commit(&c_empty[cs]);
                    tc::commit(&u_empty[us]);
                }
                if (!ok) break;
                tc::commit(&d_full[b]);
            }
            tc::commit(done);
            if (!ok) {
                fail(flag, status);
                drain(done, 0);
            }
        }
    } else if (warp < 2 + kAConv) {
        // conversion: task t = (fiber j, group p of 8 values i of the unit), two
        // 16-byte pieces of FP32 box p / 4 in, one 16-byte piece per bf16 part out
        const int ct = tid - 64;
        bool ok = true;
        int64_t g = 0;
        constexpr int kTasks = (kAJB * 8) / (kAConv * 32);
        for (int64_t k = 0; k < nloc && ok; ++k) {
            for (int u = 0; u < nu; ++u, ++g) {
                const int fs = (int)(g % fst), cs = (int)(g % kACStages);
                if (!wait_bar(&f_full[fs], (uint32_t)((g / fst) & 1), flag)) {
                    ok = false;
                    break;
                }
                const unsigned char* src = F + (size_t)fs * kAUnit;
                uint4 hi[kTasks], lo[kTasks];
#pragma unroll
                for (int r = 0; r < kTasks; ++r) {
                    const int t = ct + kAConv * 32 * r;
                    float x[8];
                    if (STRIDED) {
                        // task: fiber f of the tile (lanes: 32 consecutive fibers), values
                        // 8 p .. 8 p + 7 of the unit, read down rows of box (f / 32, p / 4)
                        const int f = t & 127, p = t >> 7;
                        const unsigned char* box = src + (2 * (f >> 5) + (p >> 2)) * 4096;
                        const int c = (f & 31) >> 2, e = (f & 3) * 4;
#pragma unroll
                        for (int w = 0; w < 8; ++w) {
                            const int row = (p & 3) * 8 + w;
                            x[w] = *reinterpret_cast<const float*>(box + row * 128 + ((c ^ (row & 7)) << 4) + e);
                        }
                    } else {
                        const int j = t >> 3, p = t & 7;
                        const int q0 = (p & 3) * 2;
                        const unsigned char* row = src + (p >> 2) * kABox + j * 128;
                        const float4 a = *reinterpret_cast<const float4*>(row + ((q0 ^ (j & 7)) << 4));
                        const float4 c = *reinterpret_cast<const float4*>(row + (((q0 + 1) ^ (j & 7)) << 4));
                        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = c.x; x[5] = c.y; x[6] = c.z; x[7] = c.w;
                    }
                    cvt8<SPLIT>(x, hi[r], lo[r]);
                }
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&f_empty[fs]);
                if (g >= kACStages && !wait_bar(&c_empty[cs], (uint32_t)((g / kACStages - 1) & 1), flag)) {
                    ok = false;
                    break;
                }
                unsigned char* dhi = Cb + (size_t)cs * parts * kAHalf;
#pragma unroll
                for (int r = 0; r < kTasks; ++r) {
                    const int t = ct + kAConv * 32 * r;
                    const int j = STRIDED ? (t & 127) : (t >> 3), p = STRIDED ? (t >> 7) : (t & 7);
                    const int off = j * 128 + ((p ^ (j & 7)) << 4);
                    *reinterpret_cast<uint4*>(dhi + off) = hi[r];
                    if (SPLIT) *reinterpret_cast<uint4*>(dhi + kAHalf + off) = lo[r];
                }
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&c_full[cs]);
            }
        }
        if (!ok) fail(flag, status);
    } else {
        // read-back: warp w reaches lanes 32 (w % 4) .. + 31 = fibers of the tile
        const int quarter = warp & 3;
        for (int64_t k = 0; k < nloc; ++k) {
            const int b = (int)(k & 1);
            if (!wait_bar(&d_full[b], (uint32_t)((k >> 1) & 1), flag)) {
                if (!*flag) fail(flag, status);
                break;
            }
            tc::fence_after_sync();
            const int64_t j = (blockIdx.x + k * gridDim.x) * kAJB + quarter * 32 + lane;
            const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * Np);
            // the W image covers whole 64-fiber chunks: fibers J .. of the last one
            // are written too (as zeros: their tensor columns load as zeros)
            const int64_t jend = OUT == 1 ? (J + 63) / 64 * 64 : J;
            for (int c0 = 0; c0 < Np; c0 += 16) {
                uint32_t r[16];
                tc::tmem_ld16(ta + (uint32_t)c0, r);
                if (j >= jend) continue;
                if (OUT == 2) {
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        if (c0 + c < K_out) out[j + J * (int64_t)(c0 + c)] = __uint_as_float(r[c]);
                } else if (OUT == 0 && STRIDED) {
                    // out(l, o, r) = out[l + o Lf + r Lf K_out]: lanes write consecutive l
                    const int64_t rr = j / lf, l = j - rr * lf;
                    float* o = out + l + rr * lf * K_out;
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        if (c0 + c < K_out) o[(int64_t)(c0 + c) * lf] = __uint_as_float(r[c]);
                } else if (OUT == 0) {
                    float* o = out + j * K_out;
                    if ((K_out & 3) == 0 && c0 + 16 <= K_out) {
#pragma unroll
                        for (int c = 0; c < 16; c += 4)
                            *reinterpret_cast<float4*>(o + c0 + c) =
                                make_float4(__uint_as_float(r[c]), __uint_as_float(r[c + 1]),
                                            __uint_as_float(r[c + 2]), __uint_as_float(r[c + 3]));
                    } else {
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            if (c0 + c < K_out) o[c0 + c] = __uint_as_float(r[c]);
                    }
                } else {
                    // columns l >= K_out of the accumulator are zero (M^T's image is)
                    const int64_t ch = j >> 6;
                    const int jj = (int)(j & 63);
                    const size_t base = (size_t)ch * Np * 128 + (size_t)(jj >> 3) * (Np / 8) * 128 + (jj & 7) * 16;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float x[8];
#pragma unroll
                        for (int w = 0; w < 8; ++w) x[w] = __uint_as_float(r[8 * h + w]);
                        uint4 hi, lo;
                        cvt8<SPLIT>(x, hi, lo);
                        const size_t off = base + (size_t)((c0 + 8 * h) >> 3) * 128;
                        *reinterpret_cast<uint4*>(w_hi + off) = hi;
                        if (SPLIT) *reinterpret_cast<uint4*>(w_lo + off) = lo;
                    }
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&d_empty[b]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, tcols);
}

// ------------------------------------------------------------------ wide_power2_kernel
constexpr int kBJB = 64;                   // fibers per chunk (K of the product)
constexpr int kBBox = kBJB * 128;          // FP32 box: 32 values i x 64 fibers = 8 KB
constexpr int kBUnit = 4 * kBBox;          // FP32 unit: 128 rows i x 64 fibers = 32 KB
constexpr int kBHalf = 128 * kBJB * 2;     // one bf16 part of a unit: 16 KB
constexpr int kBFMin = 3;                  // FP32 ring stages: as many as shared memory holds, 3 .. 6
constexpr int kBFMax = 6;
constexpr int kBCStages = 2;
constexpr int kBWStages = 2;
constexpr int kBConv = 8;                  // converter (and generator, read-back) warps 2 .. 9
constexpr int kBThreads = 64 + 32 * kBConv;
constexpr int kBMaxBlocks = 4;             // 128-row blocks per CTA
constexpr int kBBars = 2 * kBFMax + 2 * kBCStages + 2 * kBWStages + 1;
static_assert(kBBars * 8 + 8 <= 256, "barrier area");

struct WideBLayout {
    int Np = 0, parts = 1, nb = 0, groups = 0, fst = kBFMin;
    size_t wbytes = 0, c_off = 0, w_off = 0, bar_off = 0, bytes = 0;
};

WideBLayout wide_b_layout(int I, int L, bool split, int max_stages = kBFMax) {
    WideBLayout t;
    t.Np = (L + 15) / 16 * 16;
    t.parts = split ? 2 : 1;
    const int blocks = (I + 127) / 128;
    t.nb = std::min(kBMaxBlocks, std::min(blocks, 512 / t.Np));
    t.groups = (blocks + t.nb - 1) / t.nb;
    t.wbytes = (size_t)t.parts * t.Np * 128;
    const size_t rest = (size_t)kBCStages * t.parts * kBHalf + (size_t)kBWStages * t.wbytes + 256 + 1024;
    if (rest + (size_t)kBFMin * kBUnit <= kWSmemMax)
        t.fst = (int)std::max<size_t>(kBFMin, std::min<size_t>(std::min(kBFMax, max_stages), (kWSmemMax - rest) / kBUnit));
    t.c_off = (size_t)t.fst * kBUnit;
    t.w_off = t.c_off + (size_t)kBCStages * t.parts * kBHalf;
    t.bar_off = t.w_off + (size_t)kBWStages * t.wbytes;
    t.bytes = t.bar_off + 256 + 1024;
    return t;
}

// partial[r (I L) + l I + i] = sum over the CTA's chunks of A_(n)[i, j] B[j, l]
// for the rows of its group; r = blockIdx.x / groups.
// STRIDED: a 64-fiber chunk is two groups of 32 fibers, each in one slab,
// loaded as 3-D boxes of 32 fibers x 32 rows; the A operand is then K-major
// (fibers contiguous in each row) in the no-swizzle core-matrix layout.
template <bool SPLIT, bool RANGE, bool STRIDED>
__global__ void __launch_bounds__(kBThreads, 1)
    wide_power2_kernel(const __grid_constant__ CUtensorMap map, int I, int64_t J, int L, int Np,
                       const unsigned char* __restrict__ w_hi, const unsigned char* __restrict__ w_lo, uint64_t seed,
                       uint32_t stream_id, float* __restrict__ partial, int groups, int nb, int64_t chunks,
                       int64_t lf, int* status, int fst) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024 - (tma::smem_addr(smem_raw) & 1023)) & 1023);
    constexpr int parts = SPLIT ? 2 : 1;
    const uint32_t wbytes = (uint32_t)(parts * Np * 128);
    unsigned char* F = smem;
    unsigned char* Cb = smem + (size_t)fst * kBUnit;
    unsigned char* Ws = Cb + (size_t)kBCStages * parts * kBHalf;
    uint64_t* bar = reinterpret_cast<uint64_t*>(Ws + (size_t)kBWStages * wbytes);
    uint64_t* f_full = bar;
    uint64_t* f_empty = f_full + kBFMax;
    uint64_t* c_full = f_empty + kBFMax;
    uint64_t* c_empty = c_full + kBCStages;
    uint64_t* w_full = c_empty + kBCStages;
    uint64_t* w_empty = w_full + kBWStages;
    uint64_t* done = w_empty + kBWStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = (int)(blockIdx.x % groups);
    const int64_t r = blockIdx.x / groups, R = gridDim.x / groups;
    const int64_t nloc = chunks > r ? (chunks - 1 - r) / R + 1 : 0;
    const int blocks_total = (I + 127) / 128;
    const int nbg = min(nb, blocks_total - grp * nb);     // row blocks of this CTA
    const int row0 = grp * nb * 128;

    if (tid == 0) {
        for (int k = 0; k < kBBars; ++k) tc::mbar_init(&bar[k], 1);
        for (int k = 0; k < fst; ++k) tc::mbar_init(&f_empty[k], kBConv);
        for (int k = 0; k < kBCStages; ++k) tc::mbar_init(&c_full[k], kBConv);
        if (RANGE)
            for (int k = 0; k < kBWStages; ++k) tc::mbar_init(&w_full[k], kBConv);
        *flag = 0;
        tma::fence_barrier_init();
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int64_t g = 0, wc = 0;
            bool ok = true;
            for (int64_t kk = 0; kk < nloc && ok; ++kk) {
                const int64_t ch = r + kk * R;
                const int j0 = (int)(ch * kBJB);
                if (!RANGE) {
                    const int ws = (int)(wc % kBWStages);
                    if (wc >= kBWStages && !wait_bar(&w_empty[ws], (uint32_t)((wc / kBWStages - 1) & 1), flag)) {
                        fail(flag, status);
                        ok = false;
                        break;
                    }
                    const uint32_t pb = (uint32_t)(Np * 128);
                    tma::expect_tx(&w_full[ws], wbytes);
                    tma::bulk_load(Ws + (size_t)ws * wbytes, w_hi + (size_t)ch * pb, pb, &w_full[ws]);
                    if (SPLIT) tma::bulk_load(Ws + (size_t)ws * wbytes + pb, w_lo + (size_t)ch * pb, pb, &w_full[ws]);
                    ++wc;
                }
                for (int b = 0; b < nbg; ++b, ++g) {
                    const int fs = (int)(g % fst);
                    if (g >= fst && !wait_bar(&f_empty[fs], (uint32_t)((g / fst - 1) & 1), flag)) {
                        fail(flag, status);
                        ok = false;
                        break;
                    }
                    tma::expect_tx(&f_full[fs], (uint32_t)kBUnit);
                    unsigned char* dst = F + (size_t)fs * kBUnit;
                    const int i0 = row0 + b * 128;
                    if (STRIDED) {
#pragma unroll
                        for (int gq = 0; gq < 2; ++gq) {
                            const int64_t jg = (int64_t)j0 + 32 * gq;
                            const int r = (int)(jg / lf), l = (int)(jg - (int64_t)r * lf);
#pragma unroll
                            for (int s = 0; s < 4; ++s)
                                tma::load_3d(dst + (4 * gq + s) * 4096, &map, l, i0 + 32 * s, r, &f_full[fs]);
                        }
                    } else {
#pragma unroll
                        for (int s = 0; s < 4; ++s) tma::load_2d(dst + s * kBBox, &map, i0 + 32 * s, j0, &f_full[fs]);
                    }
                }
            }
            if (*flag) {
                const int64_t f0 = g > fst ? g - fst : 0;
                for (int64_t gg = f0; gg < g; ++gg) drain(&f_full[gg % fst], (uint32_t)((gg / fst) & 1));
                if (!RANGE) {
                    const int64_t w0 = wc > kBWStages ? wc - kBWStages : 0;
                    for (int64_t gg = w0; gg < wc; ++gg)
                        drain(&w_full[gg % kBWStages], (uint32_t)((gg / kBWStages) & 1));
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id = tc::idesc_bf16(128, Np, !STRIDED, true);
            // no-swizzle core matrices, LBO the K step, SBO the M/N step: A (rows i x 64
            // fibers) MN-major 2048 / 128 (contiguous), K-major 128 / 1024 (strided);
            // B (64 fibers x Np columns) MN-major, Np 16 / 128
            const uint64_t a_desc = STRIDED ? tc::desc(tc::smem_u32(Cb), 128, 1024) : tc::desc(tc::smem_u32(Cb), 2048, 128);
            const uint32_t a_kstep = STRIDED ? 2 * 128 : 2 * 2048;            // bytes per 16 fibers
            const uint64_t b_desc = tc::desc(tc::smem_u32(Ws), (uint32_t)(Np * 16), 128);
            const uint64_t alo = (uint64_t)(kBHalf >> 4), blo = (uint64_t)((Np * 128) >> 4);
            bool ok = true;
            int64_t g = 0;
            for (int64_t kk = 0; kk < nloc && ok; ++kk) {
                const int ws = (int)(kk % kBWStages);
                if (!wait_bar(&w_full[ws], (uint32_t)((kk / kBWStages) & 1), flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                for (int b = 0; b < nbg; ++b, ++g) {
                    const int cs = (int)(g % kBCStages);
                    if (!wait_bar(&c_full[cs], (uint32_t)((g / kBCStages) & 1), flag)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t d = tmem + (uint32_t)(b * Np);
                    const uint64_t a0 = a_desc + (uint64_t)((cs * parts * kBHalf) >> 4);
                    const uint64_t b0 = b_desc + (uint64_t)((ws * wbytes) >> 4);
#pragma unroll
                    for (int ks = 0; ks < kBJB / 16; ++ks) {
                        const uint64_t sa = (uint64_t)((ks * a_kstep) >> 4), sb = (uint64_t)((ks * 2 * Np * 16) >> 4);
                        tc::mma_bf16(d, a0 + sa, b0 + sb, id, kk > 0 || ks > 0);
                        if (SPLIT) {
                            tc::mma_bf16(d, a0 + alo + sa, b0 + sb, id, true);
                            tc::mma_bf16(d, a0 + sa, b0 + blo + sb, id, true);
                        }
                    }
                    tc::commit(&c_empty[cs]);
                }
                if (!ok) break;
                tc::commit(&w_empty[ws]);
            }
            tc::commit(done);
            if (!ok) {
                fail(flag, status);
                drain(done, 0);
            }
        }
    } else {
        const int ct = tid - 64;
        bool ok = true;
        int64_t g = 0;
        constexpr int kTasks = (128 / 8) * kBJB / (kBConv * 32);   // 4
        for (int64_t kk = 0; kk < nloc && ok; ++kk) {
            const int64_t ch = r + kk * R;
            if (RANGE) {
                // Omega rows j of the chunk (Gaussian element j L + l of the stream),
                // l contiguous in 16-byte groups of 8; zero for l >= L and j >= J
                const int ws = (int)(kk % kBWStages);
                if (kk >= kBWStages && !wait_bar(&w_empty[ws], (uint32_t)((kk / kBWStages - 1) & 1), flag)) {
                    ok = false;
                    break;
                }
                unsigned char* dst = Ws + (size_t)ws * wbytes;
                const int ng = Np / 8;
                for (int t = ct; t < kBJB * ng; t += kBConv * 32) {
                    const int jj = t % kBJB, lg = t / kBJB;
                    const int64_t j = ch * kBJB + jj;
                    float x[8];
#pragma unroll
                    for (int w = 0; w < 8; ++w) {
                        const int l = 8 * lg + w;
                        x[w] = (j < J && l < L) ? gaussian_at<float>(seed, stream_id, (uint64_t)(j * L + l)) : 0.f;
                    }
                    uint4 hi, lo;
                    cvt8<SPLIT>(x, hi, lo);
                    const size_t off = (size_t)(jj >> 3) * ng * 128 + (size_t)lg * 128 + (jj & 7) * 16;
                    *reinterpret_cast<uint4*>(dst + off) = hi;
                    if (SPLIT) *reinterpret_cast<uint4*>(dst + Np * 128 + off) = lo;
                }
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&w_full[ws]);
            }
            for (int b = 0; b < nbg; ++b, ++g) {
                const int fs = (int)(g % fst), cs = (int)(g % kBCStages);
                if (!wait_bar(&f_full[fs], (uint32_t)((g / fst) & 1), flag)) {
                    ok = false;
                    break;
                }
                // contiguous, task t: fiber jj = 8 (t / 128) + t % 8, rows i = 8 ((t / 8) % 16) .. + 7;
                // strided, task t: row i = t % 8 + 8 (t / 64), fibers 8 q .. 8 q + 7, q = (t / 8) % 8
                const unsigned char* src = F + (size_t)fs * kBUnit;
                uint4 hi[kTasks], lo[kTasks];
#pragma unroll
                for (int q = 0; q < kTasks; ++q) {
                    const int t = ct + kBConv * 32 * q;
                    float4 a, c;
                    if (STRIDED) {
                        const int i = (t & 7) + 8 * (t >> 6), g8 = (t >> 3) & 7;
                        const unsigned char* row = src + (4 * (g8 >> 2) + (i >> 5)) * 4096 + (i & 31) * 128;
                        const int c0 = (g8 & 3) * 2;
                        a = *reinterpret_cast<const float4*>(row + ((c0 ^ (i & 7)) << 4));
                        c = *reinterpret_cast<const float4*>(row + (((c0 + 1) ^ (i & 7)) << 4));
                    } else {
                        const int jlo = t & 7, ig = (t >> 3) & 15, jhi = t >> 7;
                        const int jj = jhi * 8 + jlo;
                        const int c0 = (ig & 3) * 2;
                        const unsigned char* row = src + (ig >> 2) * kBBox + jj * 128;
                        a = *reinterpret_cast<const float4*>(row + ((c0 ^ (jj & 7)) << 4));
                        c = *reinterpret_cast<const float4*>(row + (((c0 + 1) ^ (jj & 7)) << 4));
                    }
                    const float x[8] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
                    cvt8<SPLIT>(x, hi[q], lo[q]);
                }
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&f_empty[fs]);
                if (g >= kBCStages && !wait_bar(&c_empty[cs], (uint32_t)((g / kBCStages - 1) & 1), flag)) {
                    ok = false;
                    break;
                }
                unsigned char* dst = Cb + (size_t)cs * parts * kBHalf;
#pragma unroll
                for (int q = 0; q < kTasks; ++q) {
                    const int t = ct + kBConv * 32 * q;
                    // strided: core matrix (i / 8, fibers g8) at (i / 8) 1024 + g8 128, row i % 8
                    const int off = STRIDED ? ((t >> 6) * 1024 + ((t >> 3) & 7) * 128 + (t & 7) * 16)
                                            : ((t >> 7) * 2048 + ((t >> 3) & 15) * 128 + (t & 7) * 16);
                    *reinterpret_cast<uint4*>(dst + off) = hi[q];
                    if (SPLIT) *reinterpret_cast<uint4*>(dst + kBHalf + off) = lo[q];
                }
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&c_full[cs]);
            }
        }
        if (!ok) fail(flag, status);
        // the CTA's partial: block b row i on lane i % 128, columns l
        if (ok && wait_bar(done, 0, flag) && !*flag) {
            tc::fence_after_sync();
            const int quarter = warp & 3, half = (warp - 2) >> 2;
            float* out = partial + r * ((int64_t)I * L);
            for (int b = half; b < nbg; b += 2) {
                const int i = row0 + b * 128 + quarter * 32 + lane;
                const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * Np);
                for (int c0 = 0; c0 < Np; c0 += 16) {
                    uint32_t v[16];
                    tc::tmem_ld16(ta + (uint32_t)c0, v);
                    if (i < I)
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            if (c0 + c < L) out[(int64_t)(c0 + c) * I + i] = __uint_as_float(v[c]);
                }
            }
        } else if (!*flag) {
            fail(flag, status);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// Tensor map of the fibers: contiguous (I, J) with boxes of 32 values x `box_fibers`;
// strided (Lf, I, Rt) with boxes of 32 fibers x 32 values x 1 slab.
bool make_fiber_map(CUtensorMap* map, const float* A, const ModeView& v, uint32_t box_fibers) {
    if (v.lf == 1) {
        const uint64_t dims[2] = {(uint64_t)v.i, (uint64_t)v.fibers()};
        const uint64_t strides[1] = {(uint64_t)v.i * sizeof(float)};
        const uint32_t box[2] = {32, box_fibers};
        return tma::make_map_f32(map, A, 2, dims, strides, box, true);
    }
    const uint64_t dims[3] = {(uint64_t)v.lf, (uint64_t)v.i, (uint64_t)v.rt};
    const uint64_t strides[2] = {(uint64_t)v.lf * sizeof(float), (uint64_t)v.lf * v.i * sizeof(float)};
    const uint32_t box[3] = {32, 32, 1};
    return tma::make_map_f32(map, A, 3, dims, strides, box, true);
}

int grid_for(int64_t units, int num_sms) {
    int g = (int)(units < num_sms ? units : num_sms);
    return g < 1 ? 1 : g;
}

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// contiguous fibers (I_n % 4 == 0 for the row stride), or strided ones whose
// stride is a multiple of 32 (a 32-fiber group never crosses a slab)
bool layout_ok(const ModeView& v) {
    if (v.lf == 1) return v.i % 4 == 0;
    return v.lf % 32 == 0 && v.lf <= (int64_t)INT_MAX && v.rt <= (int64_t)INT_MAX;
}

// ------------------------------------------------------------------ gram_wide_kernel
// Strategy B (remark after Algorithm 1): G = A_(n) A_(n)^T (I_n x I_n, I_n <= 128)
// in one streaming pass, partial[r I^2 + i' I + i] = sum over the CTA's 64-fiber
// chunks of A_(n)[i, j] A_(n)[i', j]. The units are loaded and converted exactly
// as in wide_power2_kernel (one 128-row block, rows >= I_n load as zeros), and
// the converted unit is both operands of D = T T^T: A = rows i x fibers and
// B = fibers x columns i', the same core matrices read with the same strides
// (i contiguous for contiguous fibers: MN-major A and B; fibers contiguous for
// strided ones: K-major A and B). N = I_n padded to 16; split: hi.hi + lo.hi +
// hi.lo.
constexpr int kGBars = 2 * kBFMax + 2 * kBCStages + 1;
static_assert(kGBars * 8 + 8 <= 256, "barrier area");

struct GramLayout {
    int Np = 0, parts = 1, fst = kBFMin;
    size_t c_off = 0, bar_off = 0, bytes = 0;
};

GramLayout gram_layout(int I, bool split, int max_stages = kBFMax) {
    GramLayout t;
    t.Np = (I + 15) / 16 * 16;
    t.parts = split ? 2 : 1;
    const size_t rest = (size_t)kBCStages * t.parts * kBHalf + 256 + 1024;
    if (rest + (size_t)kBFMin * kBUnit <= kWSmemMax)
        t.fst = (int)std::max<size_t>(kBFMin, std::min<size_t>(std::min(kBFMax, max_stages), (kWSmemMax - rest) / kBUnit));
    t.c_off = (size_t)t.fst * kBUnit;
    t.bar_off = t.c_off + (size_t)kBCStages * t.parts * kBHalf;
    t.bytes = t.bar_off + 256 + 1024;
    return t;
}

template <bool SPLIT, bool STRIDED>
__global__ void __launch_bounds__(kBThreads, 1)
    gram_wide_kernel(const __grid_constant__ CUtensorMap map, int I, int64_t J, int Np, float* __restrict__ partial,
                     int64_t chunks, int64_t lf, int* status, int fst) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024 - (tma::smem_addr(smem_raw) & 1023)) & 1023);
    constexpr int parts = SPLIT ? 2 : 1;
    unsigned char* F = smem;
    unsigned char* Cb = smem + (size_t)fst * kBUnit;
    uint64_t* bar = reinterpret_cast<uint64_t*>(Cb + (size_t)kBCStages * parts * kBHalf);
    uint64_t* f_full = bar;
    uint64_t* f_empty = f_full + kBFMax;
    uint64_t* c_full = f_empty + kBFMax;
    uint64_t* c_empty = c_full + kBCStages;
    uint64_t* done = c_empty + kBCStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r = blockIdx.x, R = gridDim.x;
    const int64_t nloc = chunks > r ? (chunks - 1 - r) / R + 1 : 0;

    if (tid == 0) {
        for (int k = 0; k < kGBars; ++k) tc::mbar_init(&bar[k], 1);
        for (int k = 0; k < fst; ++k) tc::mbar_init(&f_empty[k], kBConv);
        for (int k = 0; k < kBCStages; ++k) tc::mbar_init(&c_full[k], kBConv);
        *flag = 0;
        tma::fence_barrier_init();
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, 128);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int64_t g = 0;
            for (int64_t kk = 0; kk < nloc; ++kk, ++g) {
                const int64_t ch = r + kk * R;
                const int j0 = (int)(ch * kBJB);
                const int fs = (int)(g % fst);
                if (g >= fst && !wait_bar(&f_empty[fs], (uint32_t)((g / fst - 1) & 1), flag)) {
                    fail(flag, status);
                    break;
                }
                tma::expect_tx(&f_full[fs], (uint32_t)kBUnit);
                unsigned char* dst = F + (size_t)fs * kBUnit;
                if (STRIDED) {
#pragma unroll
                    for (int gq = 0; gq < 2; ++gq) {
                        const int64_t jg = (int64_t)j0 + 32 * gq;
                        const int rr = (int)(jg / lf), l = (int)(jg - (int64_t)rr * lf);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            tma::load_3d(dst + (4 * gq + q) * 4096, &map, l, 32 * q, rr, &f_full[fs]);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) tma::load_2d(dst + q * kBBox, &map, 32 * q, j0, &f_full[fs]);
                }
            }
            if (*flag) {
                const int64_t f0 = g > fst ? g - fst : 0;
                for (int64_t gg = f0; gg < g; ++gg) drain(&f_full[gg % fst], (uint32_t)((gg / fst) & 1));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id = tc::idesc_bf16(128, Np, !STRIDED, !STRIDED);
            // the converted unit read as A (rows i x 64 fibers) and as B (64 fibers x columns i'):
            // no-swizzle core matrices, LBO the fiber step, SBO the row step; MN-major 2048 / 128
            // (contiguous), K-major 128 / 1024 (strided), the same for both operands
            const uint64_t desc0 = STRIDED ? tc::desc(tc::smem_u32(Cb), 128, 1024) : tc::desc(tc::smem_u32(Cb), 2048, 128);
            const uint32_t kstep = STRIDED ? 2 * 128 : 2 * 2048;                 // bytes per 16 fibers
            const uint64_t lo = (uint64_t)(kBHalf >> 4);
            bool ok = true;
            for (int64_t kk = 0; kk < nloc; ++kk) {
                const int cs = (int)(kk % kBCStages);
                if (!wait_bar(&c_full[cs], (uint32_t)((kk / kBCStages) & 1), flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint64_t a0 = desc0 + (uint64_t)((cs * parts * kBHalf) >> 4);
#pragma unroll
                for (int ks = 0; ks < kBJB / 16; ++ks) {
                    const uint64_t sk = (uint64_t)((ks * kstep) >> 4);
                    tc::mma_bf16(tmem, a0 + sk, a0 + sk, id, kk > 0 || ks > 0);
                    if (SPLIT) {
                        tc::mma_bf16(tmem, a0 + lo + sk, a0 + sk, id, true);
                        tc::mma_bf16(tmem, a0 + sk, a0 + lo + sk, id, true);
                    }
                }
                tc::commit(&c_empty[cs]);
            }
            tc::commit(done);
            if (!ok) {
                fail(flag, status);
                drain(done, 0);
            }
        }
    } else {
        const int ct = tid - 64;
        bool ok = true;
        constexpr int kTasks = (128 / 8) * kBJB / (kBConv * 32);   // 4
        for (int64_t kk = 0; kk < nloc && ok; ++kk) {
            const int fs = (int)(kk % fst), cs = (int)(kk % kBCStages);
            if (!wait_bar(&f_full[fs], (uint32_t)((kk / fst) & 1), flag)) {
                ok = false;
                break;
            }
            const unsigned char* src = F + (size_t)fs * kBUnit;
            uint4 hi[kTasks], lw[kTasks];
#pragma unroll
            for (int q = 0; q < kTasks; ++q) {
                const int t = ct + kBConv * 32 * q;
                float4 a, c;
                if (STRIDED) {
                    const int i = (t & 7) + 8 * (t >> 6), g8 = (t >> 3) & 7;
                    const unsigned char* row = src + (4 * (g8 >> 2) + (i >> 5)) * 4096 + (i & 31) * 128;
                    const int c0 = (g8 & 3) * 2;
                    a = *reinterpret_cast<const float4*>(row + ((c0 ^ (i & 7)) << 4));
                    c = *reinterpret_cast<const float4*>(row + (((c0 + 1) ^ (i & 7)) << 4));
                } else {
                    const int jlo = t & 7, ig = (t >> 3) & 15, jhi = t >> 7;
                    const int jj = jhi * 8 + jlo;
                    const int c0 = (ig & 3) * 2;
                    const unsigned char* row = src + (ig >> 2) * kBBox + jj * 128;
                    a = *reinterpret_cast<const float4*>(row + ((c0 ^ (jj & 7)) << 4));
                    c = *reinterpret_cast<const float4*>(row + (((c0 + 1) ^ (jj & 7)) << 4));
                }
                const float x[8] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
                cvt8<SPLIT>(x, hi[q], lw[q]);
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&f_empty[fs]);
            if (kk >= kBCStages && !wait_bar(&c_empty[cs], (uint32_t)((kk / kBCStages - 1) & 1), flag)) {
                ok = false;
                break;
            }
            unsigned char* dst = Cb + (size_t)cs * parts * kBHalf;
#pragma unroll
            for (int q = 0; q < kTasks; ++q) {
                const int t = ct + kBConv * 32 * q;
                const int off = STRIDED ? ((t >> 6) * 1024 + ((t >> 3) & 7) * 128 + (t & 7) * 16)
                                        : ((t >> 7) * 2048 + ((t >> 3) & 15) * 128 + (t & 7) * 16);
                *reinterpret_cast<uint4*>(dst + off) = hi[q];
                if (SPLIT) *reinterpret_cast<uint4*>(dst + kBHalf + off) = lw[q];
            }
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&c_full[cs]);
        }
        if (!ok) fail(flag, status);
        // the CTA's partial: row i on lane i, columns i'; the first four converter warps
        const bool ready = ok && warp < 6 && wait_bar(done, 0, flag);
        if (ok && warp < 6 && !ready && !*flag) fail(flag, status);
        if (ready && !*flag) {
            tc::fence_after_sync();
            const int quarter = warp & 3;
            float* out = partial + r * ((int64_t)I * I);
            const int i = quarter * 32 + lane;
            const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16);
            for (int c0 = 0; c0 < Np; c0 += 16) {
                uint32_t v[16];
                tc::tmem_ld16(ta + (uint32_t)c0, v);
                if (i < I)
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        if (c0 + c < I) out[(int64_t)(c0 + c) * I + i] = __uint_as_float(v[c]);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, 128);
}

// A wait that nothing completes: one CTA takes tensor memory as the kernels
// above do, initialises an mbarrier that no thread and no copy arrives at,
// waits for it with the bound `iters`, records the timeout as every kernel here
// does, frees its tensor memory and returns. No copy or product is in flight,
// so nothing needs draining: it checks that a bounded wait ends, that its
// status reaches the host and that the context stays usable.
__global__ void __launch_bounds__(64) wait_timeout_kernel(int iters, int* status) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int flag;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        flag = 0;
        tma::fence_barrier_init();
    }
    if (warp == 1) tc::tmem_alloc(&tmem_slot, 32);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
        bool ok = false;
        for (int it = 0; it < iters && !ok; ++it) ok = tc::mbar_try(&bar, 0);
        if (!ok) fail(&flag, status);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem_slot, 32);
}

}  // namespace

bool wide_ttm_supported(const ModeView& v, int64_t K_out) {
    return layout_ok(v) && v.i >= 1 && v.i <= 16384 && K_out >= 1 && K_out <= 128 &&
           v.fibers() <= (int64_t)INT_MAX - 256 && wide_a_layout((int)v.i, (int)K_out, true).bytes <= kWSmemMax;
}

bool wide_supported(const ModeView& v, int64_t cols) {
    return wide_ttm_supported(v, cols) && wide_b_layout((int)v.i, (int)cols, true).bytes <= kWSmemMax;
}

size_t wide_ttm_scratch_bytes(const ModeView& v, int64_t K_out) {
    const WideALayout a = wide_a_layout((int)v.i, (int)K_out, true);
    return round256((size_t)a.nu * a.ubytes);
}

size_t wide_power_scratch_bytes(const ModeView& v, int L, int num_sms) {
    const WideALayout a = wide_a_layout((int)v.i, L, true);
    const WideBLayout b = wide_b_layout((int)v.i, L, true);
    const int64_t chunks = (v.fibers() + kBJB - 1) / kBJB;
    const int64_t R = std::max<int64_t>(1, std::min<int64_t>(chunks, num_sms / b.groups));
    return round256((size_t)a.nu * a.ubytes) + 2 * round256((size_t)chunks * a.Np * 128) +
           round256((size_t)R * v.i * L * sizeof(float));
}

cudaError_t launch_ttm_wide(const float* A, const ModeView& v, const float* Mp, int64_t K_out, int64_t ld_i,
                            int64_t ld_k, float* out, void* scratch, int* status, int num_sms, cudaStream_t s,
                            int max_stages) {
    if (!wide_ttm_supported(v, K_out) || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return cudaErrorNotSupported;
    const int I = (int)v.i;
    const int64_t J = v.fibers();
    const bool strided = v.lf > 1;
    const WideALayout t = wide_a_layout(I, (int)K_out, true, max_stages);
    CUtensorMap map;
    if (!make_fiber_map(&map, A, v, kAJB)) return cudaErrorNotSupported;
    unsigned char* img = reinterpret_cast<unsigned char*>(scratch);
    image_kernel<true><<<grid_for(((int64_t)t.nu * t.Np * 8 + 255) / 256, 4 * num_sms), 256, 0, s>>>(
        Mp, I, (int)K_out, ld_i, ld_k, t.Np, t.nu, img);
    note_launch();
    const int64_t tiles = (J + kAJB - 1) / kAJB;
    const double elems = (double)I * (double)J;
    {
        ProfScope prof(kKTtmWide, (elems + (double)J * K_out) * sizeof(float), 2.0 * elems * K_out, s);
        auto k = strided ? wide_ttm_kernel<true, 0, true> : wide_ttm_kernel<true, 0, false>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.bytes);
        k<<<grid_for(tiles, num_sms), kAThreads, t.bytes, s>>>(map, I, J, img, (int)K_out, t.Np, out, nullptr,
                                                                 nullptr, tiles, t.nu, v.lf, status, t.fst);
        note_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_power_wide(const float* A, const ModeView& v, const float* X_in, int L, float* X_out, bool split,
                              bool range, uint64_t seed, uint32_t stream_id, void* scratch, int* status, int num_sms,
                              cudaStream_t s, int max_stages) {
    if (!wide_supported(v, L) || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return cudaErrorNotSupported;
    const int I = (int)v.i;
    const int64_t J = v.fibers();
    const bool strided = v.lf > 1;
    const WideALayout ta = wide_a_layout(I, L, split, max_stages);
    const WideBLayout tb = wide_b_layout(I, L, split, max_stages);
    const int64_t chunks = (J + kBJB - 1) / kBJB;
    const int64_t R = std::max<int64_t>(1, std::min<int64_t>(chunks, num_sms / tb.groups));
    // scratch carve: M^T image | W hi | W lo | partials (sizes as wide_power_scratch_bytes, split)
    const WideALayout tmax = wide_a_layout(I, L, true);
    unsigned char* p = reinterpret_cast<unsigned char*>(scratch);
    unsigned char* img = p;
    p += round256((size_t)tmax.nu * tmax.ubytes);
    unsigned char* whi = p;
    p += round256((size_t)chunks * ta.Np * 128);
    unsigned char* wlo = p;
    p += round256((size_t)chunks * ta.Np * 128);
    float* part = reinterpret_cast<float*>(p);
    const double elems = (double)I * (double)J;
    if (!range) {
        CUtensorMap map;
        if (!make_fiber_map(&map, A, v, kAJB)) return cudaErrorNotSupported;
        if (split)
            image_kernel<true><<<grid_for(((int64_t)ta.nu * ta.Np * 8 + 255) / 256, 4 * num_sms), 256, 0, s>>>(
                X_in, I, L, 1, I, ta.Np, ta.nu, img);
        else
            image_kernel<false><<<grid_for(((int64_t)ta.nu * ta.Np * 8 + 255) / 256, 4 * num_sms), 256, 0, s>>>(
                X_in, I, L, 1, I, ta.Np, ta.nu, img);
        note_launch();
        const int64_t tiles = (J + kAJB - 1) / kAJB;
        ProfScope prof(kKPowerWide1, elems * sizeof(float) + (double)J * ta.Np * 2 * ta.parts, 2.0 * elems * L, s);
        auto k = split ? (strided ? wide_ttm_kernel<true, 1, true> : wide_ttm_kernel<true, 1, false>)
                       : (strided ? wide_ttm_kernel<false, 1, true> : wide_ttm_kernel<false, 1, false>);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ta.bytes);
        k<<<grid_for(tiles, num_sms), kAThreads, ta.bytes, s>>>(map, I, J, img, L, ta.Np, nullptr, whi, wlo, tiles,
                                                                  ta.nu, v.lf, status, ta.fst);
        note_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    {
        CUtensorMap map;
        if (!make_fiber_map(&map, A, v, kBJB)) return cudaErrorNotSupported;
        ProfScope prof(range ? kKRangeWide : kKPowerWide2,
                       elems * sizeof(float) + (range ? 0.0 : (double)J * tb.Np * 2 * tb.parts * tb.groups),
                       2.0 * elems * L, s);
        decltype(&wide_power2_kernel<true, true, true>) k;
        if (strided)
            k = split ? (range ? wide_power2_kernel<true, true, true> : wide_power2_kernel<true, false, true>)
                      : (range ? wide_power2_kernel<false, true, true> : wide_power2_kernel<false, false, true>);
        else
            k = split ? (range ? wide_power2_kernel<true, true, false> : wide_power2_kernel<true, false, false>)
                      : (range ? wide_power2_kernel<false, true, false> : wide_power2_kernel<false, false, false>);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tb.bytes);
        k<<<(int)(R * tb.groups), kBThreads, tb.bytes, s>>>(map, I, J, L, tb.Np, whi, wlo, seed, stream_id, part,
                                                              tb.groups, tb.nb, chunks, v.lf, status, tb.fst);
        note_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_reduce_partials<float>(part, (int)R, (int64_t)I * L, X_out, s);
}

}  // namespace tk

namespace tk {

// Y (J x L, column-major FP32) = A_(n)^T X: the first half of a half step of
// the AMM sketch, on the tensor cores (split bf16). Scratch as launch_power_wide.
cudaError_t launch_wide_tn(const float* A, const ModeView& v, const float* X, int L, float* Y, void* scratch,
                           int* status, int num_sms, cudaStream_t s, int max_stages) {
    if (!wide_supported(v, L) || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return cudaErrorNotSupported;
    const int I = (int)v.i;
    const int64_t J = v.fibers();
    const WideALayout ta = wide_a_layout(I, L, true, max_stages);
    CUtensorMap map;
    if (!make_fiber_map(&map, A, v, kAJB)) return cudaErrorNotSupported;
    unsigned char* img = reinterpret_cast<unsigned char*>(scratch);
    image_kernel<true><<<grid_for(((int64_t)ta.nu * ta.Np * 8 + 255) / 256, 4 * num_sms), 256, 0, s>>>(
        X, I, L, 1, I, ta.Np, ta.nu, img);
    note_launch();
    const int64_t tiles = (J + kAJB - 1) / kAJB;
    const double elems = (double)I * (double)J;
    ProfScope prof(kKPowerWide1, (elems + (double)J * L) * sizeof(float), 2.0 * elems * L, s);
    auto k = v.lf > 1 ? wide_ttm_kernel<true, 2, true> : wide_ttm_kernel<true, 2, false>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ta.bytes);
    k<<<grid_for(tiles, num_sms), kAThreads, ta.bytes, s>>>(map, I, J, img, L, ta.Np, Y, nullptr, nullptr, tiles,
                                                              ta.nu, v.lf, status, ta.fst);
    note_launch();
    return cudaGetLastError();
}

// X_out (I x L) = A_(n) Q with Q (J x L, column-major FP32): the second half of a
// half step, on the tensor cores (split bf16). Scratch as launch_power_wide.
cudaError_t launch_wide_nn(const float* A, const ModeView& v, const float* Q, int L, float* X_out, void* scratch,
                           int* status, int num_sms, cudaStream_t s, int max_stages) {
    if (!wide_supported(v, L) || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return cudaErrorNotSupported;
    const int I = (int)v.i;
    const int64_t J = v.fibers();
    const WideALayout ta = wide_a_layout(I, L, true);
    const WideBLayout tb = wide_b_layout(I, L, true, max_stages);
    const int64_t chunks = (J + kBJB - 1) / kBJB;
    const int64_t R = std::max<int64_t>(1, std::min<int64_t>(chunks, num_sms / tb.groups));
    unsigned char* p = reinterpret_cast<unsigned char*>(scratch);
    p += round256((size_t)ta.nu * ta.ubytes);
    unsigned char* whi = p;
    p += round256((size_t)chunks * ta.Np * 128);
    unsigned char* wlo = p;
    p += round256((size_t)chunks * ta.Np * 128);
    float* part = reinterpret_cast<float*>(p);
    bimage_kernel<true><<<grid_for((chunks * 64 * (ta.Np / 8) + 255) / 256, 4 * num_sms), 256, 0, s>>>(
        Q, J, L, ta.Np, chunks, whi, wlo);
    note_launch();
    CUtensorMap map;
    if (!make_fiber_map(&map, A, v, kBJB)) return cudaErrorNotSupported;
    const double elems = (double)I * (double)J;
    {
        ProfScope prof(kKPowerWide2, elems * sizeof(float) + (double)J * tb.Np * 2 * tb.parts * tb.groups,
                       2.0 * elems * L, s);
        auto k = v.lf > 1 ? wide_power2_kernel<true, false, true> : wide_power2_kernel<true, false, false>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tb.bytes);
        k<<<(int)(R * tb.groups), kBThreads, tb.bytes, s>>>(map, I, J, L, tb.Np, whi, wlo, 0, 0, part, tb.groups,
                                                              tb.nb, chunks, v.lf, status, tb.fst);
        note_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_reduce_partials<float>(part, (int)R, (int64_t)I * L, X_out, s);
}

cudaError_t launch_wait_timeout(int iters, int* status, cudaStream_t s) {
    if (iters < 1) return cudaErrorInvalidValue;
    wait_timeout_kernel<<<1, 64, 0, s>>>(iters, status);
    note_launch();
    return cudaGetLastError();
}

bool gram_wide_supported(const ModeView& v) {
    return layout_ok(v) && v.i >= 1 && v.i <= 128 && v.fibers() <= (int64_t)INT_MAX - 256;
}

size_t gram_wide_scratch_bytes(const ModeView& v, int num_sms) {
    const int64_t chunks = (v.fibers() + kBJB - 1) / kBJB;
    const int64_t R = std::max<int64_t>(1, std::min<int64_t>(chunks, num_sms));
    return round256((size_t)R * v.i * v.i * sizeof(float));
}

cudaError_t launch_gram_wide(const float* A, const ModeView& v, float* G, bool split, void* scratch, int* status,
                             int num_sms, cudaStream_t s, int max_stages) {
    if (!gram_wide_supported(v) || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return cudaErrorNotSupported;
    const int I = (int)v.i;
    const int64_t J = v.fibers();
    const bool strided = v.lf > 1;
    const GramLayout t = gram_layout(I, split, max_stages);
    if (t.bytes > kWSmemMax) return cudaErrorNotSupported;
    const int64_t chunks = (J + kBJB - 1) / kBJB;
    const int64_t R = std::max<int64_t>(1, std::min<int64_t>(chunks, num_sms));
    CUtensorMap map;
    if (!make_fiber_map(&map, A, v, kBJB)) return cudaErrorNotSupported;
    float* part = reinterpret_cast<float*>(scratch);
    {
        const double elems = (double)I * (double)J;
        ProfScope prof(kKGramWide, elems * sizeof(float), 2.0 * elems * I, s);
        auto k = split ? (strided ? gram_wide_kernel<true, true> : gram_wide_kernel<true, false>)
                       : (strided ? gram_wide_kernel<false, true> : gram_wide_kernel<false, false>);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.bytes);
        k<<<(int)R, kBThreads, t.bytes, s>>>(map, I, J, t.Np, part, chunks, v.lf, status, t.fst);
        note_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_reduce_partials<float>(part, (int)R, (int64_t)I * I, G, s);
}

}  // namespace tk
