// Power step of Strategy A on the 5th-generation tensor cores with single-pass
// BF16 operands (tcgen05 kind::f16, FP32 accumulation in tensor memory):
// X_out = A_(n) (A_(n)^T X_in) for contiguous mode-n fibers (mode 1). A, X_in
// and W = A^T X are each rounded to bf16 (8 significant bits, to nearest) once;
// the sums are FP32. This is the form whose rounding the power steps win back:
// a relative error of order 2^-8 in the sketch moves the captured subspace by
// an angle of that order and the decomposition's relative error only to second
// order.
//
// TMA loads 64-fiber tiles in FP32 sub-stages of 128 values i (four 128-byte
// swizzled rows per fiber) into a 4-slot ring. Eight transposer warps read each
// sub-stage once (a warp reads one fiber's 32 consecutive values per load, no
// bank conflicts), round to bf16 and write it twice: into tensor memory
// transposed (T': rows i on lanes, pairs of fibers packed in 32-bit columns),
// and into shared memory K-major (one 128-byte row of 64 values per fiber) for
// the first product; the FP32 slot is released as soon as it has been read.
//   D1 = X^T T      M = 64 (X^T's 32 stored rows plus 32 that read the next
//                   4 KB and yield accumulator rows never read), N = 64 fibers,
//                   K = I_n in steps of 16; accumulated over the sub-stages.
//   W  = D1^T       read back by two warps, rounded to bf16, K-major.
//   Xacc += T' W    M = 128 rows of I_n per block, A from tensor memory,
//                   N = 32 columns l, K = 64 fibers.
// Packed in bf16, T' takes 128 columns, so it and D1 are double-buffered
// (Xacc 128 + D1 2 x 64 + T' 2 x 128 = 512 columns) and the products of tile k
// overlap the transposition of tile k + 1. Xacc stays in tensor memory across
// the CTA's tiles and is written once as its partial; the partials are summed
// in a fixed order afterwards.
//
// Strided fibers (modes 2..N, stride Lf >= 64): TMA loads 3-D boxes of 32
// fibers x 32 values (fibers contiguous, one 128-byte row per value i), a tile
// being 64 consecutive fibers of one slab (columns past Lf load as zeros), and a
// transposer lane reads its own row instead of a column; the rest is the same.
//
// Warp roles (one CTA per SM, persistent over tiles j = blockIdx.x + k gridDim.x):
// warps 0-1 read W back (tensor-memory lane quarters 0 and 1), warp 2 issues
// the TMA loads, warp 3 the MMAs (first product of tile k, then the second
// product of tile k - 1), warps 4-11 transpose and finally read Xacc. Every
// mbarrier wait is bounded: on a timeout the kernel records kStatTimeout, lets
// the copies and products it issued finish (with the same bound), frees its
// tensor memory and returns.
#include <climits>

#include "internal.h"
#include "tc.cuh"
#include "tma.cuh"

namespace tk {
namespace {

constexpr int kHThreads = 384;
constexpr int kHJB = 64;                   // fibers per tile
constexpr int kHBox = kHJB * 128;          // FP32 box: 32 values i x 64 fibers = 8 KB
constexpr int kHSubChunks = 4;             // FP32 boxes per sub-stage (128 values i)
constexpr int kHSub = kHSubChunks * kHBox; // 32 KB
constexpr int kHStages = 4;                // FP32 sub-stages in the ring
constexpr int kHBChunk = kHJB * 128;       // bf16 chunk: 64 values i x 64 fibers = 8 KB
constexpr int kHBSub = 2 * kHBChunk;       // bf16 sub-stage (128 values i) = 16 KB
constexpr int kHCStages = 2;               // bf16 sub-stages
constexpr int kHXChunk = 4096;             // X^T bf16 chunk: 32 rows l x 128 bytes (64 values i)
constexpr int kHWBytes = 4096;             // W^T bf16: 32 rows l x 128 bytes (64 fibers)
constexpr int kHWBufs = 2;                 // W^T buffers
constexpr int kHTransposers = 8;           // warps 4 .. 11
constexpr int kHWaitIters = 1 << 22;
constexpr size_t kHSmemMax = 227 * 1024;
constexpr uint32_t kHTmemCols = 512;
constexpr uint32_t kHD1Col = 128;          // D1: 2 x 64 columns
constexpr uint32_t kHTpCol = 256;          // T': 2 x (4 blocks x 32 columns)
constexpr int kHBars = 2 * kHStages + 17;        // 8 bytes each; 256 reserved
static_assert(kHBars * 8 + 8 <= 256, "barrier area");

struct HLayout {
    int nc = 0;     // FP32 chunks of 32 values
    int nsub = 0;   // sub-stages per tile = 128-row blocks of I_n
    int nbc = 0;    // bf16 chunks of 64 values
    size_t c_off = 0, x_off = 0, w_off = 0, bar_off = 0, bytes = 0;
};

HLayout h_layout(int I) {
    HLayout t;
    t.nc = (I + 31) / 32;
    t.nsub = (t.nc + kHSubChunks - 1) / kHSubChunks;
    t.nbc = (I + 63) / 64;
    t.c_off = (size_t)kHStages * kHSub;
    t.x_off = t.c_off + (size_t)kHCStages * kHBSub;
    t.w_off = t.x_off + (size_t)t.nbc * kHXChunk;
    t.bar_off = t.w_off + (size_t)kHWBufs * kHWBytes;
    t.bytes = t.bar_off + 256 + 1024;
    return t;
}

__device__ __forceinline__ bool wait_bar(uint64_t* b, uint32_t parity, volatile int* flag) {
    for (int it = 0; it < kHWaitIters; ++it) {
        if (tc::mbar_try(b, parity)) return true;
        if ((it & 255) == 255 && *flag) return false;
    }
    return false;
}

__device__ __forceinline__ void fail(volatile int* flag, int* status) {
    *flag = 1;
    set_status(status, kStatTimeout);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&p);
}

template <bool STRIDED>
__global__ void __launch_bounds__(kHThreads, 1)
    power_bf16x1_kernel(const __grid_constant__ CUtensorMap map, int I, const float* __restrict__ X, int L,
                        float* __restrict__ partial, int64_t tiles, int64_t tiles_per_slab, int nc, int nbc,
                        int* status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // swizzled buffers start on 1024-byte boundaries (the launch adds 1 KB of slack)
    unsigned char* smem = smem_raw + ((1024 - (tma::smem_addr(smem_raw) & 1023)) & 1023);
    unsigned char* Cb = smem + (size_t)kHStages * kHSub;               // bf16 sub-stages
    unsigned char* Xs = Cb + (size_t)kHCStages * kHBSub;               // X^T bf16
    unsigned char* Ws = Xs + (size_t)nbc * kHXChunk;                   // W^T bf16 [2]
    uint64_t* bar = reinterpret_cast<uint64_t*>(Ws + kHWBufs * kHWBytes);
    uint64_t* f_full = bar;                    // FP32 sub-stage loaded (TMA bytes)
    uint64_t* f_empty = f_full + kHStages;     // FP32 sub-stage read (8 warps)
    uint64_t* c_full = f_empty + kHStages;     // [2] bf16 sub-stage written (8 warps)
    uint64_t* c_empty = c_full + 2;            // [2] bf16 sub-stage consumed by the first product
    uint64_t* d1_full = c_empty + 2;           // [2] first product done
    uint64_t* d1_empty = d1_full + 2;          // [2] first product read back (2 warps)
    uint64_t* w_full = d1_empty + 2;           // [kHWBufs] W written (2 warps)
    uint64_t* w_empty = w_full + 2;            // [kHWBufs] second product done with W
    uint64_t* tp_full = w_empty + 2;           // [2] T' of a tile written (8 warps)
    uint64_t* tp_empty = tp_full + 2;          // [2] second product done with T'
    uint64_t* done = tp_empty + 2;             // every product done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + kHBars);
    volatile int* flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nsub = (nc + kHSubChunks - 1) / kHSubChunks;
    const int64_t nloc = tiles > (int64_t)blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    // X^T in bf16 as the K-major A operand of the first product: rows l < 32,
    // chunk c of 64 values i per 128-byte row; zero beyond L and I
    const int ipt = nbc * 64;
    for (int e = tid; e < 32 * (ipt / 2); e += kHThreads) {
        const int l = e / (ipt / 2), i = 2 * (e - l * (ipt / 2));
        const float x0 = (l < L && i < I) ? __ldg(X + (int64_t)l * I + i) : 0.f;
        const float x1 = (l < L && i + 1 < I) ? __ldg(X + (int64_t)l * I + i + 1) : 0.f;
        const int c = i >> 6, p = (i >> 3) & 7;
        *reinterpret_cast<uint32_t*>(Xs + c * kHXChunk + (l >> 3) * 1024 + (l & 7) * 128 + ((p ^ (l & 7)) << 4) +
                                     (i & 7) * 2) = pack_bf16(x0, x1);
    }
    if (tid == 0) {
        for (int k = 0; k < kHBars; ++k) {
            const uint64_t* b = &bar[k];
            uint32_t count = 1;                                            // TMA, commits, done
            if ((b >= f_empty && b < f_empty + kHStages) || (b >= c_full && b < c_full + 2) ||
                (b >= tp_full && b < tp_full + 2))
                count = kHTransposers;
            if ((b >= d1_empty && b < d1_empty + 2) || (b >= w_full && b < w_full + 2)) count = 2;
            tc::mbar_init(&bar[k], count);
        }
        *flag = 0;
        tma::fence_barrier_init();
    }
    if (warp == 3) tc::tmem_alloc(tmem_slot, kHTmemCols);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 2) {
        if (lane == 0) {
            int64_t g = 0;
            bool ok = true;
            for (int64_t k = 0; k < nloc && ok; ++k) {
                const int64_t tile = blockIdx.x + k * gridDim.x;
                // contiguous: fibers tile * 64 ..; strided: slab r, fibers a0 .. a0 + 63 of it
                const int j0 = (int)(tile * kHJB);
                const int r = STRIDED ? (int)(tile / tiles_per_slab) : 0;
                const int a0 = STRIDED ? (int)((tile % tiles_per_slab) * kHJB) : 0;
                for (int u = 0; u < nsub; ++u, ++g) {
                    const int slot = (int)(g % kHStages);
                    if (g >= kHStages && !wait_bar(&f_empty[slot], (uint32_t)((g / kHStages - 1) & 1), flag)) {
                        fail(flag, status);
                        ok = false;
                        break;
                    }
                    const int nch = min(kHSubChunks, nc - u * kHSubChunks);
                    tma::expect_tx(&f_full[slot], (uint32_t)(nch * kHBox));
                    unsigned char* dst = smem + (size_t)slot * kHSub;
                    for (int cc = 0; cc < nch; ++cc) {
                        const int i0 = (u * kHSubChunks + cc) * 32;
                        if (STRIDED) {
                            // chunk cc: values i0 .. i0 + 31 (rows) x fibers a0 .. a0 + 31, then a0 + 32 ..
                            tma::load_3d(dst + cc * kHBox, &map, a0, i0, r, &f_full[slot]);
                            tma::load_3d(dst + cc * kHBox + kHBox / 2, &map, a0 + 32, i0, r, &f_full[slot]);
                        } else {
                            tma::load_2d(dst + cc * kHBox, &map, i0, j0, &f_full[slot]);
                        }
                    }
                }
            }
            if (*flag) {
                const int64_t g0 = g > kHStages ? g - kHStages : 0;
                for (int64_t gg = g0; gg < g; ++gg)
                    for (int it = 0; it < kHWaitIters; ++it)
                        if (tc::mbar_try(&f_full[gg % kHStages], (uint32_t)((gg / kHStages) & 1))) break;
            }
        }
    } else if (warp == 3) {
        if (lane == 0) {
            const uint32_t id1 = tc::idesc_bf16(64, kHJB, false, false);
            const uint32_t id2 = tc::idesc_bf16(128, 32, false, false);
            // descriptors built once; a K step (16 bf16 = 32 bytes) advances the
            // start address field by 2, a 64-value chunk by its region size >> 4
            const uint64_t x_desc = tc::desc_sw128(tc::smem_u32(Xs), 16, 1024);
            const uint64_t c_desc = tc::desc_sw128(tc::smem_u32(Cb), 16, 1024);
            const uint64_t w_desc = tc::desc_sw128(tc::smem_u32(Ws), 16, 1024);
            auto second = [&](int64_t k) -> bool {
                const int b = (int)(k & 1), bw = (int)(k % kHWBufs);
                if (!wait_bar(&w_full[bw], (uint32_t)((k / kHWBufs) & 1), flag) ||
                    !wait_bar(&tp_full[b], (uint32_t)((k >> 1) & 1), flag))
                    return false;
                tc::fence_after_sync();
                const uint64_t wb = w_desc + (uint64_t)((bw * kHWBytes) >> 4);
                const uint32_t tb = tmem + kHTpCol + (uint32_t)(b * 128);
                for (int mb = 0; mb < nsub; ++mb) {
#pragma unroll
                    for (int ks = 0; ks < kHJB / 16; ++ks)
                        tc::mma_bf16_ts(tmem + (uint32_t)(mb * 32), tb + (uint32_t)(mb * 32 + ks * 8),
                                        wb + (uint64_t)(ks * 2), id2, k > 0 || ks > 0);
                }
                tc::commit(&tp_empty[b]);
                tc::commit(&w_empty[bw]);
                return true;
            };
            bool ok = true;
            int64_t g = 0;
            for (int64_t k = 0; k < nloc && ok; ++k) {
                const int b = (int)(k & 1);
                const uint32_t d1 = tmem + kHD1Col + (uint32_t)(b * kHJB);
                for (int u = 0; u < nsub; ++u, ++g) {
                    const int cs = (int)(g % kHCStages);
                    if (!wait_bar(&c_full[cs], (uint32_t)((g / kHCStages) & 1), flag) ||
                        (u == 0 && k >= 2 && !wait_bar(&d1_empty[b], (uint32_t)(((k >> 1) - 1) & 1), flag))) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const int ncb = min(2, nbc - 2 * u);        // bf16 chunks of this sub-stage
                    for (int cb = 0; cb < ncb; ++cb) {
                        const uint64_t a = x_desc + (uint64_t)(((2 * u + cb) * kHXChunk) >> 4);
                        const uint64_t bd = c_desc + (uint64_t)((cs * kHBSub + cb * kHBChunk) >> 4);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            tc::mma_bf16(d1, a + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), id1,
                                         u > 0 || cb > 0 || kk > 0);
                    }
                    tc::commit(&c_empty[cs]);
                }
                if (!ok) break;
                tc::commit(&d1_full[b]);
                if (k >= 1 && !second(k - 1)) {
                    ok = false;
                    break;
                }
            }
            if (ok && nloc > 0 && !second(nloc - 1)) ok = false;
            tc::commit(done);
            if (!ok) {
                fail(flag, status);
                for (int it = 0; it < kHWaitIters; ++it)
                    if (tc::mbar_try(done, 0)) break;
            }
        }
    } else if (warp < 2) {
        // D1 (M = 64): row l sits in lane (l % 16) + 32 (l / 16), so rows 0..31 are
        // lanes 0..15 of quarters 0 and 1
        const int quarter = warp;
        for (int64_t k = 0; k < nloc; ++k) {
            const int b = (int)(k & 1);
            if (!wait_bar(&d1_full[b], (uint32_t)((k >> 1) & 1), flag)) {
                fail(flag, status);
                break;
            }
            tc::fence_after_sync();
            uint32_t r[kHJB];
            const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + kHD1Col + (uint32_t)(b * kHJB);
#pragma unroll
            for (int h = 0; h < kHJB / 16; ++h)
                tc::tmem_ld16(ta + (uint32_t)(h * 16), *reinterpret_cast<uint32_t(*)[16]>(&r[h * 16]));
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&d1_empty[b]);
            const int bw = (int)(k % kHWBufs);
            if (k >= kHWBufs && !wait_bar(&w_empty[bw], (uint32_t)((k / kHWBufs - 1) & 1), flag)) {
                fail(flag, status);
                break;
            }
            if (lane < 16) {
                // row l of W^T in bf16: fibers 8 q .. 8 q + 7 in 16-byte group q
                const int l = quarter * 16 + lane;
                unsigned char* row = Ws + bw * kHWBytes + (l >> 3) * 1024 + (l & 7) * 128;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float* f = reinterpret_cast<const float*>(&r[8 * q]);
                    *reinterpret_cast<uint4*>(row + ((q ^ (l & 7)) << 4)) =
                        make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]),
                                   pack_bf16(f[6], f[7]));
                }
            }
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&w_full[bw]);
        }
    } else {
        // transposers: warp w reads FP32 chunk 4 u + w % 4 (rows i = its lanes) of
        // sub-stage u for fibers 32 half .. 32 half + 31, and writes (a) those
        // values packed in pairs of fibers into tensor memory, lanes 32 (w % 4) ..,
        // and (b) the K-major bf16 rows of those fibers for the first product
        const int quarter = warp & 3, half = (warp - 4) >> 2;
        bool ok = true;
        int64_t g = 0;
        for (int64_t k = 0; k < nloc && ok; ++k) {
            const int b2 = (int)(k & 1);
            for (int u = 0; u < nsub; ++u, ++g) {
                const int slot = (int)(g % kHStages), cs = (int)(g % kHCStages);
                if (!wait_bar(&f_full[slot], (uint32_t)((g / kHStages) & 1), flag)) {
                    ok = false;
                    break;
                }
                const int c = u * kHSubChunks + quarter;
                float v[32];
                if (c < nc && STRIDED) {
                    // row i = this lane of the chunk: fibers 32 half .. + 31 in 16-byte pieces
                    const unsigned char* row = smem + (size_t)slot * kHSub + quarter * kHBox + half * (kHBox / 2) +
                                               lane * 128;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 x = *reinterpret_cast<const float4*>(row + ((q ^ (lane & 7)) << 4));
                        v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
                    }
                } else if (c < nc) {
                    // fiber j's row of the chunk: value i = this lane
                    const unsigned char* src = smem + (size_t)slot * kHSub + quarter * kHBox +
                                               half * 32 * 128 + (lane & 3) * 4;
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        v[j] = *reinterpret_cast<const float*>(src + j * 128 + (((lane >> 2) ^ (j & 7)) << 4));
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = 0.f;
                }
                // the FP32 values are in registers: release the slot to the TMA
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&f_empty[slot]);
                if ((u == 0 && k >= 2 && !wait_bar(&tp_empty[b2], (uint32_t)(((k >> 1) - 1) & 1), flag)) ||
                    (g >= kHCStages && !wait_bar(&c_empty[cs], (uint32_t)((g / kHCStages - 1) & 1), flag))) {
                    ok = false;
                    break;
                }
                uint32_t pk[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) pk[q] = pack_bf16(v[2 * q], v[2 * q + 1]);
                tc::tmem_st16(tmem + ((uint32_t)(quarter * 32) << 16) + kHTpCol +
                                  (uint32_t)(b2 * 128 + u * 32 + half * 16), pk);
                // K-major bf16 rows: value i (this lane) of fiber j at byte
                // cl 8192 + j 128 + ((p ^ (j % 8)) << 4) + (i % 8) 2, cl = quarter / 2,
                // p = ((quarter % 2) 32 + lane) / 8
                unsigned char* dst = Cb + (size_t)cs * kHBSub + (quarter >> 1) * kHBChunk + (lane & 7) * 2;
                const int p = ((quarter & 1) * 32 + lane) >> 3;
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const int j = half * 32 + jj;
                    *reinterpret_cast<__nv_bfloat16*>(dst + j * 128 + ((p ^ (j & 7)) << 4)) =
                        __float2bfloat16_rn(v[jj]);
                }
                tc::fence_async_smem();
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&c_full[cs]);
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tp_full[b2]);
        }
        if (!ok) fail(flag, status);
        // Xacc: row i of block mb in lane i % 128, columns l
        if (ok && wait_bar(done, 0, flag) && !*flag) {
            tc::fence_after_sync();
            float* out = partial + (int64_t)blockIdx.x * ((int64_t)I * L);
            for (int mb = half; mb < nsub; mb += 2) {
                uint32_t r[32];
                const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(mb * 32);
                tc::tmem_ld16(ta, *reinterpret_cast<uint32_t(*)[16]>(&r[0]));
                tc::tmem_ld16(ta + 16, *reinterpret_cast<uint32_t(*)[16]>(&r[16]));
                const int i = mb * 128 + quarter * 32 + lane;
                if (i < I)
#pragma unroll
                    for (int l = 0; l < 32; ++l)
                        if (l < L) out[(int64_t)l * I + i] = __uint_as_float(r[l]);
            }
        } else if (!*flag) {
            fail(flag, status);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 3) tc::tmem_dealloc(tmem, kHTmemCols);
}

}  // namespace

bool power_bf16x1_supported(const ModeView& v, int L) {
    const bool layout = v.lf == 1 || (v.lf >= kHJB && v.lf % 4 == 0);
    return layout && v.i >= 1 && v.i % 4 == 0 && v.i <= 512 && L >= 1 && L <= 32 &&
           v.fibers() <= (int64_t)INT_MAX - kHJB && v.rt <= (int64_t)INT_MAX &&
           h_layout((int)v.i).bytes <= kHSmemMax;
}

cudaError_t launch_power_bf16x1(const float* A, const ModeView& v, const float* X_in, int L, float* X_out,
                                void* partials, int* status, int num_sms, cudaStream_t s) {
    if (!power_bf16x1_supported(v, L) || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return cudaErrorNotSupported;
    const int I = (int)v.i;
    const int64_t J = v.fibers();
    const bool strided = v.lf > 1;
    CUtensorMap map;
    int64_t tiles, per_slab = 1;
    if (!strided) {
        const uint64_t dims[2] = {(uint64_t)I, (uint64_t)J};
        const uint64_t strides[1] = {(uint64_t)I * sizeof(float)};
        const uint32_t box[2] = {32, (uint32_t)kHJB};
        if (!tma::make_map_f32(&map, A, 2, dims, strides, box, true)) return cudaErrorNotSupported;
        tiles = (J + kHJB - 1) / kHJB;
    } else {
        // (Lf, I, Rt) with Lf fastest; a box is 32 fibers x 32 values of one slab
        const uint64_t dims[3] = {(uint64_t)v.lf, (uint64_t)I, (uint64_t)v.rt};
        const uint64_t strides[2] = {(uint64_t)v.lf * sizeof(float), (uint64_t)v.lf * I * sizeof(float)};
        const uint32_t box[3] = {32, 32, 1};
        if (!tma::make_map_f32(&map, A, 3, dims, strides, box, true)) return cudaErrorNotSupported;
        per_slab = (v.lf + kHJB - 1) / kHJB;
        tiles = per_slab * v.rt;
    }
    const HLayout t = h_layout(I);
    int grid = (int)(tiles < num_sms ? tiles : num_sms);
    if (grid < 1) grid = 1;
    float* part = reinterpret_cast<float*>(partials);
    const double elems = (double)I * (double)J;
    {
        ProfScope prof(kKPowerBf16x1, elems * sizeof(float), 4.0 * elems * L, s);
        auto k = strided ? power_bf16x1_kernel<true> : power_bf16x1_kernel<false>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.bytes);
        k<<<grid, kHThreads, t.bytes, s>>>(map, I, X_in, L, part, tiles, per_slab, t.nc, t.nbc, status);
        note_launch();
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce_partials<float>(part, grid, (int64_t)I * L, X_out, s);
}

}  // namespace tk
