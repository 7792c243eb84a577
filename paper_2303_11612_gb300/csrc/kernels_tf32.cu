// Power step of Strategy A on the 5th-generation tensor cores with TF32
// operands (tcgen05 kind::tf32, FP32 accumulation in tensor memory):
// X_out = A_(n) (A_(n)^T X_in) for contiguous mode-n fibers (mode 1).
//
// The tensor is read once, by TMA, straight into the 128-byte-swizzled shared
// layout the tensor cores read, in FP32: there is no conversion pass. The
// tensor cores use the top 19 bits of each FP32 operand (TF32, about 2^-11
// relative), so the products are of A and X rounded to TF32 and summed in FP32.
//
// A tile T holds 64 fibers x I_n and streams through a ring of sub-stages of
// 128 values i (four i-chunks of 32 values = one 128-byte row per fiber each).
// Per tile:
//   D1 = X^T T      M = 64 (rows l of X^T; only the first 32 are stored, the
//                   rest of the operand reads the next 4 KB and yields
//                   accumulator rows that are never read), N = 64 fibers,
//                   K = I_n; both operands K-major in shared memory,
//                   accumulated over the sub-stages.
//   W  = D1^T       read back by two warps and written as the K-major operand
//                   of the second product (one 256-byte row per l).
//   T'              the tile transposed into tensor memory (rows i on lanes,
//                   fibers along columns) by eight warps as each sub-stage
//                   lands: a warp reads one fiber's 32 consecutive values per
//                   load (a whole 128-byte row, no bank conflict) and stores 32
//                   columns of its lanes; sub-stage u fills 128-row block u.
//   Xacc += T' W    M = 128 rows of I_n per block, A from tensor memory,
//                   N = 32 columns l, K = 64 fibers.
// The tensor cores take TF32 operands K-major only, so the fiber-contracting
// product cannot read the tile in its loaded layout; and an instruction of
// these shapes costs about the same whatever its N, so the tile is as wide as
// tensor memory allows (Xacc 128 columns, D1 2 x 64, T' 256). Xacc stays in
// tensor memory across all tiles of the CTA and is written once as the CTA's
// partial; the partials are summed in a fixed order afterwards.
//
// Warp roles (one CTA per SM, persistent over tiles j = blockIdx.x + k gridDim.x):
// warps 0-1 read W back (tensor-memory lane quarters 0 and 1), warp 2 issues
// the TMA loads, warp 3 issues the MMAs (first product of tile k, then its
// second product once W and T' are in place), warps 4-11 transpose and finally
// read Xacc. Every mbarrier wait is bounded: on a timeout the kernel records
// kStatTimeout, lets the copies and products it issued finish (with the same
// bound), frees its tensor memory and returns.
#include <climits>

#include "internal.h"
#include "tc.cuh"
#include "tma.cuh"

namespace tk {
namespace {

constexpr int kFThreads = 384;
constexpr int kFJB = 64;                   // fibers per tile (N of the first product)
constexpr int kFBox = kFJB * 128;          // one i-chunk (32 values) of a tile: 8 KB
constexpr int kFSubChunks = 4;             // i-chunks per sub-stage (128 values i)
constexpr int kFSubBytes = kFSubChunks * kFBox;
constexpr int kFStages = 4;                // sub-stages in the ring
constexpr int kFRowChunk = 4096;           // one i-chunk of X^T: 32 rows l x 128 bytes
constexpr int kFWBytes = 2 * 4096;         // W: 32 rows l x 256 bytes (two 128-byte atoms along K)
constexpr int kFTransposers = 8;           // warps 4 .. 11
constexpr int kFWaitIters = 1 << 22;
constexpr size_t kFSmemMax = 227 * 1024;
// tensor memory columns: Xacc at 0 (32 per 128-row block, up to 4 blocks), D1
// double buffer at 128 (64 columns each), T' at 256 (64 columns per block)
constexpr uint32_t kFTmemCols = 512;
constexpr uint32_t kFD1Col = 128;
constexpr uint32_t kFTpCol = 256;

struct TfLayout {
    int nc = 0;              // i-chunks of 32
    int nsub = 0;            // sub-stages per tile = 128-row blocks of I_n
    size_t x_off = 0, w_off = 0, bar_off = 0, bytes = 0;
};

TfLayout tf_layout(int I) {
    TfLayout t;
    t.nc = (I + 31) / 32;
    t.nsub = (t.nc + kFSubChunks - 1) / kFSubChunks;
    t.x_off = (size_t)kFStages * kFSubBytes;
    t.w_off = t.x_off + (size_t)t.nc * kFRowChunk;
    t.bar_off = t.w_off + 2 * kFWBytes;
    t.bytes = t.bar_off + 256 + 1024;
    return t;
}

__device__ __forceinline__ bool wait_bar(uint64_t* b, uint32_t parity, volatile int* flag) {
    for (int it = 0; it < kFWaitIters; ++it) {
        if (tc::mbar_try(b, parity)) return true;
        if ((it & 255) == 255 && *flag) return false;
    }
    return false;
}

__device__ __forceinline__ void fail(volatile int* flag, int* status) {
    *flag = 1;
    set_status(status, kStatTimeout);
}

__global__ void __launch_bounds__(kFThreads, 1)
    power_tf32_kernel(const __grid_constant__ CUtensorMap map, int I, const float* __restrict__ X, int L,
                      float* __restrict__ partial, int64_t tiles, int nc, int* status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the 128-byte swizzle is a function of the address: the ring, X^T and W start
    // on 1024-byte boundaries (the launch adds 1 KB of slack)
    unsigned char* smem = smem_raw + ((1024 - (tma::smem_addr(smem_raw) & 1023)) & 1023);
    unsigned char* Xs = smem + (size_t)kFStages * kFSubBytes;
    unsigned char* Ws = Xs + (size_t)nc * kFRowChunk;
    uint64_t* bar = reinterpret_cast<uint64_t*>(Ws + 2 * kFWBytes);
    uint64_t* full = bar;              // [4] sub-stage loaded (TMA bytes)
    uint64_t* empty = bar + 4;         // [4] sub-stage read by the first product and the transposers
    uint64_t* d1_full = bar + 8;       // [2] first product done
    uint64_t* d1_empty = bar + 10;     // [2] first product read back (2 warps)
    uint64_t* w_full = bar + 12;       // [2] W written (2 warps)
    uint64_t* w_empty = bar + 14;      // [2] second product done with W
    uint64_t* tp_full = bar + 16;      // T' of the tile written (8 warps)
    uint64_t* tp_empty = bar + 17;     // second product done with T'
    uint64_t* done = bar + 18;         // every product done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 19);
    volatile int* flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nsub = (nc + kFSubChunks - 1) / kFSubChunks;
    const int64_t nloc = tiles > (int64_t)blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    // X^T as the K-major A operand of the first product: rows l < 32, chunk c of
    // 32 values i per 128-byte row; zero beyond L and I
    const int ipt = nc * 32;
    for (int e = tid; e < 32 * ipt; e += kFThreads) {
        const int l = e / ipt, i = e - l * ipt;
        const float x = (l < L && i < I) ? __ldg(X + (int64_t)l * I + i) : 0.f;
        const int c = i >> 5, q = (i >> 2) & 7;
        *reinterpret_cast<float*>(Xs + c * kFRowChunk + (l >> 3) * 1024 + (l & 7) * 128 + ((q ^ (l & 7)) << 4) +
                                  (i & 3) * 4) = x;
    }
    if (tid == 0) {
        for (int k = 0; k < 19; ++k) {
            uint32_t count = 1;
            if (k >= 4 && k < 8) count = 1 + kFTransposers;       // empty: MMA commit + transposers
            if (k >= 10 && k < 14) count = 2;                     // d1_empty, w_full
            if (k == 16) count = kFTransposers;                   // tp_full
            tc::mbar_init(&bar[k], count);
        }
        *flag = 0;
        tma::fence_barrier_init();
    }
    if (warp == 3) tc::tmem_alloc(tmem_slot, kFTmemCols);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 2) {
        if (lane == 0) {
            // producer: sub-stage g = k nsub + u into slot g % kFStages once sub-stage
            // g - kFStages has been read
            int64_t g = 0;
            bool ok = true;
            for (int64_t k = 0; k < nloc && ok; ++k) {
                const int j0 = (int)((blockIdx.x + k * gridDim.x) * kFJB);
                for (int u = 0; u < nsub; ++u, ++g) {
                    const int slot = (int)(g % kFStages);
                    if (g >= kFStages && !wait_bar(&empty[slot], (uint32_t)((g / kFStages - 1) & 1), flag)) {
                        fail(flag, status);
                        ok = false;
                        break;
                    }
                    const int nch = min(kFSubChunks, nc - u * kFSubChunks);
                    tma::expect_tx(&full[slot], (uint32_t)(nch * kFBox));
                    unsigned char* dst = smem + (size_t)slot * kFSubBytes;
                    for (int cc = 0; cc < nch; ++cc)
                        tma::load_2d(dst + cc * kFBox, &map, (u * kFSubChunks + cc) * 32, j0, &full[slot]);
                }
            }
            if (*flag) {
                // let the copies still in flight land before the CTA ends
                const int64_t g0 = g > kFStages ? g - kFStages : 0;
                for (int64_t gg = g0; gg < g; ++gg)
                    for (int it = 0; it < kFWaitIters; ++it)
                        if (tc::mbar_try(&full[gg % kFStages], (uint32_t)((gg / kFStages) & 1))) break;
            }
        }
    } else if (warp == 3) {
        if (lane == 0) {
            const uint32_t id1 = tc::idesc_tf32(64, kFJB, false, false);
            const uint32_t id2 = tc::idesc_tf32(128, 32, false, false);
            const uint32_t xa = tc::smem_u32(Xs), wa = tc::smem_u32(Ws), sa = tc::smem_u32(smem);
            // descriptors are built once; a K step advances the start address field
            // (address >> 4, bits 0-13) by 32 bytes
            const uint64_t x_desc = tc::desc_sw128(xa, 16, 1024);
            const uint64_t w_desc = tc::desc_sw128(wa, 16, 1024);
            const uint64_t t_desc = tc::desc_sw128(sa, 16, 1024);
            bool ok = true;
            int64_t g = 0;
            for (int64_t k = 0; k < nloc && ok; ++k) {
                const int b = (int)(k & 1);
                const uint32_t d1 = tmem + kFD1Col + (uint32_t)(b * kFJB);
                for (int u = 0; u < nsub; ++u, ++g) {
                    const int slot = (int)(g % kFStages);
                    if (!wait_bar(&full[slot], (uint32_t)((g / kFStages) & 1), flag) ||
                        (u == 0 && k >= 2 && !wait_bar(&d1_empty[b], (uint32_t)(((k >> 1) - 1) & 1), flag))) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const int nch = min(kFSubChunks, nc - u * kFSubChunks);
                    uint64_t a = x_desc + (uint64_t)((u * kFSubChunks * kFRowChunk) >> 4);
                    uint64_t bd = t_desc + (uint64_t)((slot * kFSubBytes) >> 4);
                    for (int cc = 0; cc < nch; ++cc) {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            tc::mma_tf32(d1, a + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), id1,
                                         u > 0 || cc > 0 || kk > 0);
                        a += (uint64_t)(kFRowChunk >> 4);
                        bd += (uint64_t)(kFBox >> 4);
                    }
                    tc::commit(&empty[slot]);
                }
                if (!ok) break;
                tc::commit(&d1_full[b]);
                // second product of tile k: W and the whole T' in place
                if (!wait_bar(&w_full[b], (uint32_t)((k >> 1) & 1), flag) ||
                    !wait_bar(tp_full, (uint32_t)(k & 1), flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint64_t wb = w_desc + (uint64_t)((b * kFWBytes) >> 4);
                for (int mb = 0; mb < nsub; ++mb) {
#pragma unroll
                    for (int ks = 0; ks < kFJB / 8; ++ks)
                        tc::mma_tf32_ts(tmem + (uint32_t)(mb * 32), tmem + kFTpCol + (uint32_t)(mb * kFJB + ks * 8),
                                        wb + (uint64_t)((ks >> 2) * (4096 >> 4) + (ks & 3) * 2), id2, k > 0 || ks > 0);
                }
                tc::commit(tp_empty);
                tc::commit(&w_empty[b]);
            }
            tc::commit(done);
            if (!ok) {
                fail(flag, status);
                // the products already issued finish before the tensor memory is freed
                for (int it = 0; it < kFWaitIters; ++it)
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
            uint32_t r[kFJB];
            const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + kFD1Col + (uint32_t)(b * kFJB);
#pragma unroll
            for (int h = 0; h < kFJB / 16; ++h)
                tc::tmem_ld16(ta + (uint32_t)(h * 16), *reinterpret_cast<uint32_t(*)[16]>(&r[h * 16]));
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&d1_empty[b]);
            if (k >= 2 && !wait_bar(&w_empty[b], (uint32_t)(((k >> 1) - 1) & 1), flag)) {
                fail(flag, status);
                break;
            }
            if (lane < 16) {
                // row l of W^T: fibers 32 a .. 32 a + 31 in the 128-byte row l of atom a
                const int l = quarter * 16 + lane;
#pragma unroll
                for (int at = 0; at < kFJB / 32; ++at) {
                    unsigned char* row = Ws + b * kFWBytes + at * 4096 + (l >> 3) * 1024 + (l & 7) * 128;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *reinterpret_cast<uint4*>(row + ((q ^ (l & 7)) << 4)) =
                            make_uint4(r[32 * at + 4 * q], r[32 * at + 4 * q + 1], r[32 * at + 4 * q + 2],
                                       r[32 * at + 4 * q + 3]);
                }
            }
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&w_full[b]);
        }
    } else {
        // transposers: warp w reaches lanes 32 (w % 4) .. + 31 = rows i of chunk
        // 4 u + w % 4 in block u; the two warps of a quarter take fibers 0-31 and 32-63
        const int quarter = warp & 3, half = (warp - 4) >> 2;
        bool ok = true;
        int64_t g = 0;
        for (int64_t k = 0; k < nloc && ok; ++k) {
            if (k >= 1 && !wait_bar(tp_empty, (uint32_t)((k - 1) & 1), flag)) {
                ok = false;
                break;
            }
            for (int u = 0; u < nsub; ++u, ++g) {
                const int slot = (int)(g % kFStages);
                if (!wait_bar(&full[slot], (uint32_t)((g / kFStages) & 1), flag)) {
                    ok = false;
                    break;
                }
                const int c = u * kFSubChunks + quarter;
                uint32_t v[32];
                if (c < nc) {
                    const unsigned char* src = smem + (size_t)slot * kFSubBytes + quarter * kFBox +
                                               half * 32 * 128 + (lane & 3) * 4;
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        v[j] = *reinterpret_cast<const uint32_t*>(src + j * 128 + (((lane >> 2) ^ (j & 7)) << 4));
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = 0u;
                }
                tc::tmem_st32(tmem + ((uint32_t)(quarter * 32) << 16) + kFTpCol + (uint32_t)(u * kFJB + half * 32), v);
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&empty[slot]);
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tp_full);
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
    if (warp == 3) tc::tmem_dealloc(tmem, kFTmemCols);
}

}  // namespace

bool power_tf32_supported(const ModeView& v, int L) {
    return v.lf == 1 && v.i >= 1 && v.i % 4 == 0 && v.i <= 512 && L >= 1 && L <= 32 &&
           v.fibers() <= (int64_t)INT_MAX - kFJB && tf_layout((int)v.i).bytes <= kFSmemMax;
}

cudaError_t launch_power_tf32(const float* A, const ModeView& v, const float* X_in, int L, float* X_out,
                              void* partials, int* status, int num_sms, cudaStream_t s) {
    if (!power_tf32_supported(v, L) || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return cudaErrorNotSupported;
    const int I = (int)v.i;
    const int64_t J = v.fibers();
    CUtensorMap map;
    const uint64_t dims[2] = {(uint64_t)I, (uint64_t)J};
    const uint64_t strides[1] = {(uint64_t)I * sizeof(float)};
    const uint32_t box[2] = {32, (uint32_t)kFJB};
    if (!tma::make_map_f32(&map, A, 2, dims, strides, box, true)) return cudaErrorNotSupported;
    const TfLayout t = tf_layout(I);
    const int64_t tiles = (J + kFJB - 1) / kFJB;
    int grid = (int)(tiles < num_sms ? tiles : num_sms);
    if (grid < 1) grid = 1;
    float* part = reinterpret_cast<float*>(partials);
    const double elems = (double)I * (double)J;
    {
        ProfScope prof(kKPowerTf32, elems * sizeof(float), 4.0 * elems * L, s);
        cudaFuncSetAttribute(power_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.bytes);
        power_tf32_kernel<<<grid, kFThreads, t.bytes, s>>>(map, I, X_in, L, part, tiles, t.nc, status);
        note_launch();
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce_partials<float>(part, grid, (int64_t)I * L, X_out, s);
}

}  // namespace tk
