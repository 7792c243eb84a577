// Mode-n product on the 5th-generation tensor cores for contiguous fibers
// (mode 1), split-BF16 operands with FP32 accumulation in tensor memory:
//   out[j, o] = sum_i A_(n)[i, j] M[i, o]     (the truncation B x_n U^T of
//                                              Algorithm 2 with M = U).
// Each FP32 value a is held as a_hi + a_lo with a_hi = bf16(a) and
// a_lo = bf16(a - a_hi), which represents a to 2^-16 relative (bf16 keeps 8
// significant bits, rounded to nearest), M the same way, and
//   D = A_hi M_hi + A_lo M_hi + A_hi M_lo          (A_lo M_lo, <= 2^-16, dropped)
// so each term is of a and m themselves to about 3 x 2^-16, with unbiased
// (round-to-nearest) splitting; bf16 x bf16 products are exact in FP32.
//
// A tile is 128 fibers (M of the product, one fiber per accumulator lane); it
// streams through units of 64 values i. TMA loads a unit as two FP32 boxes of
// 32 values x 128 fibers in the 128-byte-swizzled layout; sixteen converter warps
// rewrite it as bf16 high and low parts in the K-major swizzled layout of the
// product (one 128-byte row of 64 values per fiber); the MMA thread issues
// 4 K-steps x 3 products per unit into the tile's accumulator (N = 32 columns
// for the K_out <= 32 outputs, double-buffered), and four warps read finished
// accumulators back and store the tile's outputs.
//
// Warp roles: warp 0 TMA, warp 1 MMA (and tensor-memory allocation), warps 2-17
// conversion, warps 18-21 read-back. Every mbarrier wait is bounded: on a
// timeout the kernel records kStatTimeout, lets the copies and products it
// issued finish (with the same bound), frees its tensor memory and returns.
#include <climits>

#include "internal.h"
#include "tc.cuh"
#include "tma.cuh"

namespace tk {
namespace {

constexpr int kGThreads = 64 + 32 * 16 + 32 * 4;  // TMA, MMA, 16 converter and 4 read-back warps
constexpr int kGJB = 128;                  // fibers per tile
constexpr int kGBox = kGJB * 128;          // FP32 box: 32 values i x 128 fibers
constexpr int kGUnit = 2 * kGBox;          // FP32 unit: 64 values i
constexpr int kGHalf = kGJB * 128;         // one bf16 part of a unit: 64 values i x 128 fibers
constexpr int kGFStages = 3;               // FP32 units in the TMA ring
constexpr int kGCStages = 2;               // converted units
constexpr int kGConv = (kGThreads - 64 - 128) / 32;   // converter warps 2 .. 2 + kGConv - 1
constexpr int kGEpi = 4;                   // read-back warps 10 .. 13
constexpr int kGUChunk = 32 * 128;         // one unit of one part of M^T: 32 rows o x 128 bytes
constexpr int kGWaitIters = 1 << 22;
constexpr size_t kGSmemMax = 227 * 1024;
constexpr uint32_t kGTmemCols = 64;
constexpr int kGBars = 2 * kGFStages + 2 * kGCStages + 5;    // 8 bytes each, 256 reserved
static_assert(kGBars * 8 + 8 <= 256, "barrier area");

struct TtmTcLayout {
    int nu = 0;                // units of 64 values i
    size_t c_off = 0, u_off = 0, bar_off = 0, bytes = 0;
};

TtmTcLayout ttm_tc_layout(int I) {
    TtmTcLayout t;
    t.nu = (I + 63) / 64;
    t.c_off = (size_t)kGFStages * kGUnit;
    t.u_off = t.c_off + (size_t)kGCStages * 2 * kGHalf;
    t.bar_off = t.u_off + (size_t)2 * t.nu * kGUChunk;
    t.bytes = t.bar_off + 256 + 1024;
    return t;
}

__device__ __forceinline__ bool wait_bar(uint64_t* b, uint32_t parity, volatile int* flag) {
    for (int it = 0; it < kGWaitIters; ++it) {
        if (tc::mbar_try(b, parity)) return true;
        if ((it & 255) == 255 && *flag) return false;
    }
    return false;
}

__device__ __forceinline__ void fail(volatile int* flag, int* status) {
    *flag = 1;
    set_status(status, kStatTimeout);
}

__device__ __forceinline__ uint32_t bf2(float a, float b) {
    __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&p);
}

// Two FP32 values -> their bf16 high parts (packed, round to nearest) and the
// bf16 low parts of the remainders x - hi (exact in FP32); a packed bf16 value
// widens to FP32 by a 16-bit shift.
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    hi = bf2(a, b);
    const float ha = __uint_as_float(hi << 16), hb = __uint_as_float(hi & 0xFFFF0000u);
    lo = bf2(a - ha, b - hb);
}

// Eight FP32 values -> bf16 high parts and bf16 low parts (x - hi), packed in order.
__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo) {
    split2(x[0], x[1], hi.x, lo.x);
    split2(x[2], x[3], hi.y, lo.y);
    split2(x[4], x[5], hi.z, lo.z);
    split2(x[6], x[7], hi.w, lo.w);
}

__global__ void __launch_bounds__(kGThreads, 1)
    ttm_tc_kernel(const __grid_constant__ CUtensorMap map, int I, int64_t J, const float* __restrict__ Mp,
                  int K_out, int64_t ld_i, int64_t ld_k, float* __restrict__ out, int64_t tiles, int nu,
                  int* status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // swizzled buffers start on 1024-byte boundaries (the launch adds 1 KB of slack)
    unsigned char* smem = smem_raw + ((1024 - (tma::smem_addr(smem_raw) & 1023)) & 1023);
    unsigned char* F = smem;                                            // [3] FP32 units
    unsigned char* Cb = smem + (size_t)kGFStages * kGUnit;              // [2] (hi, lo) bf16 units
    unsigned char* Us = Cb + (size_t)kGCStages * 2 * kGHalf;            // M^T hi [nu], then lo [nu]
    uint64_t* bar = reinterpret_cast<uint64_t*>(Us + (size_t)2 * nu * kGUChunk);
    uint64_t* f_full = bar;                          // FP32 unit loaded (TMA bytes)
    uint64_t* f_empty = f_full + kGFStages;          // FP32 unit converted (converter warps)
    uint64_t* c_full = f_empty + kGFStages;          // bf16 unit written (converter warps)
    uint64_t* c_empty = c_full + kGCStages;          // bf16 unit consumed by the products
    uint64_t* d_full = c_empty + kGCStages;          // [2] tile accumulated
    uint64_t* d_empty = d_full + 2;                  // [2] tile read back (4 warps)
    uint64_t* done = d_empty + 2;                    // every product done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nloc = tiles > (int64_t)blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    // M^T split, K-major swizzled bf16: unit u, row o, 16-byte group q (values
    // i = 64 u + 8 q .. + 7) at group position q ^ (o % 8); zero beyond K_out and I
    for (int e = tid; e < 32 * nu * 8; e += kGThreads) {
        const int o = e / (nu * 8), rem = e - o * (nu * 8), u = rem >> 3, q = rem & 7;
        float x[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int i = 64 * u + 8 * q + w;
            x[w] = (o < K_out && i < I) ? __ldg(Mp + (int64_t)i * ld_i + (int64_t)o * ld_k) : 0.f;
        }
        uint4 hi, lo;
        split8(x, hi, lo);
        const int off = u * kGUChunk + (o >> 3) * 1024 + (o & 7) * 128 + ((q ^ (o & 7)) << 4);
        *reinterpret_cast<uint4*>(Us + off) = hi;
        *reinterpret_cast<uint4*>(Us + (size_t)nu * kGUChunk + off) = lo;
    }
    if (tid == 0) {
        for (int k = 0; k < kGBars; ++k) tc::mbar_init(&bar[k], 1);
        for (int k = 0; k < kGFStages; ++k) tc::mbar_init(&f_empty[k], kGConv);
        for (int k = 0; k < kGCStages; ++k) tc::mbar_init(&c_full[k], kGConv);
        for (int k = 0; k < 2; ++k) tc::mbar_init(&d_empty[k], kGEpi);
        *flag = 0;
        tma::fence_barrier_init();
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, kGTmemCols);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int64_t g = 0;
            bool ok = true;
            for (int64_t k = 0; k < nloc && ok; ++k) {
                const int j0 = (int)((blockIdx.x + k * gridDim.x) * kGJB);
                for (int u = 0; u < nu; ++u, ++g) {
                    const int fs = (int)(g % kGFStages);
                    if (g >= kGFStages && !wait_bar(&f_empty[fs], (uint32_t)((g / kGFStages - 1) & 1), flag)) {
                        fail(flag, status);
                        ok = false;
                        break;
                    }
                    tma::expect_tx(&f_full[fs], (uint32_t)kGUnit);
                    unsigned char* dst = F + (size_t)fs * kGUnit;
                    // the second box may lie wholly beyond I_n: it then loads zeros
                    tma::load_2d(dst, &map, 64 * u, j0, &f_full[fs]);
                    tma::load_2d(dst + kGBox, &map, 64 * u + 32, j0, &f_full[fs]);
                }
            }
            if (*flag) {
                const int64_t g0 = g > kGFStages ? g - kGFStages : 0;
                for (int64_t gg = g0; gg < g; ++gg)
                    for (int it = 0; it < kGWaitIters; ++it)
                        if (tc::mbar_try(&f_full[gg % kGFStages], (uint32_t)((gg / kGFStages) & 1))) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id = tc::idesc_bf16(128, 32, false, false);
            const uint64_t c_desc = tc::desc_sw128(tc::smem_u32(Cb), 16, 1024);
            const uint64_t u_desc = tc::desc_sw128(tc::smem_u32(Us), 16, 1024);
            const uint64_t lo_step = (uint64_t)(kGHalf >> 4), ulo_step = (uint64_t)((nu * kGUChunk) >> 4);
            bool ok = true;
            int64_t g = 0;
            for (int64_t k = 0; k < nloc && ok; ++k) {
                const int b = (int)(k & 1);
                if (k >= 2 && !wait_bar(&d_empty[b], (uint32_t)(((k >> 1) - 1) & 1), flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d = tmem + (uint32_t)(b * 32);
                for (int u = 0; u < nu; ++u, ++g) {
                    const int cs = (int)(g % kGCStages);
                    if (!wait_bar(&c_full[cs], (uint32_t)((g / kGCStages) & 1), flag)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint64_t ahi = c_desc + (uint64_t)((cs * 2 * kGHalf) >> 4), alo = ahi + lo_step;
                    const uint64_t bhi = u_desc + (uint64_t)((u * kGUChunk) >> 4), blo = bhi + ulo_step;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t s2 = (uint64_t)(ks * 2);
                        tc::mma_bf16(d, ahi + s2, bhi + s2, id, u > 0 || ks > 0);
                        tc::mma_bf16(d, alo + s2, bhi + s2, id, true);
                        tc::mma_bf16(d, ahi + s2, blo + s2, id, true);
                    }
                    tc::commit(&c_empty[cs]);
                }
                if (!ok) break;
                tc::commit(&d_full[b]);
            }
            tc::commit(done);
            if (!ok) {
                fail(flag, status);
                for (int it = 0; it < kGWaitIters; ++it)
                    if (tc::mbar_try(done, 0)) break;
            }
        }
    } else if (warp < 2 + kGConv) {
        // conversion: task t = (fiber j, group p of 8 values i of the unit); a
        // group is two 16-byte pieces of FP32 box p / 4 and one 16-byte piece of
        // each bf16 part
        const int ct = tid - 64;
        bool ok = true;
        int64_t g = 0;
        for (int64_t k = 0; k < nloc && ok; ++k) {
            for (int u = 0; u < nu; ++u, ++g) {
                const int fs = (int)(g % kGFStages), cs = (int)(g % kGCStages);
                if (!wait_bar(&f_full[fs], (uint32_t)((g / kGFStages) & 1), flag)) {
                    ok = false;
                    break;
                }
                // split into registers first (this consumes the loads), release the
                // FP32 slot to the TMA at once, then store once a bf16 slot is free
                constexpr int kTasks = (kGJB * 8) / (kGConv * 32);
                const unsigned char* src = F + (size_t)fs * kGUnit;
                uint4 hi[kTasks], lo[kTasks];
#pragma unroll
                for (int r = 0; r < kTasks; ++r) {
                    const int t = ct + kGConv * 32 * r;
                    const int j = t >> 3, p = t & 7;
                    const int q0 = (p & 3) * 2;
                    const unsigned char* row = src + (p >> 2) * kGBox + j * 128;
                    const float4 a = *reinterpret_cast<const float4*>(row + ((q0 ^ (j & 7)) << 4));
                    const float4 c = *reinterpret_cast<const float4*>(row + (((q0 + 1) ^ (j & 7)) << 4));
                    const float x[8] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
                    split8(x, hi[r], lo[r]);
                }
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&f_empty[fs]);
                if (g >= kGCStages && !wait_bar(&c_empty[cs], (uint32_t)((g / kGCStages - 1) & 1), flag)) {
                    ok = false;
                    break;
                }
                unsigned char* dhi = Cb + (size_t)cs * 2 * kGHalf;
#pragma unroll
                for (int r = 0; r < kTasks; ++r) {
                    const int t = ct + kGConv * 32 * r;
                    const int j = t >> 3, p = t & 7;
                    const int off = j * 128 + ((p ^ (j & 7)) << 4);
                    *reinterpret_cast<uint4*>(dhi + off) = hi[r];
                    *reinterpret_cast<uint4*>(dhi + kGHalf + off) = lo[r];
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
            uint32_t r[32];
            const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 32);
            tc::tmem_ld16(ta, *reinterpret_cast<uint32_t(*)[16]>(&r[0]));
            tc::tmem_ld16(ta + 16, *reinterpret_cast<uint32_t(*)[16]>(&r[16]));
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&d_empty[b]);
            const int64_t j = (blockIdx.x + k * gridDim.x) * kGJB + quarter * 32 + lane;
            if (j < J) {
                float* o = out + j * K_out;
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (c < K_out) o[c] = __uint_as_float(r[c]);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, kGTmemCols);
}

}  // namespace

bool ttm_tc_supported(const ModeView& v, int64_t K_out) {
    return v.lf == 1 && v.i >= 1 && v.i % 4 == 0 && v.i <= 512 && K_out >= 1 && K_out <= 32 &&
           v.fibers() <= (int64_t)INT_MAX - kGJB && ttm_tc_layout((int)v.i).bytes <= kGSmemMax;
}

cudaError_t launch_ttm_tc(const float* A, const ModeView& v, const float* Mp, int64_t K_out, int64_t ld_i,
                          int64_t ld_k, float* out, int* status, int num_sms, cudaStream_t s) {
    if (!ttm_tc_supported(v, K_out) || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return cudaErrorNotSupported;
    const int I = (int)v.i;
    const int64_t J = v.fibers();
    CUtensorMap map;
    const uint64_t dims[2] = {(uint64_t)I, (uint64_t)J};
    const uint64_t strides[1] = {(uint64_t)I * sizeof(float)};
    const uint32_t box[2] = {32, (uint32_t)kGJB};
    if (!tma::make_map_f32(&map, A, 2, dims, strides, box, true)) return cudaErrorNotSupported;
    const TtmTcLayout t = ttm_tc_layout(I);
    const int64_t tiles = (J + kGJB - 1) / kGJB;
    int grid = (int)(tiles < num_sms ? tiles : num_sms);
    if (grid < 1) grid = 1;
    const double elems = (double)I * (double)J;
    ProfScope prof(kKTtmBf16, (elems + (double)J * K_out) * sizeof(float), 2.0 * elems * K_out, s);
    cudaFuncSetAttribute(ttm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.bytes);
    ttm_tc_kernel<<<grid, kGThreads, t.bytes, s>>>(map, I, J, Mp, (int)K_out, ld_i, ld_k, out, tiles, t.nu, status);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tk
