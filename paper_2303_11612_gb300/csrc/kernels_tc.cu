// Power step of Strategy A on the 5th-generation tensor cores (tcgen05, BF16
// operands, FP32 accumulation in tensor memory): X_out = A_(n) (A_(n)^T X_in).
//
// Split-BF16 arithmetic: each FP32 entry a of A is held as a_hi + a_lo with
// a_hi = bf16(a) and a_lo = bf16(a - a_hi), which represents a to 2^-16
// relative (bf16 keeps 8 significant bits, rounded to nearest), and the FP32
// product W = T^T X is split the same way. The products
//   W    = T_hi X + T_lo X
//   Xacc += T_hi W_hi + T_lo W_hi + T_hi W_lo          (T_lo W_lo, <= 2^-16, dropped)
// therefore sketch A itself rather than its BF16 rounding (which alone would
// set a relative-error floor near 1e-3), at the same HBM traffic: A is read
// once, in FP32, and the extra tensor-core work stays far below the ridge.
// X_in is rounded to bf16 once: that only replaces the starting block by a
// nearby full-rank one, and the range of A A^T X is still a sketch of A.
//
// Each CTA streams tiles of 64 mode-n fibers. A tile T (64 fibers x I_n) is
// converted into two shared-memory buffers (hi, lo) in the no-swizzle
// core-matrix layout, which serve both products:
//   W    = T X     (M = 64 fibers, N = L, K = I_n)       accumulator in TMEM
//   Xacc += T^T W  (M = 128 rows of I_n per block, K = 64 fibers)
// For contiguous fibers (mode 1) the buffers are K-major for the first product
// and MN-major for the second; for strided fibers it is the other way round.
// With M = 64, accumulator row m sits in TMEM lane (m % 16) + 32 (m / 16).
// W travels TMEM -> registers -> bf16 shared memory to become the second
// product's B operand. X_acc stays in TMEM across all tiles of the CTA and is
// written once as the CTA's partial; partials are summed in a fixed order.
// Every mbarrier wait is bounded: on a timeout the kernel records
// kStatTimeout, frees its tensor memory and stops.
#include "internal.h"
#include "tc.cuh"

namespace tk {
namespace {

constexpr int kTcThreads = 256;
constexpr int kJB = 64;                  // fibers per tile (M of the first product)
// Descriptor convention for MN-major operands: LBO is the stride between core
// matrices along K, SBO the stride along M/N (checked on the device).
constexpr bool kMnLboIsK = true;
constexpr int kWaitIters = 1 << 24;

__host__ __device__ __forceinline__ int round_up(int x, int m) { return (x + m - 1) / m * m; }

__device__ __forceinline__ uint32_t t_off(bool contig, int jj, int i, int ipt) {
    return contig ? (uint32_t)((jj >> 3) * (ipt >> 3) * 128 + (i >> 3) * 128 + (jj & 7) * 16 + (i & 7) * 2)
                  : (uint32_t)((i >> 3) * (kJB >> 3) * 128 + (jj >> 3) * 128 + (i & 7) * 16 + (jj & 7) * 2);
}

__device__ __forceinline__ uint32_t bf2(float a, float b) {
    __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&p);
}
// Eight FP32 values -> their bf16 high parts and bf16 low parts (x - hi).
__device__ __forceinline__ void pack8_split(const float* x, uint4& hi, uint4& lo) {
    float r[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = x[k] - __bfloat162float(__float2bfloat16_rn(x[k]));
    hi = make_uint4(bf2(x[0], x[1]), bf2(x[2], x[3]), bf2(x[4], x[5]), bf2(x[6], x[7]));
    lo = make_uint4(bf2(r[0], r[1]), bf2(r[2], r[3]), bf2(r[4], r[5]), bf2(r[6], r[7]));
}

// Loads are issued in batches of kBatch chunks per thread before any of them is
// converted and stored, so that enough bytes are in flight to cover HBM latency
// with one CTA per SM.
constexpr int kBatch = 8;

template <bool CONTIG>
__device__ __forceinline__ void load_tile_bf16(const float* __restrict__ A, const ModeView& v, int64_t j0, int64_t J,
                                               unsigned char* T, unsigned char* Tlo, int ipt, const int64_t* bases,
                                               bool vec4) {
    const int I = (int)v.i;
    const int tid = threadIdx.x;
    if (CONTIG) {
        // chunk = 8 consecutive elements of one fiber; 8 neighbouring threads take 8
        // fibers so that their 16-byte stores fill a whole core matrix
        const int n8 = ipt >> 3;
        const int nchunks = kJB * n8;
        for (int e0 = tid; e0 < nchunks; e0 += kTcThreads * kBatch) {
            float x[kBatch][8];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int e = e0 + u * kTcThreads;
                const int jlo = e & 7, rest = e >> 3;
                const int i8 = rest % n8, jj = (rest / n8) * 8 + jlo;
                const int64_t j = j0 + jj;
                const int i0 = i8 * 8;
                if (e < nchunks && j < J && i0 + 8 <= I && vec4) {
                    const float4* src = reinterpret_cast<const float4*>(A + j * (int64_t)I + i0);
                    const float4 a = __ldg(src), b = __ldg(src + 1);
                    x[u][0] = a.x; x[u][1] = a.y; x[u][2] = a.z; x[u][3] = a.w;
                    x[u][4] = b.x; x[u][5] = b.y; x[u][6] = b.z; x[u][7] = b.w;
                } else {
#pragma unroll
                    for (int w = 0; w < 8; ++w)
                        x[u][w] = (e < nchunks && j < J && i0 + w < I) ? __ldg(A + j * (int64_t)I + i0 + w) : 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int e = e0 + u * kTcThreads;
                if (e < nchunks) {
                    const int jlo = e & 7, rest = e >> 3;
                    const int i8 = rest % n8, jj = (rest / n8) * 8 + jlo;
                    const uint32_t o = t_off(true, jj, i8 * 8, ipt);
                    uint4 h, l;
                    pack8_split(x[u], h, l);
                    *reinterpret_cast<uint4*>(T + o) = h;
                    *reinterpret_cast<uint4*>(Tlo + o) = l;
                }
            }
        }
    } else {
        // chunk = one element of 8 consecutive fibers; 8 neighbouring threads take 8
        // consecutive rows i of the same core matrix
        const int nchunks = (kJB >> 3) * ipt;
        const int64_t lf = v.lf;
        constexpr int kB = kBatch / 2;
        for (int e0 = tid; e0 < nchunks; e0 += kTcThreads * kB) {
            float x[kB][8];
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int e = e0 + u * kTcThreads;
                const int ilo = e & 7, rest = e >> 3;
                const int j8 = rest % (kJB >> 3), i = (rest / (kJB >> 3)) * 8 + ilo;
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    const int64_t b = e < nchunks ? bases[j8 * 8 + w] : -1;
                    x[u][w] = (b >= 0 && i < I) ? __ldg(A + b + (int64_t)i * lf) : 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int e = e0 + u * kTcThreads;
                if (e < nchunks) {
                    const int ilo = e & 7, rest = e >> 3;
                    const int j8 = rest % (kJB >> 3), i = (rest / (kJB >> 3)) * 8 + ilo;
                    const uint32_t o = t_off(false, j8 * 8, i, ipt);
                    uint4 h, l;
                    pack8_split(x[u], h, l);
                    *reinterpret_cast<uint4*>(T + o) = h;
                    *reinterpret_cast<uint4*>(Tlo + o) = l;
                }
            }
        }
    }
}

template <bool CONTIG, int LP>
__global__ void __launch_bounds__(kTcThreads, 1) power_tc_kernel(const float* __restrict__ A, ModeView v,
                                                                 const float* __restrict__ X, int L,
                                                                 float* __restrict__ partial, int64_t tiles,
                                                                 int* status, int vec4) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int I = (int)v.i;
    const int nb = (I + 127) / 128;                 // 128-row blocks of I_n
    const int ipt = nb * 128;                       // padded I_n of the tile and X buffers
    const int64_t J = v.fibers();
    unsigned char* T = smem;                                        // kJB x ipt bf16, high parts
    unsigned char* Tlo = T + (size_t)kJB * ipt * 2;                 // kJB x ipt bf16, low parts
    unsigned char* Xs = Tlo + (size_t)kJB * ipt * 2;                // LP x ipt bf16
    unsigned char* Ws = Xs + (size_t)LP * ipt * 2;                  // LP x kJB bf16, high parts
    unsigned char* Wlo = Ws + (size_t)LP * kJB * 2;                 // LP x kJB bf16, low parts
    const size_t used = ((size_t)2 * kJB * ipt + (size_t)LP * ipt + (size_t)2 * LP * kJB) * 2;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + used);      // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
    int* flag = reinterpret_cast<int*>(tmem_slot + 1);
    int64_t* bases = reinterpret_cast<int64_t*>(smem + used + 64);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, half = warp >> 2;

    // X_in -> bf16 B operand of the first product: (N = l, K = i), K-major
    for (int e = tid; e < LP * ipt; e += kTcThreads) {
        const int l = e / ipt, i = e % ipt;
        const float x = (l < L && i < I) ? X[(int64_t)l * I + i] : 0.f;
        *reinterpret_cast<__nv_bfloat16*>(Xs + (l >> 3) * (ipt >> 3) * 128 + (i >> 3) * 128 + (l & 7) * 16 + (i & 7) * 2) =
            __float2bfloat16_rn(x);
    }
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(LP * (1 + nb))) ncols <<= 1;
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        *flag = 0;
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, ncols);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    const uint32_t t_base = tc::smem_u32(T), x_base = tc::smem_u32(Xs), w_base = tc::smem_u32(Ws);
    const uint32_t tlo_off = (uint32_t)(Tlo - T), wlo_off = (uint32_t)(Wlo - Ws);
    const uint32_t id1 = tc::idesc_bf16(kJB, LP, !CONTIG, false);
    const uint32_t id2 = tc::idesc_bf16(128, LP, CONTIG, false);
    const uint32_t kdir_t = CONTIG ? 128u : (uint32_t)(kJB / 8) * 128u;        // i-group stride in T
    const uint32_t jdir_t = CONTIG ? (uint32_t)(ipt / 8) * 128u : 128u;        // fiber-group stride in T
    const uint32_t xsbo = (uint32_t)(ipt / 8) * 128u;

    int it = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++it) {
        const int64_t j0 = tile * kJB;
        if (!CONTIG && tid < kJB) {
            const int64_t j = j0 + tid;
            bases[tid] = j < J ? v.base(j) : -1;
        }
        __syncthreads();
        load_tile_bf16<CONTIG>(A, v, j0, J, T, Tlo, ipt, bases, vec4 != 0);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            // W = T_hi X + T_lo X: K runs over I_n in steps of 16 (two core matrices)
            for (int part = 0; part < 2; ++part) {
                const uint32_t tb = t_base + (part ? tlo_off : 0u);
                for (int s = 0; s < ipt / 16; ++s) {
                    uint64_t a;
                    if (CONTIG) a = tc::desc(tb + s * 2 * kdir_t, kdir_t, jdir_t);      // K-major
                    else a = kMnLboIsK ? tc::desc(tb + s * 2 * kdir_t, kdir_t, jdir_t)  // MN-major
                                       : tc::desc(tb + s * 2 * kdir_t, jdir_t, kdir_t);
                    const uint64_t b = tc::desc(x_base + s * 256, 128, xsbo);
                    tc::mma_bf16(tmem, a, b, id1, part > 0 || s > 0);
                }
            }
            tc::commit(&mbar[0]);
            if (!tc::mbar_wait(&mbar[0], it & 1, kWaitIters)) { *flag = 1; set_status(status, kStatTimeout); }
        }
        __syncthreads();
        if (*flag) { ok = false; break; }
        tc::fence_after_sync();
        // W (TMEM: fiber m in lane (m % 16) + 32 (m / 16), columns = l) -> bf16 high
        // and low B operands (N = l, K = fiber), K-major. Warp q reads lanes
        // 32 q .. 32 q + 31, of which the first 16 hold fibers 16 q .. 16 q + 15.
        for (int c = half; c < LP / 16; c += 2) {
            uint32_t r[16];
            tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * 16), r);
            const int jj = q * 16 + lane;
            if (lane < 16) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int l = c * 16 + u;
                    const uint32_t o = (l >> 3) * (kJB >> 3) * 128 + (jj >> 3) * 128 + (l & 7) * 16 + (jj & 7) * 2;
                    const float w = __uint_as_float(r[u]);
                    const __nv_bfloat16 h = __float2bfloat16_rn(w);
                    *reinterpret_cast<__nv_bfloat16*>(Ws + o) = h;
                    *reinterpret_cast<__nv_bfloat16*>(Wlo + o) = __float2bfloat16_rn(w - __bfloat162float(h));
                }
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            // X_acc[b] += T_hi W_hi + T_lo W_hi + T_hi W_lo: K runs over the fibers in steps of 16
            for (int b = 0; b < nb; ++b) {
                for (int part = 0; part < 3; ++part) {
                    const uint32_t ta = t_base + (part == 1 ? tlo_off : 0u);
                    const uint32_t wb = w_base + (part == 2 ? wlo_off : 0u);
                    for (int s = 0; s < kJB / 16; ++s) {
                        const uint32_t start = ta + b * 16 * kdir_t + s * 2 * jdir_t;
                        uint64_t a;
                        if (CONTIG) a = kMnLboIsK ? tc::desc(start, jdir_t, kdir_t) : tc::desc(start, kdir_t, jdir_t);
                        else a = tc::desc(start, jdir_t, kdir_t);                        // K-major
                        const uint64_t bd = tc::desc(wb + s * 256, 128, (uint32_t)(kJB / 8) * 128u);
                        tc::mma_bf16(tmem + (uint32_t)(LP * (1 + b)), a, bd, id2, it > 0 || part > 0 || s > 0);
                    }
                }
            }
            tc::commit(&mbar[1]);
            // T and Ws are reused by the next tile: wait for these products to finish
            if (!tc::mbar_wait(&mbar[1], it & 1, kWaitIters)) { *flag = 1; set_status(status, kStatTimeout); }
        }
        __syncthreads();
        if (*flag) { ok = false; break; }
    }
    tc::fence_after_sync();
    float* out = partial + (int64_t)blockIdx.x * ((int64_t)I * L);
    if (ok) {
        for (int b = 0; b < nb; ++b) {
            for (int c = half; c < LP / 16; c += 2) {
                const int i = b * 128 + q * 32 + lane;
                uint32_t r[16];
                if (it > 0) tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(LP * (1 + b) + c * 16), r);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int l = c * 16 + u;
                    if (i < I && l < L) out[(int64_t)l * I + i] = it > 0 ? __uint_as_float(r[u]) : 0.f;
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

size_t tc_smem_bytes(int I, int LP) {
    const int ipt = round_up(I, 128);
    return ((size_t)2 * kJB * ipt + (size_t)LP * ipt + (size_t)2 * LP * kJB) * 2 + 64 + sizeof(int64_t) * kJB + 64;
}

template <bool CONTIG, int LP>
cudaError_t launch_tc_t(const float* A, const ModeView& v, const float* X, int L, float* partials, int grid,
                        int64_t tiles, int* status, cudaStream_t s) {
    auto k = power_tc_kernel<CONTIG, LP>;
    const size_t smem = tc_smem_bytes((int)v.i, LP);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int vec4 = (v.i % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    k<<<grid, kTcThreads, smem, s>>>(A, v, X, L, partials, tiles, status, vec4);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

bool power_tc_supported(const ModeView& v, int L) {
    return v.i <= 512 && L >= 1 && L <= 64 && tc_smem_bytes((int)v.i, round_up(L, 16)) <= 220 * 1024;
}

size_t power_tc_partials_bytes(const ModeView& v, int L, int num_sms) {
    return (size_t)num_sms * (size_t)v.i * (size_t)L * sizeof(float);
}

cudaError_t launch_power_tc(const float* A, const ModeView& v, const float* X_in, int L, float* X_out, void* partials,
                            int* status, int num_sms, cudaStream_t s) {
    const int64_t tiles = (v.fibers() + kJB - 1) / kJB;
    int grid = (int)(tiles < num_sms ? tiles : num_sms);
    if (grid < 1) grid = 1;
    float* part = reinterpret_cast<float*>(partials);
    const int LP = round_up(L, 16);
    const bool contig = v.lf == 1;
    const double elems = (double)v.i * (double)v.fibers();
    cudaError_t e;
    {
        ProfScope prof(kKPowerBf16, elems * sizeof(float), 4.0 * elems * L, s);
        switch (LP) {
            case 16: e = contig ? launch_tc_t<true, 16>(A, v, X_in, L, part, grid, tiles, status, s)
                                : launch_tc_t<false, 16>(A, v, X_in, L, part, grid, tiles, status, s); break;
            case 32: e = contig ? launch_tc_t<true, 32>(A, v, X_in, L, part, grid, tiles, status, s)
                                : launch_tc_t<false, 32>(A, v, X_in, L, part, grid, tiles, status, s); break;
            case 48: e = contig ? launch_tc_t<true, 48>(A, v, X_in, L, part, grid, tiles, status, s)
                                : launch_tc_t<false, 48>(A, v, X_in, L, part, grid, tiles, status, s); break;
            case 64: e = contig ? launch_tc_t<true, 64>(A, v, X_in, L, part, grid, tiles, status, s)
                                : launch_tc_t<false, 64>(A, v, X_in, L, part, grid, tiles, status, s); break;
            default: return cudaErrorInvalidValue;
        }
    }
    if (e != cudaSuccess) return e;
    return launch_reduce_partials<float>(part, grid, v.i * (int64_t)L, X_out, s);
}

}  // namespace tk
