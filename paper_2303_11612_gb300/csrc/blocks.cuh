// Block programs of the streaming steps, shared by their own kernels and by the
// work-list kernel of batched runs (worklist.cu). Each takes its block's
// coordinates as arguments instead of reading blockIdx / gridDim, so the same
// code computes the same block of results whichever kernel runs it: the
// Gaussian test matrix (Alg. 1), the fused power step of Strategy A (remark
// after Alg. 1), the fixed-order sum of its per-CTA partials and the
// register-staged mode-n product (Section 2).
//
// NC selects the load path for data another CTA may have written: true reads
// through the read-only cache (the data are fixed for the kernel's lifetime);
// false reads at L2 (__ldcg), as the work-list kernel must for data that items
// earlier in the same launch produced.
#pragma once

#include "common.cuh"

namespace tk {
namespace blk {

template <bool NC, typename T> __device__ __forceinline__ T ld(const T* p) {
    if constexpr (NC) return __ldg(p);
    else return __ldcg(p);
}

// ---------------------------------------------------------------- Gaussian test matrix
// out (rows x cols, column-major) from the Philox stream; block bid of nblk
// takes the entries bid * kThreads + k nblk kThreads (any split gives the same matrix).
template <typename T>
__device__ __forceinline__ void gaussian_block(T* __restrict__ out, int64_t rows, int64_t cols, uint64_t seed,
                                               uint32_t stream_id, int64_t bid, int64_t nblk) {
    const int64_t n = rows * cols;
    for (int64_t k = bid * kThreads + threadIdx.x; k < n; k += nblk * kThreads) {
        const int64_t l = k / rows, i = k - l * rows;      // column-major position
        out[k] = gaussian_at<T>(seed, stream_id, (uint64_t)(i * cols + l));
    }
}

// ---------------------------------------------------------------- power step
// Loads the JB x I tile of fibers j0 .. j0+JB-1 into Ts (row stride ldt).
template <typename T, int JB, bool NC>
__device__ __forceinline__ void load_tile(const T* __restrict__ A, const ModeView& v, int64_t j0, int64_t J, T* Ts,
                                          int ldt, int64_t* bases) {
    constexpr int kT = kThreads;
    const int I = (int)v.i;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (v.lf == 1) {
        // fibers are contiguous runs of I elements
        for (int jj = warp; jj < JB; jj += kT / 32) {
            const int64_t j = j0 + jj;
            T* dst = Ts + jj * ldt;
            if (j < J) {
                const T* src = A + j * (int64_t)I;
                for (int i = lane; i < I; i += 32) dst[i] = ld<NC>(src + i);
            } else {
                for (int i = lane; i < I; i += 32) dst[i] = T(0);
            }
        }
    } else {
        if (tid < JB) {
            const int64_t j = j0 + tid;
            bases[tid] = j < J ? v.base(j) : -1;
        }
        __syncthreads();
        const int64_t lf = v.lf;
        for (int e = tid; e < JB * I; e += kT) {
            const int jj = e % JB, i = e / JB;
            const int64_t b = bases[jj];
            Ts[jj * ldt + i] = b >= 0 ? ld<NC>(A + b + (int64_t)i * lf) : T(0);
        }
    }
}

// Shared-memory bytes of one power-step block.
template <typename T, int JB, int LG, bool RANGE>
__host__ __device__ constexpr size_t power_block_smem(int I) {
    return sizeof(T) * ((RANGE ? 0 : (size_t)I * LG) + (size_t)JB * (size_t)(I | 1) + (size_t)(kThreads / JB) * JB * LG +
                        (size_t)JB * LG) + sizeof(int64_t) * JB + 16;
}

// Columns gx * LG .. of X_out over the tiles ty, ty + ny, ... of JB fibers:
//   W = T X        (JB x LG)   phase 1, split over I_n and reduced in smem
//   X_acc += T^T W (I_n x LG)  phase 2, accumulated in registers
// written to partial[ty] (I_n x L). RANGE: W = Omega rows generated by Philox.
template <typename T, int JB, int LG, int KR, bool RANGE, bool NC>
__device__ __forceinline__ void power_block(const T* __restrict__ A, const ModeView& v, const T* __restrict__ X,
                                            int L, T* __restrict__ partial, int64_t tiles, uint64_t seed,
                                            uint32_t stream_id, int gx, int64_t ty, int64_t ny,
                                            unsigned char* smem_raw) {
    constexpr int kT = kThreads;
    constexpr int KS = kT / JB;            // phase-1 split of the I dimension
    const int I = (int)v.i;
    const int64_t J = v.fibers();
    const int l0 = gx * LG;
    const int lg = min(LG, L - l0);
    const int ldt = I | 1;                 // odd row stride: conflict-free column reads
    T* Xs = reinterpret_cast<T*>(smem_raw);               // [I][LG]
    T* Ts = Xs + (RANGE ? 0 : I * LG);                     // [JB][ldt]
    T* Wp = Ts + JB * ldt;                                 // [KS][JB][LG]
    T* Ws = Wp + KS * JB * LG;                             // [JB][LG]
    int64_t* bases = reinterpret_cast<int64_t*>(Ws + JB * LG);
    const int tid = threadIdx.x;

    if (!RANGE) {
        for (int e = tid; e < I * LG; e += kT) {
            const int i = e / LG, l = e % LG;
            Xs[e] = l < lg ? (NC ? X[(int64_t)(l0 + l) * I + i] : ld<false>(X + (int64_t)(l0 + l) * I + i)) : T(0);
        }
    }
    T acc2[KR][LG];
#pragma unroll
    for (int k = 0; k < KR; ++k)
#pragma unroll
        for (int l = 0; l < LG; ++l) acc2[k][l] = T(0);

    for (int64_t tile = ty; tile < tiles; tile += ny) {
        const int64_t j0 = tile * JB;
        __syncthreads();                    // previous tile fully consumed
        load_tile<T, JB, NC>(A, v, j0, J, Ts, ldt, bases);
        if (RANGE) {
            for (int e = tid; e < JB * LG; e += kT) {
                const int jj = e / LG, l = e % LG;
                const int64_t j = j0 + jj;
                Ws[e] = (j < J && l < lg)
                            ? gaussian_at<T>(seed, stream_id, (uint64_t)(j * L + l0 + l))
                            : T(0);
            }
            __syncthreads();
        } else {
            __syncthreads();
            // phase 1: W(jj, :) partial over this thread's slice of I
            const int jj = tid % JB, ks = tid / JB;
            const int ib = (int)((int64_t)I * ks / KS), ie = (int)((int64_t)I * (ks + 1) / KS);
            T acc[LG];
#pragma unroll
            for (int l = 0; l < LG; ++l) acc[l] = T(0);
            const T* trow = Ts + jj * ldt;
            for (int i = ib; i < ie; ++i) {
                const T t = trow[i];
                const T* xr = Xs + i * LG;
#pragma unroll
                for (int l = 0; l < LG; ++l) acc[l] = fma(t, xr[l], acc[l]);
            }
            T* wp = Wp + (ks * JB + jj) * LG;
#pragma unroll
            for (int l = 0; l < LG; ++l) wp[l] = acc[l];
            __syncthreads();
            for (int e = tid; e < JB * LG; e += kT) {
                T s = T(0);
#pragma unroll 4
                for (int k = 0; k < KS; ++k) s += Wp[k * JB * LG + e];
                Ws[e] = s;
            }
            __syncthreads();
        }
        // phase 2: X_acc(i, :) += sum_jj T(jj, i) W(jj, :)
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            const int i = tid + k * kT;
            if (i < I) {
                for (int jj = 0; jj < JB; ++jj) {
                    const T t = Ts[jj * ldt + i];
                    const T* w = Ws + jj * LG;
#pragma unroll
                    for (int l = 0; l < LG; ++l) acc2[k][l] = fma(t, w[l], acc2[k][l]);
                }
            }
        }
    }
    T* out = partial + ty * ((int64_t)I * L);
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        const int i = tid + k * kT;
        if (i < I) {
#pragma unroll
            for (int l = 0; l < LG; ++l)
                if (l < lg) out[(int64_t)(l0 + l) * I + i] = acc2[k][l];
        }
    }
}

// out[e] = sum over parts of partial[p * count + e]: 32 consecutive outputs per
// step (coalesced), the parts split over the block's warps (warp w sums parts
// w, w + warps, ... in increasing order), the warps' sums combined in warp
// order, so every output is the same whichever block computes it. Block bid of
// nblk takes the steps bid, bid + nblk, ...
template <typename T, bool NC>
__device__ __forceinline__ void reduce_block(const T* __restrict__ partial, int parts, int64_t count,
                                             T* __restrict__ out, int64_t bid, int64_t nblk) {
    constexpr int kG = kThreads / 32;
    __shared__ T sh[kG][32];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    for (int64_t e0 = bid * 32; e0 < count; e0 += nblk * 32) {
        const int64_t e = e0 + lane;
        T s = T(0);
        if (e < count) {
            int p = g;
            for (; p + 3 * kG < parts; p += 4 * kG) {
                const T x0 = ld<NC>(partial + (int64_t)p * count + e);
                const T x1 = ld<NC>(partial + (int64_t)(p + kG) * count + e);
                const T x2 = ld<NC>(partial + (int64_t)(p + 2 * kG) * count + e);
                const T x3 = ld<NC>(partial + (int64_t)(p + 3 * kG) * count + e);
                s += x0;
                s += x1;
                s += x2;
                s += x3;
            }
            for (; p < parts; p += kG) s += ld<NC>(partial + (int64_t)p * count + e);
        }
        sh[g][lane] = s;
        __syncthreads();
        if (g == 0 && e < count) {
            T t = sh[0][lane];
#pragma unroll
            for (int q = 1; q < kG; ++q) t += sh[q][lane];
            out[e] = t;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- mode-n product
constexpr int kTtmKC = 32, kTtmKP = kTtmKC + 4;   // rows padded to 36 elements: 16-byte aligned, conflict-free

// four consecutive values from 16-byte aligned shared memory
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
    const double2 x = *reinterpret_cast<const double2*>(p), y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

// Shared-memory bytes of one mode-product block (tiles, then the output block;
// the fiber bases after them).
template <typename T, int OPT, int NF>
__host__ __device__ constexpr size_t ttm_block_tile_bytes() {
    return sizeof(T) * (64 * NF * kTtmKP + 4 * OPT * kTtmKP) > sizeof(T) * 64 * NF * (4 * OPT + 1)
               ? sizeof(T) * (64 * NF * kTtmKP + 4 * OPT * kTtmKP)
               : sizeof(T) * 64 * NF * (4 * OPT + 1);
}
template <typename T, int OPT, int NF>
__host__ __device__ constexpr size_t ttm_block_smem() {
    return ((ttm_block_tile_bytes<T, OPT, NF>() + 15) & ~size_t(15)) + sizeof(int64_t) * 64 * NF;
}

// Block (bx, by): fibers bx JB .. of v and outputs by OB .. of out = A x_n M,
// M(k, i) = Mp[i ld_i + k ld_k]. Thread (lane64 = tid % 64, og = tid / 64) owns
// fibers lane64 + 64 f (f < NF) and outputs og * OPT .. og * OPT + OPT - 1.
// Both shared tiles keep the input index contiguous, so stores are unit-stride
// and the inner loop reads four input indices per 128-bit load; the M rows are
// the same across a warp (broadcast) and each serves 4 NF multiply-adds. The
// next chunk's global loads are issued into registers before the current chunk
// is multiplied.
template <typename T, int OPT, int NF, bool NC>
__device__ __forceinline__ void ttm_block(const T* __restrict__ A, const ModeView& v, const T* __restrict__ Mp,
                                          int64_t K_out, int64_t ld_i, int64_t ld_k, T* __restrict__ out,
                                          int64_t bx, int64_t by, unsigned char* smem) {
    constexpr int kT = kThreads, KC = kTtmKC, KP = kTtmKP;
    constexpr int JB = 64 * NF, OB = 4 * OPT;
    constexpr int TPT = JB * KC / kT;                    // tile elements loaded per thread and chunk
    constexpr int MPT = (OB * KC + kT - 1) / kT;         // M elements loaded per thread and chunk
    auto Ts = reinterpret_cast<T(*)[KP]>(smem);                       // [JB][KP]
    auto Ms = reinterpret_cast<T(*)[KP]>(smem + sizeof(T) * JB * KP);  // [OB][KP]
    auto Os = reinterpret_cast<T(*)[OB + 1]>(smem);                   // [JB][OB + 1], after the products
    int64_t* bases = reinterpret_cast<int64_t*>(smem + ((ttm_block_tile_bytes<T, OPT, NF>() + 15) & ~size_t(15)));
    const int tid = threadIdx.x;
    const int64_t J = v.fibers();
    const int64_t j0 = bx * JB;
    const int64_t o0 = by * OB;
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
            tr[u] = (b >= 0 && i < I) ? ld<NC>(A + b + (int64_t)i * v.lf) : T(0);
        }
#pragma unroll
        for (int u = 0; u < MPT; ++u) {
            const int e = tid + u * kT;
            int kk, oo;
            if (ld_i == 1) { kk = e % KC; oo = e / KC; } // unit stride along the input index
            else { oo = e % OB; kk = e / OB; }
            const int i = i0 + kk;
            const int64_t o = o0 + oo;
            mr[u] = (e < OB * KC && i < I && o < K_out) ? ld<NC>(Mp + (int64_t)i * ld_i + o * ld_k) : T(0);
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

}  // namespace blk
}  // namespace tk
