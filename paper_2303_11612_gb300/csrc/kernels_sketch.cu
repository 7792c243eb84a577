// Sketch kernels: Gaussian test matrices, the fused power step of Strategy A
// (remark after Algorithm 1) and the range-form sketch with the Gaussian
// generated inside the kernel.
//
// Power step X_out = A_(n) (A_(n)^T X_in). The unfolding's columns (mode-n
// fibers) are streamed in tiles of JB fibers; for each tile T (JB x I_n):
//   W = T X_in           (JB x L)   phase 1, split over I_n and reduced in smem
//   X_acc += T^T W       (I_n x L)  phase 2, accumulated in registers
// so every element of A is read once per power step. Each CTA accumulates the
// tiles it owns and writes one partial; a second kernel sums the partials in a
// fixed order, which makes the result independent of scheduling.
#include <string>
#include <utility>
#include <vector>

#include "blocks.cuh"
#include "internal.h"

namespace tk {

namespace {

constexpr int kT = kThreads;

template <typename T>
__global__ void __launch_bounds__(kT) gaussian_kernel(T* __restrict__ out, int64_t rows, int64_t cols,
                                                      uint64_t seed, uint32_t stream_id) {
    blk::gaussian_block<T>(out, rows, cols, seed, stream_id, blockIdx.x, gridDim.x);
}

// Block (l-group blockIdx.x, tiles blockIdx.y + k gridDim.y) of the power step;
// RANGE == false: W = T X (phase 1). RANGE == true: W = Omega rows (Philox).
template <typename T, int JB, int LG, int KR, bool RANGE>
__global__ void __launch_bounds__(kT) power_kernel(const T* __restrict__ A, ModeView v,
                                                   const T* __restrict__ X, int L,
                                                   T* __restrict__ partial, int64_t tiles,
                                                   uint64_t seed, uint32_t stream_id) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    blk::power_block<T, JB, LG, KR, RANGE, true>(A, v, X, L, partial, tiles, seed, stream_id, blockIdx.x, blockIdx.y,
                                                 gridDim.y, smem_raw);
}

// out[e] = sum over parts of partial[p * count + e] in a fixed order (the block
// program's), so the result does not depend on scheduling.
template <typename T>
__global__ void __launch_bounds__(kT) reduce_partials_kernel(const T* __restrict__ partial, int parts,
                                                             int64_t count, T* __restrict__ out) {
    blk::reduce_block<T, true>(partial, parts, count, out, blockIdx.x, gridDim.x);
}

template <typename T, int JB, int LG, int KR, bool RANGE>
size_t power_smem(int I) {
    return blk::power_block_smem<T, JB, LG, RANGE>(I);
}

}  // namespace

PowerPlan power_plan(const ModeView& v, int L, int elem_size, int num_sms) {
    PowerPlan p{};
    const int I = (int)v.i;
    const bool dbl = elem_size == 8;
    p.jb = (dbl || I > 512) ? 16 : 32;
    p.lg = (dbl || I > 512) ? 16 : 32;
    if (L < p.lg) p.lg = L <= 8 ? 8 : (L <= 16 ? 16 : p.lg);
    p.groups = (L + p.lg - 1) / p.lg;
    p.tiles = (v.fibers() + p.jb - 1) / p.jb;
    int64_t want = (int64_t)num_sms / p.groups;
    if (want < 1) want = 1;
    p.parts = (int)(want < p.tiles ? want : p.tiles);
    const int ldt = I | 1;
    p.smem = (size_t)elem_size * ((size_t)I * p.lg + (size_t)p.jb * ldt + (size_t)(kThreads / p.jb) * p.jb * p.lg +
                                  (size_t)p.jb * p.lg) + sizeof(int64_t) * p.jb + 16;
    return p;
}

size_t power_partials_bytes(const PowerPlan& p, const ModeView& v, int L, int elem_size) {
    return (size_t)p.parts * (size_t)v.i * (size_t)L * elem_size;
}

template <typename T>
cudaError_t launch_gaussian(T* out, int64_t rows, int64_t cols, uint64_t seed, uint32_t stream_id,
                            cudaStream_t s) {
    const int64_t n = rows * cols;
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + kT - 1) / kT;
    if (blocks > 4096) blocks = 4096;
    gaussian_kernel<T><<<(unsigned)blocks, kT, 0, s>>>(out, rows, cols, seed, stream_id);
    note_launch();
    return cudaGetLastError();
}

namespace {
template <typename T, int JB, int LG, int KR>
cudaError_t launch_power_t(const T* A, const ModeView& v, const T* X_in, int L, T* partials,
                           const PowerPlan& plan, bool range, uint64_t seed, uint32_t sid, cudaStream_t s) {
    dim3 grid(plan.groups, plan.parts);
    const int I = (int)v.i;
    const double elems = (double)v.i * (double)v.fibers();
    ProfScope prof(kKPower, elems * sizeof(T), (range ? 2.0 : 4.0) * elems * L, s);
    if (range) {
        auto k = power_kernel<T, JB, LG, KR, true>;
        const size_t smem = power_smem<T, JB, LG, KR, true>(I);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, kT, smem, s>>>(A, v, X_in, L, partials, plan.tiles, seed, sid);
        note_launch();
    } else {
        auto k = power_kernel<T, JB, LG, KR, false>;
        const size_t smem = power_smem<T, JB, LG, KR, false>(I);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, kT, smem, s>>>(A, v, X_in, L, partials, plan.tiles, seed, sid);
        note_launch();
    }
    return cudaGetLastError();
}

template <typename T, int JB, int LG>
cudaError_t dispatch_kr(const T* A, const ModeView& v, const T* X_in, int L, T* partials,
                        const PowerPlan& plan, bool range, uint64_t seed, uint32_t sid, cudaStream_t s) {
    const int kr = (int)((v.i + kT - 1) / kT);
    switch (kr) {
        case 1: return launch_power_t<T, JB, LG, 1>(A, v, X_in, L, partials, plan, range, seed, sid, s);
        case 2: return launch_power_t<T, JB, LG, 2>(A, v, X_in, L, partials, plan, range, seed, sid, s);
        case 3: return launch_power_t<T, JB, LG, 3>(A, v, X_in, L, partials, plan, range, seed, sid, s);
        case 4: return launch_power_t<T, JB, LG, 4>(A, v, X_in, L, partials, plan, range, seed, sid, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

namespace {
// The plan with tile shape (jb, lg): more fiber groups share the SMs, so the
// number of partials (and their memory) never exceeds the base plan's.
PowerPlan plan_with(const PowerPlan& base, const ModeView& v, int L, int jb, int lg) {
    PowerPlan p = base;
    p.jb = jb;
    p.lg = lg;
    p.groups = (L + lg - 1) / lg;
    p.tiles = (v.fibers() + jb - 1) / jb;
    int64_t parts = (int64_t)base.parts * base.groups / p.groups;
    if (parts < 1) parts = 1;
    if (parts > p.tiles) parts = p.tiles;
    if (parts > base.parts) parts = base.parts;
    p.parts = (int)parts;
    return p;
}
}  // namespace

template <typename T>
cudaError_t launch_power_plan(const T* A, const ModeView& v, const T* X_in, int L, T* X_out, void* partials,
                              const PowerPlan& plan, bool range, uint64_t seed, uint32_t stream_id, cudaStream_t s);

template <typename T>
cudaError_t launch_power(const T* A, const ModeView& v, const T* X_in, int L, T* X_out, void* partials,
                         const PowerPlan& plan, bool range, uint64_t seed, uint32_t stream_id,
                         cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        // FP32: the autotuner may pick another tile shape (jb fibers x lg columns)
        // for this shape class; shapes differ in summation order, so a tuned run
        // can differ from an untuned one in the last bits
        std::vector<std::pair<int, int>> shapes;
        std::vector<std::string> names;
        for (auto jl : {std::pair<int, int>{32, 32}, {32, 16}, {16, 16}, {32, 8}, {16, 8}}) {
            if (jl.second > plan.lg || (jl.first == 32 && v.i > 512)) continue;
            shapes.push_back(jl);
            names.push_back("jb" + std::to_string(jl.first) + "/lg" + std::to_string(jl.second));
        }
        const TuneKey key{kTunePower, {v.i, L, v.lf * (range ? -1 : 1), v.fibers()}};
        int choice = tune_get(key);
        if (choice < 0 && shapes.size() > 1 && tune_active(s)) {
            int base = 0;
            for (size_t c = 0; c < shapes.size(); ++c)
                if (shapes[c].first == plan.jb && shapes[c].second == plan.lg) base = (int)c;
            choice = tune_pick(
                s, key, "FP32 power step (I, L, +-L_f, J)", names,
                [&](int c) {
                    return launch_power_plan<T>(A, v, X_in, L, X_out, partials,
                                                plan_with(plan, v, L, shapes[c].first, shapes[c].second), range,
                                                seed, stream_id, s);
                },
                base);
        }
        if (choice >= 0 && choice < (int)shapes.size())
            return launch_power_plan<T>(A, v, X_in, L, X_out, partials,
                                        plan_with(plan, v, L, shapes[choice].first, shapes[choice].second), range,
                                        seed, stream_id, s);
    }
    return launch_power_plan<T>(A, v, X_in, L, X_out, partials, plan, range, seed, stream_id, s);
}

template <typename T>
cudaError_t launch_power_plan(const T* A, const ModeView& v, const T* X_in, int L, T* X_out, void* partials,
                              const PowerPlan& plan, bool range, uint64_t seed, uint32_t stream_id,
                              cudaStream_t s) {
    T* part = reinterpret_cast<T*>(partials);
    cudaError_t e;
    if constexpr (sizeof(T) == 8) {
        if (plan.jb == 16 && plan.lg == 16)
            e = dispatch_kr<T, 16, 16>(A, v, X_in, L, part, plan, range, seed, stream_id, s);
        else if (plan.jb == 16 && plan.lg == 8)
            e = dispatch_kr<T, 16, 8>(A, v, X_in, L, part, plan, range, seed, stream_id, s);
        else
            return cudaErrorInvalidValue;
    } else if (plan.jb == 32 && plan.lg == 32)
        e = dispatch_kr<T, 32, 32>(A, v, X_in, L, part, plan, range, seed, stream_id, s);
    else if (plan.jb == 32 && plan.lg == 16)
        e = dispatch_kr<T, 32, 16>(A, v, X_in, L, part, plan, range, seed, stream_id, s);
    else if (plan.jb == 32 && plan.lg == 8)
        e = dispatch_kr<T, 32, 8>(A, v, X_in, L, part, plan, range, seed, stream_id, s);
    else if (plan.jb == 16 && plan.lg == 16)
        e = dispatch_kr<T, 16, 16>(A, v, X_in, L, part, plan, range, seed, stream_id, s);
    else if (plan.jb == 16 && plan.lg == 8)
        e = dispatch_kr<T, 16, 8>(A, v, X_in, L, part, plan, range, seed, stream_id, s);
    else
        return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    return launch_reduce_partials<T>(part, plan.parts, v.i * (int64_t)L, X_out, s);
}

template <typename T>
cudaError_t launch_reduce_partials(const T* partial, int parts, int64_t count, T* out, cudaStream_t s) {
    int64_t blocks = (count + 31) / 32;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    reduce_partials_kernel<T><<<(unsigned)blocks, kT, 0, s>>>(partial, parts, count, out);
    note_launch();
    return cudaGetLastError();
}
template cudaError_t launch_reduce_partials<float>(const float*, int, int64_t, float*, cudaStream_t);
template cudaError_t launch_reduce_partials<double>(const double*, int, int64_t, double*, cudaStream_t);

template cudaError_t launch_gaussian<float>(float*, int64_t, int64_t, uint64_t, uint32_t, cudaStream_t);
template cudaError_t launch_gaussian<double>(double*, int64_t, int64_t, uint64_t, uint32_t, cudaStream_t);
template cudaError_t launch_power<float>(const float*, const ModeView&, const float*, int, float*, void*,
                                         const PowerPlan&, bool, uint64_t, uint32_t, cudaStream_t);
template cudaError_t launch_power<double>(const double*, const ModeView&, const double*, int, double*, void*,
                                          const PowerPlan&, bool, uint64_t, uint32_t, cudaStream_t);

}  // namespace tk
