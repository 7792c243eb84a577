// Work-list kernel of batched runs. A batch of decompositions is cut into
// tasks - one stage of one request's mode: the Gaussian test matrix, the power
// step's per-CTA partials, their fixed-order sum, the mode-n product, the
// status word's reset - and each task into items, the blocks its own kernel
// would launch. The tasks of one phase (for every request of the batch) are
// independent, and one persistent launch per phase walks their items: a CTA
// claims the next item with an atomic ticket, runs the item's block program
// (blocks.cuh, the same code and results as the stage's own kernel) and claims
// again until the list is exhausted. What a task reads was written by an
// earlier phase, an earlier launch on the same stream, so no CTA ever waits for
// another.
#include "blocks.cuh"
#include "internal.h"

namespace tk {
namespace {

constexpr int kT = kThreads;
template <typename T, int JB, int LG>
__device__ __forceinline__ void pow_item(const WTask& t, const WItem& w, unsigned char* smem) {
    blk::power_block<T, JB, LG, 1, false, false>((const T*)t.in, t.v, (const T*)t.X, t.L, (T*)t.out, t.tiles, 0, 0,
                                                 w.x, w.y, t.parts, smem);
}

template <typename T, int OPT>
__device__ __forceinline__ void ttm_item(const WTask& t, const WItem& w, unsigned char* smem) {
    constexpr int NF = sizeof(T) == 4 ? 2 : 1;
    blk::ttm_block<T, OPT, NF, false>((const T*)t.in, t.v, (const T*)t.X, t.K, 1, t.v.i, (T*)t.out, w.x, w.y, smem);
}

// HEAVY: every tile shape; else only the light ones (power-step column groups of
// at most 16, mode products of at most 16 outputs per block), which keeps the
// kernel within 128 registers so two CTAs share an SM.
template <typename T, bool HEAVY>
__device__ void run_item(const WTask& t, const WItem& w, unsigned char* smem) {
    switch (t.kind) {
        case kWInit:
            if (threadIdx.x == 0) *t.status = 0;
            break;
        case kWGen:
            blk::gaussian_block<T>((T*)t.out, t.rows, t.cols, t.seed, t.sid, w.x, t.nitems);
            break;
        case kWPow:
            if constexpr (sizeof(T) == 4) {
                if constexpr (HEAVY) {
                    if (t.lg == 32) pow_item<T, 32, 32>(t, w, smem);
                    else if (t.lg == 16) pow_item<T, 32, 16>(t, w, smem);
                    else pow_item<T, 32, 8>(t, w, smem);
                } else {
                    if (t.lg == 16) pow_item<T, 32, 16>(t, w, smem);
                    else pow_item<T, 32, 8>(t, w, smem);
                }
            } else {
                if (t.lg == 16) pow_item<T, 16, 16>(t, w, smem);
                else pow_item<T, 16, 8>(t, w, smem);
            }
            break;
        case kWRed:
            blk::reduce_block<T, false>((const T*)t.in, t.parts, t.count, (T*)t.out, w.x, t.nitems);
            break;
        case kWTtm:
            if constexpr (HEAVY) {
                switch (t.opt) {
                    case 1: ttm_item<T, 1>(t, w, smem); break;
                    case 2: ttm_item<T, 2>(t, w, smem); break;
                    case 3: ttm_item<T, 3>(t, w, smem); break;
                    case 4: ttm_item<T, 4>(t, w, smem); break;
                    case 5: ttm_item<T, 5>(t, w, smem); break;
                    case 6: ttm_item<T, 6>(t, w, smem); break;
                    default: ttm_item<T, 8>(t, w, smem); break;
                }
            } else {
                switch (t.opt) {
                    case 1: ttm_item<T, 1>(t, w, smem); break;
                    case 2: ttm_item<T, 2>(t, w, smem); break;
                    case 3: ttm_item<T, 3>(t, w, smem); break;
                    default: ttm_item<T, 4>(t, w, smem); break;
                }
            }
            break;
        default:
            break;
    }
}

template <typename T, bool HEAVY>
__global__ void __launch_bounds__(kT, HEAVY ? 1 : 2) worklist_kernel(const WTask* __restrict__ tasks,
                                                                     const WItem* __restrict__ items, int begin,
                                                                     int end, unsigned* __restrict__ claim) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = begin + (int)atomicAdd(claim, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= end) return;
        const WItem w = items[it];
        run_item<T, HEAVY>(tasks[w.task], w, smem);
        __syncthreads();                       // the item's reads of shared memory and s_item, before the next
    }
}

// Dynamic shared memory a CTA may take beside the kernel's static variables
// (0 until allow_smem has raised the limit).
size_t g_smem_cap[2][2] = {{0, 0}, {0, 0}};     // [FP64][HEAVY]

// The kernel's dynamic shared-memory limit raised to all the device allows a
// CTA beside the kernel's static shared memory.
template <typename T, bool HEAVY>
cudaError_t allow_smem() {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, worklist_kernel<T, HEAVY>);
    if (e != cudaSuccess) return e;
    const int cap = optin - (int)fa.sharedSizeBytes;
    if (cap <= 0) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(worklist_kernel<T, HEAVY>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e == cudaSuccess) g_smem_cap[sizeof(T) == 4 ? 0 : 1][HEAVY] = (size_t)cap;
    return e;
}

template <typename T, bool HEAVY>
int occupancy(size_t smem) {
    int occ = 0;
    if (allow_smem<T, HEAVY>() != cudaSuccess || smem > g_smem_cap[sizeof(T) == 4 ? 0 : 1][HEAVY] ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, worklist_kernel<T, HEAVY>, kT, smem) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    return occ;
}

}  // namespace

int worklist_grid(int elem, bool heavy, size_t smem, int items) {
    if (items < 1) return 0;
    const int occ = elem == 4 ? (heavy ? occupancy<float, true>(smem) : occupancy<float, false>(smem))
                              : (heavy ? occupancy<double, true>(smem) : occupancy<double, false>(smem));
    const int64_t g = (int64_t)num_sms() * occ;
    return (int)(g < items ? g : items);
}

size_t worklist_pow_smem(int elem, int I, int lg) {
    if (elem == 4) {
        if (lg == 32) return blk::power_block_smem<float, 32, 32, false>(I);
        if (lg == 16) return blk::power_block_smem<float, 32, 16, false>(I);
        return blk::power_block_smem<float, 32, 8, false>(I);
    }
    if (lg == 16) return blk::power_block_smem<double, 16, 16, false>(I);
    return blk::power_block_smem<double, 16, 8, false>(I);
}

size_t worklist_ttm_smem(int elem, int opt) {
    if (opt <= 4) return elem == 4 ? blk::ttm_block_smem<float, 4, 2>() : blk::ttm_block_smem<double, 4, 1>();
    return elem == 4 ? blk::ttm_block_smem<float, 8, 2>() : blk::ttm_block_smem<double, 8, 1>();
}

bool worklist_heavy(const WTask& t) { return (t.kind == kWPow && t.lg > 16) || (t.kind == kWTtm && t.opt > 4); }

int worklist_ttm_opt(int64_t K) {
    static const int kOpts[] = {1, 2, 3, 4, 5, 6, 8};
    for (int o : kOpts)
        if (4 * o >= K) return o;
    return 0;
}

template <typename T>
cudaError_t launch_worklist(const WTask* tasks, const WItem* items, int begin, int end, unsigned* claim, bool heavy,
                            size_t smem, int grid, cudaStream_t s) {
    if (end <= begin) return cudaSuccess;
    if (smem > g_smem_cap[sizeof(T) == 4 ? 0 : 1][heavy] || grid < 1) return cudaErrorInvalidValue;
    ProfScope prof(kKWorklist, 0.0, 0.0, s);
    if (heavy)
        worklist_kernel<T, true><<<(unsigned)grid, kT, smem, s>>>(tasks, items, begin, end, claim);
    else
        worklist_kernel<T, false><<<(unsigned)grid, kT, smem, s>>>(tasks, items, begin, end, claim);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t launch_worklist<float>(const WTask*, const WItem*, int, int, unsigned*, bool, size_t, int,
                                            cudaStream_t);
template cudaError_t launch_worklist<double>(const WTask*, const WItem*, int, int, unsigned*, bool, size_t, int,
                                             cudaStream_t);

}  // namespace tk
