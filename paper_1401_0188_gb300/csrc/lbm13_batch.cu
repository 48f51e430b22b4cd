// lbm13_batch.cu -- many lattices stepped by one launch: the fused
// pull-stream + wall + MRT-collision step of lbm13_step.cu over a work list of
// (lattice, tile) pairs, each lattice's arguments read from a descriptor array.
// The per-node device code is the one-lattice kernel's (lbm13_stepdev.cuh), so
// a lattice gives bit-identical results alone or in a plan.
#include "lbm13_internal.h"

// Each launch reads only what earlier launches wrote: the read-only path.
#define LBM13_LDG(p) __ldg(p)
#include "lbm13_stepdev.cuh"

namespace lbm13 {

namespace {

// Many lattices in one launch.  The work list holds (lattice, tile) pairs; a
// tile is 32 columns x (groups BY R) rows of one lattice, packed as
// (tile row << 16) | tile column, and the block walks its `groups` row groups
// of BY R rows in turn.  Each block takes a contiguous run of the work list
// (one tile when the grid has a block per tile; a longer run in a persistent
// grid), so consecutive tiles of a block mostly belong to one lattice; the next
// work item is fetched while the current one runs.  The block copies a
// lattice's arguments for this step's buffer parity into shared memory with
// 16-byte loads spread over its threads, only when the lattice changes.
// One row per thread keeps to 64 registers (half the SM's warps resident),
// two rows to 80 (24 warps: as many loads in flight as the one-lattice
// kernel); more rows per thread take what they need.
template <typename T, typename C, int R, int BY>
__global__ void __launch_bounds__(32 * BY, sizeof(T) == 4 ? (R == 1 ? 32 / BY : R == 2 ? 24 / BY : 1) : 1) batch_step_kernel(const BatchDesc<T, C> *__restrict__ descs,
                                                            const int2 *__restrict__ work, int ntiles, int parity,
                                                            int groups)
{
    __shared__ StepArgs<T, C> sa;
    __shared__ int s_force;
    __shared__ C slots[32 * BY][Q];
    constexpr int kWords = int(sizeof(StepArgs<T, C>) / 16);
    static_assert(sizeof(StepArgs<T, C>) % 16 == 0, "StepArgs must be a whole number of 16-byte words");
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int t0 = blockIdx.x * per;
    const int t_end = min(ntiles, t0 + per);
    int lattice = -1;
    int2 w = t0 < t_end ? __ldg(work + t0) : make_int2(0, 0);
    for (int t = t0; t < t_end; ++t) {
        const int2 wn = t + 1 < t_end ? __ldg(work + t + 1) : w;
        if (w.x != lattice) {
            __syncthreads();
            const int4 *src = reinterpret_cast<const int4 *>(&descs[w.x].a[parity]);
            int4 *dst = reinterpret_cast<int4 *>(&sa);
            for (int i = tid; i < kWords; i += 32 * BY) dst[i] = __ldg(src + i);
            if (tid == 0) s_force = descs[w.x].force;
            __syncthreads();
            lattice = w.x;
        }
        const int x = (w.y & 0xffff) * 32 + threadIdx.x;
        const int yb = (w.y >> 16) * groups * (BY * R);
        for (int g = 0; g < groups; ++g) {
            const int y = yb + g * (BY * R);
            if (y >= sa.ny) break;
            if (s_force)
                process_column<T, C, true, R>(sa, x, y + threadIdx.y * R, slots[tid]);
            else
                process_column<T, C, false, R>(sa, x, y + threadIdx.y * R, slots[tid]);
        }
        w = wn;
    }
}

// One block per tile (the grid the autotuner picks on uneven lattices): the
// same per-node code without the run loop, the next-item prefetch and the
// lattice comparison, so fewer registers stay live across the row groups.
template <typename T, typename C, int R, int BY>
__global__ void __launch_bounds__(32 * BY, sizeof(T) == 4 ? (R == 1 ? 32 / BY : R == 2 ? 24 / BY : 1) : 1) batch_tile_kernel(const BatchDesc<T, C> *__restrict__ descs,
                                                            const int2 *__restrict__ work, int parity, int groups)
{
    __shared__ StepArgs<T, C> sa;
    __shared__ int s_force;
    __shared__ C slots[32 * BY][Q];
    constexpr int kWords = int(sizeof(StepArgs<T, C>) / 16);
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int2 w = __ldg(work + blockIdx.x);
    {
        const int4 *src = reinterpret_cast<const int4 *>(&descs[w.x].a[parity]);
        int4 *dst = reinterpret_cast<int4 *>(&sa);
        for (int i = tid; i < kWords; i += 32 * BY) dst[i] = __ldg(src + i);
        if (tid == 0) s_force = descs[w.x].force;
    }
    __syncthreads();
    const int x = (w.y & 0xffff) * 32 + threadIdx.x;
    const int yb = (w.y >> 16) * groups * (BY * R);
    for (int g = 0; g < groups; ++g) {
        const int y = yb + g * (BY * R);
        if (y >= sa.ny) break;
        if (s_force)
            process_column<T, C, true, R>(sa, x, y + threadIdx.y * R, slots[tid]);
        else
            process_column<T, C, false, R>(sa, x, y + threadIdx.y * R, slots[tid]);
    }
}

template <typename T, typename C, int R, int BY>
cudaError_t launch_batch_rb(const BatchDesc<T, C> *descs, const int2 *work, int ntiles, int parity, int groups,
                            int grid, cudaStream_t s)
{
    if (grid >= ntiles)
        batch_tile_kernel<T, C, R, BY><<<ntiles, dim3(32, BY), 0, s>>>(descs, work, parity, groups);
    else
        batch_step_kernel<T, C, R, BY><<<grid, dim3(32, BY), 0, s>>>(descs, work, ntiles, parity, groups);
    return cudaGetLastError();
}

} // namespace

bool batch_shape_supported(int R, int BY)
{
    return (R == 1 && BY == 4) || (R == 2 && BY == 4) || (R == 4 && BY == 4) || (R == 2 && BY == 2) ||
           (R == 1 && BY == 8);
}

template <typename T, typename C>
cudaError_t launch_batch(const BatchDesc<T, C> *descs, const int2 *work, int ntiles, int parity, int R, int BY,
                         int groups, int grid, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (groups < 1) return cudaErrorInvalidValue;
    if (R == 1 && BY == 4) return launch_batch_rb<T, C, 1, 4>(descs, work, ntiles, parity, groups, grid, s);
    if (R == 2 && BY == 4) return launch_batch_rb<T, C, 2, 4>(descs, work, ntiles, parity, groups, grid, s);
    if (R == 4 && BY == 4) return launch_batch_rb<T, C, 4, 4>(descs, work, ntiles, parity, groups, grid, s);
    if (R == 2 && BY == 2) return launch_batch_rb<T, C, 2, 2>(descs, work, ntiles, parity, groups, grid, s);
    if (R == 1 && BY == 8) return launch_batch_rb<T, C, 1, 8>(descs, work, ntiles, parity, groups, grid, s);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_batch<double, double>(const BatchDesc<double, double> *, const int2 *, int, int, int, int,
                                                  int, int, cudaStream_t);
template cudaError_t launch_batch<float, float>(const BatchDesc<float, float> *, const int2 *, int, int, int, int, int,
                                                int, cudaStream_t);

} // namespace lbm13
