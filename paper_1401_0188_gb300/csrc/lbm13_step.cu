// lbm13_step.cu -- the time step: a boundary-link kernel that evaluates the
// wall rules' equilibrium terms once per wall position, and the fused
// pull-stream + wall + MRT-collision kernel, one pass over HBM.
//
// Storage: structure of arrays, population plane j at f + j * plane, row y at
// + y * pitch, x contiguous; pitch is a multiple of 32 elements so every row of
// every plane starts on a 128-byte (float) or 256-byte (double) boundary.  Two
// buffers alternate: a step reads the post-collision state f*(t) from `fin` and
// writes f*(t+1) to `fout`.
//
// Streaming is a pull: node x gathers population j from x - v_j.  A warp covers
// 32 consecutive x of one row, so each of its 13 loads per node is one
// coalesced 128/256-byte row segment, shifted by -v_x (0, +-1 or +-2 elements;
// the neighbouring warp reads the other half of the straddled sector, so DRAM
// traffic stays at one read per population); stores are aligned.
//
// Walls (Sec. 7, Sec. 9) lie half a link outside the first and last node.  A
// population leaving x_f with velocity -v_j crosses the wall and comes back
// with v_j to x_f + (2a - 1)(-v_j), a the crossed fraction of the link: the same
// node for |v_n| = 1 and for the diagonals, the other of the two wall rows for
// the distance-2 links:
//   bounce-back      f_j(x) =  f*_jbar(x_f) + 2 f_eq,odd_j(wall)
//   anti-bounce-back f_j(x) = -f*_jbar(x_f) + 2 f_eq,even_j(wall)   (Eq. d2q13-cl-abb)
// with anti-bounce-back on the links normal to a velocity+temperature wall and
// bounce-back on its diagonal links and on every link of an adiabatic wall.
// The wall state is rho_w = 1.5 rho(first node) - 0.5 rho(second node) (the
// extrapolation of Sec. 7; optionally, at temperature walls, the density that
// makes the wall's net normal mass flux zero), u_w the wall velocity, and E_w from the wall
// temperature, E_w = rho_w (26 T_w - 28) + 13 rho_w |u_w|^2, or extrapolated
// like rho_w at an adiabatic wall.  A diagonal that crosses two walls at a
// corner bounces back with the mean of the two walls' states.
#include "lbm13_internal.h"

// Each launch reads only what earlier launches wrote: the read-only path.
#define LBM13_LDG(p) __ldg(p)
#include "lbm13_stepdev.cuh"

namespace lbm13 {

namespace {

// One lattice: block 32 x 4 threads, each thread R rows of one column.  The
// register caps keep 6 blocks (24 warps) per SM for FP32 and 5 for FP64 and
// the forced two-row FP32 variant, without spills: more warps keep more
// population loads in flight.
template <typename T, typename C, bool Force, int R>
__global__ void __launch_bounds__(128, sizeof(T) == 4 && !(Force && R == 2) ? 6 : 5) step_kernel(const StepArgs<T, C> a)
{
    __shared__ C slots[128][Q];
    const int tid = threadIdx.y * 32 + threadIdx.x;
    process_column<T, C, Force, R>(a, blockIdx.x * 32 + threadIdx.x, (blockIdx.y * blockDim.y + threadIdx.y) * R,
                                   slots[tid]);
}

// Many lattices in one launch.  The work list holds (lattice, tile) pairs; a
// tile is 32 columns x (groups BY R) rows of one lattice, packed as
// (tile row << 16) | tile column, and the block walks its `groups` row groups
// of BY R rows in turn.  Each block takes a contiguous run of the work list
// (one tile when the grid has a block per tile; a longer run in a persistent
// grid), so consecutive tiles of a block mostly belong to one lattice; the next
// work item is fetched while the current one runs.  The block copies a
// lattice's arguments for this step's buffer parity into shared memory with
// 16-byte loads spread over its threads, only when the lattice changes.
// One row per thread keeps to 64 registers (half the SM's warps resident);
// more rows per thread take what they need.
template <typename T, typename C, int R, int BY>
__global__ void __launch_bounds__(32 * BY, (R == 1 && sizeof(T) == 4) ? 32 / BY : 1) batch_step_kernel(const BatchDesc<T, C> *__restrict__ descs,
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

template <typename T, typename C, int R, int BY>
cudaError_t launch_batch_rb(const BatchDesc<T, C> *descs, const int2 *work, int ntiles, int parity, int groups,
                            int grid, cudaStream_t s)
{
    batch_step_kernel<T, C, R, BY><<<grid, dim3(32, BY), 0, s>>>(descs, work, ntiles, parity, groups);
    return cudaGetLastError();
}

} // namespace

template <typename T, typename C>
cudaError_t launch_step(const StepArgs<T, C> &a, bool force, cudaStream_t s)
{
    constexpr int R = sizeof(T) == 8 ? 1 : 2;
    constexpr int BY = 4;
    dim3 block(32, BY);
    // A lattice of fewer than four R-row tiles per SM is latency-bound: one
    // row per thread doubles the blocks in flight (same per-node arithmetic).
    const long long tiles2 = (long long)((a.nx + 31) / 32) * ((a.ny + BY * R - 1) / (BY * R));
    if (R == 2 && tiles2 < 4 * 152) {
        dim3 grid1((a.nx + 31) / 32, (a.ny + BY - 1) / BY);
        if (force)
            step_kernel<T, C, true, 1><<<grid1, block, 0, s>>>(a);
        else
            step_kernel<T, C, false, 1><<<grid1, block, 0, s>>>(a);
        return cudaGetLastError();
    }
    dim3 grid((a.nx + 31) / 32, (a.ny + BY * R - 1) / (BY * R));
    if (force)
        step_kernel<T, C, true, R><<<grid, block, 0, s>>>(a);
    else
        step_kernel<T, C, false, R><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

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

template cudaError_t launch_step<double, double>(const StepArgs<double, double> &, bool, cudaStream_t);
template cudaError_t launch_step<float, float>(const StepArgs<float, float> &, bool, cudaStream_t);
template cudaError_t launch_batch<double, double>(const BatchDesc<double, double> *, const int2 *, int, int, int, int,
                                                  int, int, cudaStream_t);
template cudaError_t launch_batch<float, float>(const BatchDesc<float, float> *, const int2 *, int, int, int, int, int,
                                                int, cudaStream_t);

} // namespace lbm13
