// lbm13_multi.cu -- a persistent kernel that advances one lattice by many
// time steps in a single cooperative launch.
//
// A small lattice (both population buffers well inside the 129 MB L2) is
// bound by launch latency, not by HBM: a step is a few microseconds of work.
// Here every block of a co-resident grid takes tiles of the lattice in turn,
// and a grid barrier separates consecutive steps (each fused pull + collide +
// store, with the wall corrections evaluated by the edge nodes); the next step
// reads what the other blocks wrote, so populations are loaded L2-coherently
// (__ldcg) instead of through the read-only path.  The per-node arithmetic is the shared device code of the
// per-step kernels, so the results are bit-identical to stepping launch by
// launch.
//
// The grid barrier counts arrivals in global memory and releases by bumping a
// generation word.  Every wait is bounded: a block that waits longer than the
// timeout records it in the error word and all blocks leave the kernel; the
// host reports LBM13_ETIMEOUT at its next synchronisation.  Co-residency of all
// blocks is guaranteed by the cooperative launch (which fails instead of
// launching a grid that does not fit).
#include "lbm13_internal.h"

// One launch reads what its other blocks wrote before a grid barrier: loads go
// to L2, never to a possibly stale L1 line.
#define LBM13_LDG(p) __ldcg(p)
#include "lbm13_stepdev.cuh"

namespace lbm13 {

namespace {

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned load_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier over the nblocks blocks of the grid.  Returns false for every thread
// of the block once a timeout has been recorded (by this or any block).
__device__ bool grid_barrier(const GridSync &g, unsigned nblocks)
{
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const unsigned gen = load_acquire(g.gen);
        __threadfence();
        if (atomicAdd(g.count, 1u) == nblocks - 1) {
            atomicExch(g.count, 0u);
            __threadfence();
            atomicAdd(g.gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            unsigned it = 0;
            while (load_acquire(g.gen) == gen) {
                if ((++it & 15u) == 0u) {
                    if (load_acquire(g.error) != 0u) break;
                    if (global_ns() - t0 > g.timeout_ns) {
                        atomicExch(g.error, 1u);
                        break;
                    }
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return load_acquire(g.error) == 0u;
}

// One step of the lattice over the whole grid; false if a barrier timed out.
// The last step of a launch needs no closing barrier (the launch's end is one).
template <typename T, typename C, bool Force, int R>
__device__ __forceinline__ bool grid_step(const StepArgs<T, C> &a, int tiles_x, int ntiles, bool last, C *slot,
                                          const GridSync &g)
{
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tx = t % tiles_x, ty = t / tiles_x;
        process_column<T, C, Force, R>(a, tx * 32 + threadIdx.x, (ty * 4 + threadIdx.y) * R, slot);
    }
    return last || grid_barrier(g, gridDim.x);
}

// nsteps steps alternating a0 (the current buffer parity) and a1.
template <typename T, typename C, bool Force, int R>
__global__ void __launch_bounds__(128) multi_step_kernel(const StepArgs<T, C> a0, const StepArgs<T, C> a1,
                                                         int nsteps, const GridSync g)
{
    __shared__ C slots[128][Q];
    C *slot = slots[threadIdx.y * 32 + threadIdx.x];
    const int tiles_x = (a0.nx + 31) / 32;
    const int ntiles = tiles_x * ((a0.ny + 4 * R - 1) / (4 * R));
    for (int s = 0; s < nsteps; s += 2) {
        if (!grid_step<T, C, Force, R>(a0, tiles_x, ntiles, s + 1 >= nsteps, slot, g)) return;
        if (s + 1 < nsteps && !grid_step<T, C, Force, R>(a1, tiles_x, ntiles, s + 2 >= nsteps, slot, g)) return;
    }
}

// Barrier self-check: `rounds` barriers over a grid that may be smaller than
// the count the barrier waits for (then every wait runs into the timeout).
__global__ void __launch_bounds__(128) barrier_check_kernel(unsigned expect_blocks, int rounds, const GridSync g)
{
    for (int r = 0; r < rounds; ++r)
        if (!grid_barrier(g, expect_blocks)) return;
}

template <typename T>
constexpr int multi_rows() { return sizeof(T) == 8 ? 1 : 2; }

template <typename T, typename C>
const void *multi_fn(bool force)
{
    constexpr int R = multi_rows<T>();
    return force ? reinterpret_cast<const void *>(&multi_step_kernel<T, C, true, R>)
                 : reinterpret_cast<const void *>(&multi_step_kernel<T, C, false, R>);
}

} // namespace

template <typename T, typename C>
int multi_grid(int nx, int ny, bool force)
{
    constexpr int R = multi_rows<T>();
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, multi_fn<T, C>(force), 128, 0) != cudaSuccess)
        return 0;
    const long long tiles = (long long)((nx + 31) / 32) * ((ny + 4 * R - 1) / (4 * R));
    const long long cap = (long long)sms * per_sm;
    return int(tiles < cap ? tiles : cap);
}

template <typename T, typename C>
cudaError_t launch_multi(const StepArgs<T, C> &a0, const StepArgs<T, C> &a1, bool force, int nsteps, int grid,
                         const GridSync &g, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(g.count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    StepArgs<T, C> p0 = a0, p1 = a1;
    GridSync gs = g;
    void *args[] = {&p0, &p1, &nsteps, &gs};
    return cudaLaunchCooperativeKernel(multi_fn<T, C>(force), dim3(grid), dim3(32, 4), args, 0, s);
}

cudaError_t launch_barrier_check(int grid, unsigned expect_blocks, int rounds, const GridSync &g, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(g.count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    GridSync gs = g;
    void *args[] = {&expect_blocks, &rounds, &gs};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(&barrier_check_kernel), dim3(grid),
                                       dim3(32, 4), args, 0, s);
}

template int multi_grid<double, double>(int, int, bool);
template int multi_grid<float, float>(int, int, bool);
template cudaError_t launch_multi<double, double>(const StepArgs<double, double> &, const StepArgs<double, double> &,
                                                  bool, int, int, const GridSync &, cudaStream_t);
template cudaError_t launch_multi<float, float>(const StepArgs<float, float> &, const StepArgs<float, float> &, bool,
                                                int, int, const GridSync &, cudaStream_t);

} // namespace lbm13
