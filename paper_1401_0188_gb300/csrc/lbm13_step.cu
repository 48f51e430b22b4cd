// lbm13_step.cu -- the time step of one lattice: the fused pull-stream + wall +
// MRT-collision kernel, one launch and one pass over HBM per step.
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
// corner bounces back with each wall's correction at that wall's own state.  The nodes next
// to a wall evaluate its state at their own position and add the wall
// correction, a quadratic in (rho_w, E_w) whose coefficients the host computes
// once per lattice.
#include <atomic>

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

} // namespace

int device_sm_count()
{
    constexpr int kMaxDevices = 64;
    static std::atomic<int> cache[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < kMaxDevices) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
    if (dev >= 0 && dev < kMaxDevices) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

template <typename T, typename C>
cudaError_t launch_step(const StepArgs<T, C> &a, bool force, cudaStream_t s)
{
    constexpr int R = sizeof(T) == 8 ? 1 : 2;
    constexpr int BY = 4;
    dim3 block(32, BY);
    // A lattice of fewer than sixteen R-row tiles per SM (up to about 768^2
    // on 152 SMs, which lives in L2) is latency-bound: one row per thread doubles the
    // blocks in flight (same per-node arithmetic).  From 1024^2 on, two rows
    // per thread measured faster.
    const long long tiles2 = (long long)((a.nx + 31) / 32) * ((a.ny + BY * R - 1) / (BY * R));
    if (R == 2 && tiles2 < 16LL * device_sm_count()) {
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

template cudaError_t launch_step<double, double>(const StepArgs<double, double> &, bool, cudaStream_t);
template cudaError_t launch_step<float, float>(const StepArgs<float, float> &, bool, cudaStream_t);

} // namespace lbm13
