// lbm13_step2.cu -- two time steps per launch for a lattice periodic in x and
// y (FP32-deviation storage).
//
// The single-step kernel reads and writes every population once per update
// (104 bytes) and runs at the HBM copy bandwidth.  Here a block steps an
// output tile twice from one read of the rows and columns within four links
// of it: the first step covers the tile and a two-node border (the nodes the
// second step pulls from), in shared memory, the second the tile itself,
// written to the other buffer.  DRAM traffic halves (52 bytes per update);
// the border costs 15% more collisions.  Every node is pulled and collided
// exactly as in the single-step kernel (a periodic lattice has no wall rules),
// so two steps here equal two single steps bit for bit.
#include <atomic>

#include "lbm13_internal.h"
#include "lbm13_pair.h"
#include "lbm13_mbar.cuh"

#define LBM13_LDG(p) __ldg(p)
#include "lbm13_stepdev.cuh"

namespace lbm13 {

namespace {

__device__ __forceinline__ bool pair_staged(int x0, int y0, int nx, int ny)
{
    return x0 >= 4 && x0 + kPairX + 4 <= nx && y0 >= 4 && y0 + kPairY + 4 <= ny;
}

// Persistent: block b takes tiles b, b + gridDim.x, ...; each tile's input
// arrives by tensor copy into one of two buffers, issued as soon as the first
// step of the tile two before it has freed that buffer, so each copy has
// about a tile's time to land.  Each input buffer has its barrier; bit b of
// `phases` is the parity buffer b's next completion will have (every thread
// tracks the same).  Two block barriers per tile: after the first step (the
// intermediate tile complete, the input buffer free, every wait agreed on)
// and after the second (the intermediate tile free).
template <bool Force>
__global__ void __launch_bounds__(kPairThreads, kPairBlocksPerSm)
    pair_step_kernel(const StepArgs<float, float> a, const __grid_constant__ CUtensorMap map, unsigned *err,
                     int issue, unsigned long long wait_ns)
{
    extern __shared__ __align__(128) float pair_smem[];
    __shared__ __align__(8) unsigned long long bars[2];
    float *const mid = pair_smem + 2 * kPairInStride;  // [kPairMidY][Q][kPairMidX], origin (x0 - 2, y0 - 2)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kWarps = kPairThreads / 32;
    const int nx = a.nx, ny = a.ny;
    const int tx = (nx + kPairX - 1) / kPairX, ntiles = tx * ((ny + kPairY - 1) / kPairY);
    const unsigned bar0 = static_cast<unsigned>(__cvta_generic_to_shared(&bars[0]));
    const unsigned in0 = static_cast<unsigned>(__cvta_generic_to_shared(pair_smem));
    if (tid == 0) {
        mbar_init_count(bar0, 1u);
        mbar_init_count(bar0 + 8u, 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // tensor copy of tile t's input box into buffer b (first thread; staged tiles only)
    auto fetch = [&](int t, int b) {
        const int x0 = (t % tx) * kPairX, y0 = (t / tx) * kPairY;
        if (tid == 0 && issue && pair_staged(x0, y0, nx, ny)) {
            // the buffer may hold a seam tile's thread-written box: order those
            // writes before the copy's
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_box_3d(in0 + unsigned(b) * unsigned(kPairInStride) * 4u, &map, x0 - 4, 0, y0 - 4, bar0 + 8u * b,
                       unsigned(kPairIn) * 4u);
        }
    };
    unsigned phases = 0u;
    int k = 0;
    // the first two tiles' copies; after that, the copy of the tile two on is
    // issued as soon as the first step of the current tile has freed its buffer
    if (blockIdx.x < ntiles) fetch(blockIdx.x, 0);
    if (blockIdx.x + gridDim.x < ntiles) fetch(blockIdx.x + gridDim.x, 1);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int b = k & 1;
        float *const in = pair_smem + b * kPairInStride;  // [kPairInY][Q][kPairInX], origin (x0 - 4, y0 - 4)
        const int x0 = (t % tx) * kPairX, y0 = (t / tx) * kPairY;
        const bool staged = pair_staged(x0, y0, nx, ny);
        bool ok = true;
        unsigned ph = 0u;
        if (staged) {
            // every thread waits for the copy itself; the block agrees on the
            // outcome at the barrier after the first step (nothing reaches
            // global memory before it)
            ph = (phases >> b) & 1u;
            ok = mbar_wait(bar0 + 8u * b, ph, wait_ns);
            phases ^= 1u << b;
        } else {
            // a tile across the periodic seam: wrapped loads of the same box,
            // kSeamBatch of them in flight per thread before the first is stored
            // (a lattice at least one box wide and high wraps a coordinate with one
            // add or subtract; smaller ones take the remainder)
            constexpr int kPer = (kPairIn + kPairThreads - 1) / kPairThreads;
            constexpr int kSeamBatch = 11;
            const bool one_wrap = nx >= kPairInX && ny >= kPairInY;
            for (int b0 = 0; b0 < kPer; b0 += kSeamBatch) {
                float v[kSeamBatch];
#pragma unroll
                for (int u = 0; u < kSeamBatch; ++u) {
                    const int i = tid + (b0 + u) * kPairThreads;
                    v[u] = 0.0f;
                    if (b0 + u < kPer && i < kPairIn) {
                        const int xx = i % kPairInX, r = i / kPairInX, j = r % Q, yy = r / Q;
                        int x = x0 - 4 + xx, y = y0 - 4 + yy;
                        if (one_wrap) {
                            x += x < 0 ? nx : (x >= nx ? -nx : 0);
                            y += y < 0 ? ny : (y >= ny ? -ny : 0);
                        } else {
                            x %= nx;
                            y %= ny;
                            x += x < 0 ? nx : 0;
                            y += y < 0 ? ny : 0;
                        }
                        v[u] = ld(a, j, x, y);
                    }
                }
#pragma unroll
                for (int u = 0; u < kSeamBatch; ++u) {
                    const int i = tid + (b0 + u) * kPairThreads;
                    if (b0 + u < kPer && i < kPairIn) in[i] = v[u];
                }
            }
            __syncthreads();
        }
        // first step: the tile and its two-node border, one row of 32 per warp
        for (int iy = warp; iy < kPairMidY; iy += kWarps) {
            const int ix = lane;
            float f[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) f[j] = in[((iy + 2 - cvy(j)) * Q + j) * kPairInX + ix + 2 - cvx(j)];
            collide<Force>(f, a.k);
#pragma unroll
            for (int j = 0; j < Q; ++j) mid[(iy * Q + j) * kPairMidX + ix] = f[j];
        }
        if (__syncthreads_or(!ok)) {
            // a copy never landed within the limit: report, wait (bounded) for
            // the copies this block issued (this tile's, the next tile's) so
            // that none lands after it has left, and leave without writing
            if (tid == 0) {
                atomicOr(err, 1u);
                if (issue) {
                    if (staged) mbar_wait(bar0 + 8u * b, ph, wait_ns);
                    const int tn = t + gridDim.x;
                    if (tn < ntiles && pair_staged((tn % tx) * kPairX, (tn / tx) * kPairY, nx, ny))
                        mbar_wait(bar0 + 8u * (b ^ 1), (phases >> (b ^ 1)) & 1u, wait_ns);
                }
            }
            return;
        }
        // this input buffer is free: the copy of the tile two on goes into it
        if (t + 2 * gridDim.x < ntiles) fetch(t + 2 * gridDim.x, b);
        // second step: the tile (28 lanes of each warp), to the other buffer
        for (int oy = warp; oy < kPairY; oy += kWarps) {
            const int ox = lane, x = x0 + ox, y = y0 + oy;
            if (ox >= kPairX || x >= nx || y >= ny) continue;
            float f[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) f[j] = mid[((oy + 2 - cvy(j)) * Q + j) * kPairMidX + ox + 2 - cvx(j)];
            collide<Force>(f, a.k);
#ifdef LBM13_DEBUG
            store(a, x, y, f);
#else
            float *p = a.fout + (long long)y * a.pitch + x;
#pragma unroll
            for (int j = 0; j < Q; ++j) p[(long long)j * a.plane] = f[j];
#endif
        }
        __syncthreads();  // the intermediate tile is free again
    }
}

} // namespace

cudaError_t launch_pair_step(const StepArgs<float, float> &a, const CUtensorMap &map, bool force, unsigned *err,
                             cudaStream_t s, int issue, unsigned long long wait_ns)
{
    // the shared-memory allowance and carveout are per-device attributes: set
    // them once on each device that launches the kernel
    static std::atomic<unsigned long long> raised{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(raised.load() & bit)) {
        for (int f = 0; f < 2 && e == cudaSuccess; ++f) {
            const void *fn = f ? reinterpret_cast<const void *>(pair_step_kernel<true>)
                               : reinterpret_cast<const void *>(pair_step_kernel<false>);
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairSmem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         int(cudaSharedmemCarveoutMaxShared));
        }
        if (e != cudaSuccess) return e;
        raised.fetch_or(bit);
    }
    const int ntiles = ((a.nx + kPairX - 1) / kPairX) * ((a.ny + kPairY - 1) / kPairY);
    const int slots = kPairBlocksPerSm * device_sm_count();
    const int grid = ntiles < slots ? ntiles : slots;
    if (force)
        pair_step_kernel<true><<<grid, kPairThreads, kPairSmem, s>>>(a, map, err, issue, wait_ns);
    else
        pair_step_kernel<false><<<grid, kPairThreads, kPairSmem, s>>>(a, map, err, issue, wait_ns);
    return cudaGetLastError();
}

} // namespace lbm13
