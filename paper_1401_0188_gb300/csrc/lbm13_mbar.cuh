// lbm13_mbar.cuh -- mbarrier waits with a time limit and the tensor copy they
// complete, shared by the staged kernels (lbm13_batch.cu, lbm13_step2.cu).
//
// Every wait on a barrier is bounded by the global timer: a kernel whose copy
// never lands gives up after wait_ns, reports through its error word and
// leaves instead of hanging the GPU.
#pragma once

#include <cuda.h>

namespace lbm13 {

__device__ __forceinline__ unsigned long long tma_clock()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init_count(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned phase)
{
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    return done != 0;
}

// Wait for phase `phase` of the barrier to complete, for at most wait_ns (the
// global timer is read only once the first try has failed).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned phase, unsigned long long wait_ns)
{
    if (mbar_try(bar, phase)) return true;
    const unsigned long long end = tma_clock() + wait_ns;
    for (;;) {
        if (mbar_try(bar, phase)) return true;
        if (tma_clock() > end) return false;
    }
}

// One 3-D box of `map` at coordinates (c0, c1, c2) into shared memory at dst,
// `bytes` announced on (and completing) barrier bar.  c0 times the element
// size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_box_3d(unsigned dst, const CUtensorMap *map, int c0, int c1, int c2, unsigned bar,
                                           unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

} // namespace lbm13
