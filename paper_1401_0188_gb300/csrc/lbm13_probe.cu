// lbm13_probe.cu -- measured FP64 instruction rate of the current device.
//
// The FP64 time step is bound by its FP64 pipe, not by HBM: its roofline needs
// the rate at which this GPU retires FP64 instructions.  The probe fills every
// SM with independent FMA chains (eight per thread, so that the pipe, not the
// FMA latency, sets the rate) and times them with CUDA events.
#include <cuda_runtime.h>

#include "../../include/lbm13.h"
#include "lbm13_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;
constexpr int kChains = 8;

// One value per block keeps the chains alive (their sum is stored).
__device__ double g_sink[4096];

__global__ void __launch_bounds__(kThreads) fma_chains(int iters, double m, double a)
{
    double acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = double(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], m, a);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (threadIdx.x == 0) g_sink[blockIdx.x & 4095] = s;
}

} // namespace

extern "C" int lbm13_fp64_fma_rate(int iters, double *fma_per_s, double *seconds)
{
    if (!fma_per_s || iters < 1 || iters > (1 << 24)) return LBM13_EINVAL;
    const int blocks = lbm13::device_sm_count() * kBlocksPerSm;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.0f;
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(blocks));
        cfg.blockDim = dim3(kThreads);
        cfg.stream = s;
        const double m = 1.0 - 1e-12, a = 1e-9;
        e = cudaLaunchKernelEx(&cfg, fma_chains, iters / 8 + 1, m, a);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, fma_chains, iters, m, a);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess || !(ms > 0.0f)) return LBM13_ECUDA;
    const double fmas = double(blocks) * kThreads * kChains * double(iters);
    *fma_per_s = fmas / (double(ms) * 1e-3);
    if (seconds) *seconds = double(ms) * 1e-3;
    return LBM13_OK;
}
