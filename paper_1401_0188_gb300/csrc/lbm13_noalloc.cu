// lbm13_noalloc.cu -- conserved totals of a lattice without any allocation.
//
// lbm13_residual allocates its reduction buffers (six doubles per node plus
// block partials) through the lattice's allocator on its first call.  Some
// callers cannot allocate at the point where they need the totals: a serving
// loop whose device memory is all handed to lattices under a fixed budget by
// another allocator, a latency-bound loop that cannot take the device-wide
// synchronisation cudaMalloc/cudaFree may impose, and code inside an allocator
// callback that must not re-enter it.  lbm13_totals_noalloc serves them: the
// same deterministic FP64 sums, with the block partials in a fixed file-scope
// device array instead of allocated memory.
#include <mutex>

#include <cuda.h>  // CUcontext (the type only: the two driver calls are fetched through the runtime)

#include "../../include/lbm13.h"
#include "lbm13_internal.h"

namespace {

using namespace lbm13;

constexpr int kThreads = 256;
constexpr int kNodesPerThread = 64;
constexpr long long kNodesPerBlock = (long long)kThreads * kNodesPerThread;  // 16384
constexpr int kMaxBlocks = LBM13_NOALLOC_MAX_NODES / (int)kNodesPerBlock;     // 4096
constexpr int kSlots = 8;
static_assert((long long)kMaxBlocks * kNodesPerBlock == LBM13_NOALLOC_MAX_NODES, "block tiling");

// The scratch: one row of kSlots partial results per block (256 KiB).  Every
// GPU that loads the library holds it until the process exits.  Each call's
// blocks overwrite their own rows before the final pass reads them, so nothing
// has to be cleared between calls; calls that overlap on the GPU share it and
// race.
static __device__ __align__(256) double g_partials[kMaxBlocks * kSlots];

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double wmax(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Slots: 0 sum drho, 1 sum jx, 2 sum jy, 3 sum dE, 4 sum (T - T0), 5 non-finite
// populations, 6 max |u|.
template <typename T>
__global__ void __launch_bounds__(kThreads) totals_kernel(const T *__restrict__ f, int nx, int ny, long long pitch,
                                                         long long plane, double E0, double gx, double gy,
                                                         double rho_ref, double heat, double *partials)
{
    const long long n = (long long)nx * ny;
    const double T0 = (E0 + 28.0) / 26.0;
    double s[6] = {0, 0, 0, 0, 0, 0};
    double mx = 0.0;
    const long long first = (long long)blockIdx.x * kNodesPerBlock + threadIdx.x;
    for (int k = 0; k < kNodesPerThread; ++k) {
        const long long i = first + (long long)k * kThreads;
        if (i >= n) break;
        const int y = int(i / nx), x = int(i - (long long)y * nx);
        const long long idx = (long long)y * pitch + x;
        double g[Q];
        double bad = 0.0;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            g[j] = double(f[(long long)j * plane + idx]);
            bad += isfinite(g[j]) ? 0.0 : 1.0;
        }
        Mom<double> d;
        forward(g, d);
        const double rho = 1.0 + d.rho;
        const double w = rho - rho_ref;
        const double ux = (d.jx - 0.5 * w * gx) / rho, uy = (d.jy - 0.5 * w * gy) / rho;
        const double p = (E0 + d.E + 28.0 * rho) / 26.0 - (d.jx * d.jx + d.jy * d.jy) / (2.0 * rho) - 0.5 * heat;
        s[0] += d.rho;
        s[1] += d.jx;
        s[2] += d.jy;
        s[3] += d.E;
        s[4] += p / rho - T0;
        s[5] += bad;
        const double um = sqrt(ux * ux + uy * uy);
        mx = isnan(um) ? mx : fmax(mx, um);
    }
    __shared__ double sh[kThreads / 32][kSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 6; ++q) s[q] = wsum(s[q]);
    mx = wmax(mx);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 6; ++q) sh[wid][q] = s[q];
        sh[wid][6] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double *row = partials + (long long)blockIdx.x * kSlots;
        for (int q = 0; q < 6; ++q) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += sh[w][q];
            row[q] = t;
        }
        double t = sh[0][6];
        for (int w = 1; w < kThreads / 32; ++w) t = fmax(t, sh[w][6]);
        row[6] = t;
        row[7] = 0.0;
    }
}

// One block: rows 0..nblocks-1 combined in a fixed order into out[8].
__global__ void __launch_bounds__(kThreads) totals_final(const double *partials, int nblocks, long long n, double E0,
                                                        double *out)
{
    __shared__ double sh[kThreads];
    __shared__ double res[7];
    for (int q = 0; q < 7; ++q) {
        double t = q < 6 ? 0.0 : -1.0;
        for (int b = threadIdx.x; b < nblocks; b += kThreads) {
            const double v = partials[(long long)b * kSlots + q];
            t = q < 6 ? t + v : fmax(t, v);
        }
        sh[threadIdx.x] = t;
        __syncthreads();
        for (int w = kThreads / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w)
                sh[threadIdx.x] = q < 6 ? sh[threadIdx.x] + sh[threadIdx.x + w] : fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
            __syncthreads();
        }
        if (threadIdx.x == 0) res[q] = sh[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double T0 = (E0 + 28.0) / 26.0;
        out[0] = double(n) + res[0];
        out[1] = res[1];
        out[2] = res[2];
        out[3] = double(n) * E0 + res[3];
        out[4] = res[5];
        out[5] = res[6];
        out[6] = T0 + res[4] / double(n);
        out[7] = double(n);
    }
}

// Device address of g_partials, looked up with the device current (in host
// code the name g_partials is only a host-side stand-in) once per device and
// context: the cache is keyed by the context's unique ID, so a context that
// replaced the old one (after cudaDeviceReset) gets its own lookup.
constexpr int kMaxDevices = 64;
struct ScratchEntry {
    unsigned long long ctx_id;
    double *addr;
};
std::mutex g_mutex;
ScratchEntry g_cache[kMaxDevices] = {};

using CtxGetCurrent = CUresult (*)(CUcontext *);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long *);

template <typename Fn>
Fn driver_entry(const char *name)
{
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        return reinterpret_cast<Fn>(ptr);
    return nullptr;
}

// Unique ID of the current context (0 if the driver cannot tell).
unsigned long long current_context_id()
{
    static const CtxGetCurrent get_current = driver_entry<CtxGetCurrent>("cuCtxGetCurrent");
    static const CtxGetId get_id = driver_entry<CtxGetId>("cuCtxGetId");
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// The caller has made `device` current.
cudaError_t scratch_address(int device, double **out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lock(g_mutex);
    ScratchEntry &c = g_cache[device];
    if (!c.addr || id == 0 || c.ctx_id != id) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return e;
        c.addr = static_cast<double *>(p);
        c.ctx_id = id;
    }
    *out = c.addr;
    return cudaSuccess;
}

// Makes `dev` current for the call and restores the caller's device after it;
// ok is false when the device could not be made current.
struct Guard {
    int prev = -1;
    bool ok = false;
    explicit Guard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            prev = -1;
            return;
        }
        ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
    }
    ~Guard()
    {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

template <typename T>
cudaError_t launch_totals(const StateView &v, int nblocks, double *scratch)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(nblocks));
    cfg.blockDim = dim3(kThreads);
    cfg.stream = v.stream;
    return cudaLaunchKernelEx(&cfg, totals_kernel<T>, static_cast<const T *>(v.f), v.nx, v.ny, v.pitch, v.plane, v.E0,
                              v.gx, v.gy, v.rho_ref, v.heat, scratch);
}

} // namespace

extern "C" int lbm13_totals_noalloc(lbm13_t h, double *out)
{
    StateView v;
    if (!h || !out || !lbm13_state_view(h, &v)) return LBM13_EINVAL;
    const long long n = (long long)v.nx * v.ny;
    if (n > LBM13_NOALLOC_MAX_NODES) return LBM13_EINVAL;
    Guard g(v.device);
    if (!g.ok) return LBM13_ECUDA;
    double *scratch = nullptr;
    if (scratch_address(v.device, &scratch) != cudaSuccess) return LBM13_ECUDA;
    const int nblocks = int((n + kNodesPerBlock - 1) / kNodesPerBlock);
    // each launch's own status (not the thread's last-error slot, which may
    // hold an unrelated earlier failure)
    cudaError_t e = v.precision == LBM13_FP64 ? launch_totals<double>(v, nblocks, scratch)
                                              : launch_totals<float>(v, nblocks, scratch);
    if (e != cudaSuccess) return LBM13_ECUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = v.stream;
    e = cudaLaunchKernelEx(&cfg, totals_final, static_cast<const double *>(scratch), nblocks, n, v.E0, out);
    return e == cudaSuccess ? LBM13_OK : LBM13_ECUDA;
}
