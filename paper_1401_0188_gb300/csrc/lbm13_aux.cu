// lbm13_aux.cu -- initialisation, moment read-out and the FP64 reductions.
//
// Read-outs and reductions run in double precision in both storage modes
// (a float deviation converts to double exactly).  The reductions are
// deterministic: each thread sums its nodes in a fixed grid-stride order, a
// block combines its threads with warp shuffles and a fixed shared-memory tree,
// and one block combines the per-block partials in index order.
#include "lbm13_internal.h"

namespace lbm13 {

namespace {

template <typename T>
__device__ __forceinline__ void load_node(const ReadArgs<T> &a, long long idx, double f[Q])
{
#pragma unroll
    for (int j = 0; j < Q; ++j) f[j] = double(a.f[(long long)j * a.plane + idx]);
}

// ---------------------------------------------------------------- init

// f*_j = f_eq,j(rho, rho u, E) with E = rho (26 T - 28) + 13 rho |u|^2, stored as
// the deviation from the rest populations.
template <typename T>
__global__ void init_kernel(T *f, int nx, int ny, long long pitch, long long plane, const Coef<double> k,
                            const double *__restrict__ rho, const double *__restrict__ ux,
                            const double *__restrict__ uy, const double *__restrict__ Tf)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= nx) return;
    const long long i = (long long)y * nx + x;
    const double r = rho[i], u = ux[i], v = uy[i], t = Tf[i];
    const double dE = r * (26.0 * t - 28.0) - k.E0 + 13.0 * r * (u * u + v * v);
    double g[Q];
    equilibrium_dev(r - 1.0, dE, r * u, r * v, k, g);
    T *p = f + (long long)y * pitch + x;
#pragma unroll
    for (int j = 0; j < Q; ++j) p[(long long)j * plane] = T(g[j]);
}

// -------------------------------------------------------------- moments

struct NodeFields {
    double m[Q];  // absolute moments
    double ux, uy, T, p;
};

// The read-out fields that need only the conserved moments (rho, E, j):
// rho, E, j_x, j_y, u_x, u_y, T, p and the Sec. 7 energy.
constexpr unsigned kConservedFields = (1u << 0) | (1u << 1) | (1u << 4) | (1u << 5) | (1u << 13) | (1u << 14) |
                                      (1u << 15) | (1u << 16) | (1u << 17);

// All 13 moments and the derived fields of a node; Conserved = true leaves the
// nine non-conserved moments unset, so that their arithmetic is dropped (the
// same code, so the conserved ones and the derived fields are identical).
template <typename T, bool Conserved = false>
__device__ __forceinline__ void node_fields(const ReadArgs<T> &a, long long idx, NodeFields &o)
{
    double f[Q];
    load_node(a, idx, f);
    Mom<double> d;
    forward(f, d);
    o.m[0] = 1.0 + d.rho;
    o.m[1] = a.rest.E0 + d.E;
    o.m[4] = d.jx;
    o.m[5] = d.jy;
    if (!Conserved) {
        o.m[2] = a.rest.eps0 + d.eps;
        o.m[3] = a.rest.vpi0 + d.vpi;
        o.m[6] = d.qx;
        o.m[7] = d.qy;
        o.m[8] = d.rx;
        o.m[9] = d.ry;
        o.m[10] = d.XX;
        o.m[11] = d.XY;
        o.m[12] = d.XXe;
    }
    const double rho = o.m[0];
    const double w = rho - a.rho_ref;
    o.ux = (d.jx - 0.5 * w * a.gx) / rho;
    o.uy = (d.jy - 0.5 * w * a.gy) / rho;
    o.p = (o.m[1] + 28.0 * rho) / 26.0 - (d.jx * d.jx + d.jy * d.jy) / (2.0 * rho) - 0.5 * a.heat;
    o.T = o.p / rho;
}

template <typename T>
__global__ void moments_kernel(const ReadArgs<T> a, double *__restrict__ out, unsigned mask)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.nx) return;
    NodeFields o;
    if ((mask & ~kConservedFields) == 0u)
        node_fields<T, true>(a, (long long)y * a.pitch + x, o);
    else
        node_fields<T, false>(a, (long long)y * a.pitch + x, o);
    const long long n = (long long)a.nx * a.ny, i = (long long)y * a.nx + x;
    int plane = 0;
    for (int b = 0; b < 18; ++b) {
        if (!((mask >> b) & 1u)) continue;
        double v;
        if (b < Q) v = o.m[b];
        else if (b == 13) v = o.ux;
        else if (b == 14) v = o.uy;
        else if (b == 15) v = o.T;
        else if (b == 16) v = o.p;
        else v = o.m[1] - 6.5 * (o.ux * o.ux + o.uy * o.uy);
        out[plane * n + i] = v;
        ++plane;
    }
}

// ----------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Combine NS sums and NM maxima across the block; thread 0 writes them.
template <int NS, int NM>
__device__ void block_combine(double (&s)[NS], double (&mx)[NM], double *dst)
{
    __shared__ double sh[kReduceThreads / 32][kPartials];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NS; ++i) s[i] = warp_sum(s[i]);
#pragma unroll
    for (int i = 0; i < NM; ++i) mx[i] = warp_max(mx[i]);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NS; ++i) sh[wid][i] = s[i];
#pragma unroll
        for (int i = 0; i < NM; ++i) sh[wid][NS + i] = mx[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) {
            double t = 0.0;
            for (int w = 0; w < kReduceThreads / 32; ++w) t += sh[w][i];
            dst[i] = t;
        }
        for (int i = 0; i < NM; ++i) {
            double t = sh[0][NS + i];
            for (int w = 1; w < kReduceThreads / 32; ++w) t = fmax(t, sh[w][NS + i]);
            dst[NS + i] = t;
        }
    }
}

// Pass 1 partials: 0 sum drho, 1 sum jx, 2 sum jy, 3 sum dE, 4 sum ux, 5 sum uy,
// 6 sum (T - T0), 7 non-finite count, 8 max |u|.
template <typename T>
__global__ void __launch_bounds__(kReduceThreads) fields_kernel(const ReadArgs<T> a, ReduceBufs b, double T0)
{
    const long long n = (long long)a.nx * a.ny;
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double mx[1] = {0.0};
    for (long long i = (long long)blockIdx.x * kReduceThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kReduceThreads) {
        const int y = int(i / a.nx), x = int(i - (long long)y * a.nx);
        const long long idx = (long long)y * a.pitch + x;
        double f[Q];
        load_node(a, idx, f);
        double bad = 0.0;
#pragma unroll
        for (int j = 0; j < Q; ++j) bad += isfinite(f[j]) ? 0.0 : 1.0;
        Mom<double> d;
        forward(f, d);
        const double rho = 1.0 + d.rho;
        const double w = rho - a.rho_ref;
        const double ux = (d.jx - 0.5 * w * a.gx) / rho, uy = (d.jy - 0.5 * w * a.gy) / rho;
        const double p = (a.rest.E0 + d.E + 28.0 * rho) / 26.0 - (d.jx * d.jx + d.jy * d.jy) / (2.0 * rho) -
                         0.5 * a.heat;
        const double Tn = p / rho;
        b.fields[i] = ux;
        b.fields[n + i] = uy;
        b.fields[2 * n + i] = Tn;
        s[0] += d.rho;
        s[1] += d.jx;
        s[2] += d.jy;
        s[3] += d.E;
        s[4] += ux;
        s[5] += uy;
        s[6] += Tn - T0;
        s[7] += bad;
        const double um = sqrt(ux * ux + uy * uy);
        mx[0] = isnan(um) ? mx[0] : fmax(mx[0], um);
    }
    block_combine<8, 1>(s, mx, b.partials + (long long)blockIdx.x * kPartials);
}

// Sums of the partials of nblocks blocks, slot by slot in block order;
// slots >= nsum take the maximum instead.
__device__ void combine_partials(const double *partials, int nblocks, int nsum, int nmax, double *res)
{
    __shared__ double sh[kReduceThreads];
    for (int i = 0; i < nsum + nmax; ++i) {
        double t = i < nsum ? 0.0 : -1.0;
        for (int bI = threadIdx.x; bI < nblocks; bI += kReduceThreads) {
            const double v = partials[(long long)bI * kPartials + i];
            t = i < nsum ? t + v : fmax(t, v);
        }
        sh[threadIdx.x] = t;
        __syncthreads();
        for (int w = kReduceThreads / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sh[threadIdx.x] = i < nsum ? sh[threadIdx.x] + sh[threadIdx.x + w]
                                                           : fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
            __syncthreads();
        }
        if (threadIdx.x == 0) res[i] = sh[0];
        __syncthreads();
    }
}

// stats after pass 1: 0 mean ux, 1 mean uy, 2 mean T, 3..11 the combined pass-1 slots.
__global__ void __launch_bounds__(kReduceThreads) finalize1_kernel(ReduceBufs b, long long n, double T0)
{
    __shared__ double res[9];
    combine_partials(b.partials, b.nblocks, 8, 1, res);
    if (threadIdx.x == 0) {
        b.stats[0] = res[4] / double(n);
        b.stats[1] = res[5] / double(n);
        b.stats[2] = T0 + res[6] / double(n);
        for (int i = 0; i < 9; ++i) b.stats[3 + i] = res[i];
    }
}

// Pass 2 partials: 0..2 sum (F - snap)^2, 3..5 sum (F - mean F)^2 for F = ux, uy, T;
// 6 Nusselt sum; 7 S_u max, 8 S_T max.
template <typename T>
__global__ void __launch_bounds__(kReduceThreads) residual_kernel(const ReadArgs<T> a, ReduceBufs b, ReduceConf c)
{
    const long long n = (long long)a.nx * a.ny;
    const double mean[3] = {b.stats[0], b.stats[1], b.stats[2]};
    const double Tref_asym = c.asym_walls ? c.Tasym : mean[2];
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    double mx[2] = {0.0, 0.0};
    const double *F[3] = {b.fields, b.fields + n, b.fields + 2 * n};
    for (long long i = (long long)blockIdx.x * kReduceThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kReduceThreads) {
        const int y = int(i / a.nx), x = int(i - (long long)y * a.nx);
        double v[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            v[q] = F[q][i];
            if (c.have_snap) {
                const double dv = v[q] - b.snap[q * n + i];
                s[q] += dv * dv;
            }
            const double e = v[q] - mean[q];
            s[3 + q] += e * e;
            b.snap[q * n + i] = v[q];
        }
        if (c.nusselt) {
            const double *Tf = F[2];
            double dTdx;
            if (x == 0) dTdx = (-3.0 * Tf[i] + 4.0 * Tf[i + 1] - Tf[i + 2]) / 2.0;
            else if (x == a.nx - 1) dTdx = (3.0 * Tf[i] - 4.0 * Tf[i - 1] + Tf[i - 2]) / 2.0;
            else dTdx = (Tf[i + 1] - Tf[i - 1]) / 2.0;
            s[6] += v[0] * (v[2] - c.Tref) - c.kappa * dTdx;
        }
        const long long m = (long long)(a.ny - 1 - y) * a.nx + (a.nx - 1 - x);
        const double sx = v[0] + F[0][m], sy = v[1] + F[1][m];
        const double su = sqrt(sx * sx + sy * sy);
        const double st = fabs((v[2] - Tref_asym) + (F[2][m] - Tref_asym));
        mx[0] = isnan(su) ? mx[0] : fmax(mx[0], su);
        mx[1] = isnan(st) ? mx[1] : fmax(mx[1], st);
    }
    block_combine<7, 2>(s, mx, b.partials + (long long)blockIdx.x * kPartials);
}

__global__ void __launch_bounds__(kReduceThreads) finalize2_kernel(ReduceBufs b, ReduceConf c, long long n, int ny,
                                                                   double E0, double *out)
{
    __shared__ double res[9];
    combine_partials(b.partials, b.nblocks, 7, 2, res);
    if (threadIdx.x == 0) {
        // the velocity is one vector field: both components over its variation
        const double floor_ = 1e-6 * sqrt(double(n));
        for (int q = 0; q < 4; ++q) out[q] = 0.0;
        if (c.have_snap && c.K > 0) {
            const double du = fmax(sqrt(res[3] + res[4]), floor_), dT = fmax(sqrt(res[5]), floor_);
            const double K = double(c.K);
            out[1] = sqrt(res[0]) / (K * du);
            out[2] = sqrt(res[1]) / (K * du);
            out[3] = sqrt(res[2]) / (K * dT);
            out[0] = fmax(sqrt(res[0] + res[1]) / (K * du), out[3]);
        }
        const double *p1 = b.stats + 3;
        out[4] = double(n) + p1[0];
        out[5] = p1[1];
        out[6] = p1[2];
        out[7] = double(n) * E0 + p1[3];
        out[8] = c.nusselt ? res[6] / (double(ny) * c.kappa * c.dT) : 0.0;
        out[9] = res[7];
        out[10] = res[8];
        out[11] = p1[8];
        out[12] = p1[7];
        out[13] = c.have_snap ? double(c.K) : 0.0;
        out[14] = double(c.step);
        out[15] = b.stats[2];
    }
}

// --------------------------------------------------------- projections

// Deviations of one node from the rest state: rho - 1, ux, uy, T - T0, E - E0,
// p - T0, with u, T and p read half-way through the force and the source.
template <typename T>
__device__ __forceinline__ void node_deviations(const ReadArgs<T> &a, long long idx, double v[6])
{
    double f[Q];
    load_node(a, idx, f);
    Mom<double> d;
    forward(f, d);
    const double rho = 1.0 + d.rho;
    const double w = rho - a.rho_ref;
    const double T0 = (a.rest.E0 + 28.0) / 26.0;
    const double dp = (d.E + 28.0 * d.rho) / 26.0 - (d.jx * d.jx + d.jy * d.jy) / (2.0 * rho) - 0.5 * a.heat;
    v[0] = d.rho;
    v[1] = (d.jx - 0.5 * w * a.gx) / rho;
    v[2] = (d.jy - 0.5 * w * a.gy) / rho;
    v[3] = (dp - T0 * d.rho) / rho;
    v[4] = d.E;
    v[5] = dp;
}

// Per-block partials of the Fourier projections, [block][kProj]:
// slot 4 f + 2 h + c = sum F_f trig_c(2 pi (h + 1) m / N), m = (kx x ny + ky y nx) mod N
// (kx, ky already reduced to [0, nx) x [0, ny)).
template <typename T>
__global__ void __launch_bounds__(kReduceThreads) project_kernel(const ReadArgs<T> a, long long kx, long long ky,
                                                                 double *__restrict__ partials)
{
    const long long n = (long long)a.nx * a.ny;
    double s[kProj];
#pragma unroll
    for (int i = 0; i < kProj; ++i) s[i] = 0.0;
    for (long long i = (long long)blockIdx.x * kReduceThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kReduceThreads) {
        const int y = int(i / a.nx), x = int(i - (long long)y * a.nx);
        double v[6];
        node_deviations(a, (long long)y * a.pitch + x, v);
        const long long m = ((kx * x) % a.nx * a.ny + (ky * y) % a.ny * a.nx) % n;
        double c1, s1, c2, s2;
        sincospi(2.0 * double(m) / double(n), &s1, &c1);
        sincospi(2.0 * double((2 * m) % n) / double(n), &s2, &c2);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            s[4 * q + 0] += v[q] * c1;
            s[4 * q + 1] += v[q] * s1;
            s[4 * q + 2] += v[q] * c2;
            s[4 * q + 3] += v[q] * s2;
        }
    }
    __shared__ double sh[kReduceThreads / 32][kProj];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kProj; ++i) s[i] = warp_sum(s[i]);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < kProj; ++i) sh[wid][i] = s[i];
    }
    __syncthreads();
    if (threadIdx.x < kProj) {
        double t = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) t += sh[w][threadIdx.x];
        partials[(long long)blockIdx.x * kProj + threadIdx.x] = t;
    }
}

// out[i] = sum of the partials of slot i in block order.
__global__ void project_final_kernel(const double *__restrict__ partials, int nblocks, double *__restrict__ out)
{
    const int i = threadIdx.x;
    if (i >= kProj) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partials[(long long)b * kProj + i];
    out[i] = t;
}

} // namespace

template <typename T>
cudaError_t launch_init(T *f, int nx, int ny, long long pitch, long long plane, const Coef<double> &k,
                        const double *rho, const double *ux, const double *uy, const double *Tf, cudaStream_t s)
{
    dim3 block(128), grid((nx + 127) / 128, ny);
    init_kernel<T><<<grid, block, 0, s>>>(f, nx, ny, pitch, plane, k, rho, ux, uy, Tf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_moments(const ReadArgs<T> &a, double *out, unsigned mask, cudaStream_t s)
{
    dim3 block(128), grid((a.nx + 127) / 128, a.ny);
    moments_kernel<T><<<grid, block, 0, s>>>(a, out, mask);
    return cudaGetLastError();
}

// ------------------------------------------------------ y-slab halos
//
// Entry i of a packed halo [2 rows][4 populations][nx]: pack reads the rows
// next to the halo rows of `side` (south: 2, 3; north: ny-4, ny-3) for the
// populations that move across it (south: v_y < 0; north: v_y > 0); unpack
// writes the halo rows (south: 0, 1; north: ny-2, ny-1) for the populations
// that move in (south: v_y > 0; north: v_y < 0).
__device__ __forceinline__ int halo_plane(bool up, int k)
{
    return up ? (k == 0 ? 2 : k == 1 ? 5 : k == 2 ? 6 : 10) : (k == 0 ? 4 : k == 1 ? 7 : k == 2 ? 8 : 12);
}

template <typename T>
__global__ void halo_kernel(T *__restrict__ f, int nx, int ny, long long pitch, long long plane, int side, int pack,
                            T *__restrict__ buf)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8LL * nx) return;
    const int x = int(i % nx), k = int((i / nx) % 4), r = int(i / (4LL * nx));
    const bool south = side == SOUTH;
    const int y = pack ? (south ? 2 + r : ny - 4 + r) : (south ? r : ny - 2 + r);
    const bool up = pack ? !south : south;
    T *p = f + (long long)halo_plane(up, k) * plane + (long long)y * pitch + x;
    if (pack)
        buf[i] = *p;
    else
        *p = buf[i];
}

template <typename T>
cudaError_t launch_halo(T *f, int nx, int ny, long long pitch, long long plane, int side, bool pack, T *buf,
                        cudaStream_t s)
{
    const long long n = 8LL * nx;
    halo_kernel<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(f, nx, ny, pitch, plane, side, pack ? 1 : 0, buf);
    return cudaGetLastError();
}

template cudaError_t launch_halo<double>(double *, int, int, long long, long long, int, bool, double *, cudaStream_t);
template cudaError_t launch_halo<float>(float *, int, int, long long, long long, int, bool, float *, cudaStream_t);

int reduce_blocks(int nx, int ny)
{
    const long long n = (long long)nx * ny;
    long long b = (n + kReduceThreads - 1) / kReduceThreads;
    const long long cap = 8LL * device_sm_count();  // eight blocks per SM
    return int(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <typename T>
cudaError_t launch_reduce(const ReadArgs<T> &a, const ReduceBufs &b, const ReduceConf &c, double *out_dev,
                          cudaStream_t s)
{
    const long long n = (long long)a.nx * a.ny;
    const double T0 = (a.rest.E0 + 28.0) / 26.0;
    fields_kernel<T><<<b.nblocks, kReduceThreads, 0, s>>>(a, b, T0);
    finalize1_kernel<<<1, kReduceThreads, 0, s>>>(b, n, T0);
    residual_kernel<T><<<b.nblocks, kReduceThreads, 0, s>>>(a, b, c);
    finalize2_kernel<<<1, kReduceThreads, 0, s>>>(b, c, n, a.ny, a.rest.E0, out_dev);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_project(const ReadArgs<T> &a, int kx, int ky, double *partials, int nblocks, double *out_dev,
                           cudaStream_t s)
{
    const long long kxm = ((long long)kx % a.nx + a.nx) % a.nx, kym = ((long long)ky % a.ny + a.ny) % a.ny;
    project_kernel<T><<<nblocks, kReduceThreads, 0, s>>>(a, kxm, kym, partials);
    project_final_kernel<<<1, 32, 0, s>>>(partials, nblocks, out_dev);
    return cudaGetLastError();
}

template cudaError_t launch_init<double>(double *, int, int, long long, long long, const Coef<double> &,
                                         const double *, const double *, const double *, const double *,
                                         cudaStream_t);
template cudaError_t launch_init<float>(float *, int, int, long long, long long, const Coef<double> &,
                                        const double *, const double *, const double *, const double *,
                                        cudaStream_t);
template cudaError_t launch_moments<double>(const ReadArgs<double> &, double *, unsigned, cudaStream_t);
template cudaError_t launch_moments<float>(const ReadArgs<float> &, double *, unsigned, cudaStream_t);
template cudaError_t launch_reduce<double>(const ReadArgs<double> &, const ReduceBufs &, const ReduceConf &,
                                           double *, cudaStream_t);
template cudaError_t launch_reduce<float>(const ReadArgs<float> &, const ReduceBufs &, const ReduceConf &,
                                          double *, cudaStream_t);

template cudaError_t launch_project<double>(const ReadArgs<double> &, int, int, double *, int, double *,
                                            cudaStream_t);
template cudaError_t launch_project<float>(const ReadArgs<float> &, int, int, double *, int, double *,
                                           cudaStream_t);

} // namespace lbm13
