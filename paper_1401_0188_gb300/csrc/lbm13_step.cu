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

namespace lbm13 {

namespace {

template <typename T, typename C>
__device__ __forceinline__ C ld(const StepArgs<T, C> &a, int j, int x, int y)
{
    return C(__ldg(a.fin + (long long)j * a.plane + (long long)y * a.pitch + x));
}

// ------------------------------------------------------ boundary links

// Wall state at position `pos` along side `s`: st = (drho_w, dE_w, ux_w, uy_w).
template <typename T, typename C>
__device__ void wall_state(const StepArgs<T, C> &a, int s, int pos, C st[4])
{
    const WallArgs<C> &w = a.wall[s];
    int x0, y0, x1, y1;
    if (s == WEST) { x0 = 0; x1 = 1; y0 = y1 = pos; }
    else if (s == EAST) { x0 = a.nx - 1; x1 = a.nx - 2; y0 = y1 = pos; }
    else if (s == SOUTH) { y0 = 0; y1 = 1; x0 = x1 = pos; }
    else { y0 = a.ny - 1; y1 = a.ny - 2; x0 = x1 = pos; }
    C g0[Q], g1[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        g0[j] = ld(a, j, x0, y0);
        g1[j] = ld(a, j, x1, y1);
    }
    C drho;
    if (w.kind == WALL_MIXED && w.mass_flux) {
        // every even moment of the wall equilibrium is proportional to rho_w,
        // so the anti-bounce-back links return 2 rho_w e_j; rho_w balances the
        // outgoing normal populations (unit link from the first node, the
        // distance-2 link from both nodes): rho_w = out / (e_unit + 2 e_two)
        const int ja = s == WEST ? 3 : s == EAST ? 1 : s == SOUTH ? 4 : 2;
        const int jb = s == WEST ? 11 : s == EAST ? 9 : s == SOUTH ? 12 : 10;
        C e[Q];
        equilibrium_dev(C(0), w.eT + C(13) * (w.ux * w.ux + w.uy * w.uy), w.ux, w.uy, a.k, e);
        const C ea = C(0.5) * (e[ja] + e[copp(ja)]), eb = C(0.5) * (e[jb] + e[copp(jb)]);
        const C dout = g0[ja] + g0[jb] + g1[jb];
        drho = (dout - ea - C(2) * eb) / (w.wsum + ea + C(2) * eb);
    } else {
        drho = C(1.5) * mass_dev(g0) - C(0.5) * mass_dev(g1);
    }
    const C rho = C(1) + drho;
    C dE;
    if (w.kind == WALL_MIXED)
        dE = drho * w.base + w.eT + C(13) * rho * (w.ux * w.ux + w.uy * w.uy);
    else
        dE = C(1.5) * energy_dev(g0) - C(0.5) * energy_dev(g1);
    st[0] = drho;
    st[1] = dE;
    st[2] = w.ux;
    st[3] = w.uy;
}

template <typename C>
__device__ __forceinline__ void wall_feq(const Coef<C> &k, const C st[4], C feq[Q])
{
    const C rho = C(1) + st[0];
    equilibrium_dev(st[0], st[1], rho * st[2], rho * st[3], k, feq);
}

// One wall position (or corner) of one lattice: items below 2 ny are the
// west/east positions, then 2 nx south/north positions, then the 4 corners.
template <typename T, typename C>
__device__ void wall_item(const StepArgs<T, C> &a, int item)
{
    const int nx = a.nx, ny = a.ny;
    C st[4], feq[Q];
    if (item < 2 * ny + 2 * nx) {
        const int s = item < 2 * ny ? (item < ny ? WEST : EAST) : (item - 2 * ny < nx ? SOUTH : NORTH);
        const int pos = item < 2 * ny ? item % ny : (item - 2 * ny) % nx;
        const WallArgs<C> &w = a.wall[s];
        if (w.kind == PERIODIC || !w.needs_data) return;
        wall_state(a, s, pos, st);
        wall_feq(a.k, st, feq);
        C *out = a.corr + ((long long)s * a.corr_stride + pos) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int j = wall_link(s, i), jb = copp(j);
            const bool normal = s <= EAST ? cvy(j) == 0 : cvx(j) == 0;
            out[i] = (w.kind == WALL_MIXED && normal) ? feq[j] + feq[jb] : feq[j] - feq[jb];
        }
    } else if (item < 2 * ny + 2 * nx + 4) {
        const int c = item - 2 * ny - 2 * nx;
        const int sx = (c & 1) ? EAST : WEST, sy = (c & 2) ? NORTH : SOUTH;
        if (a.per_x || a.per_y || !(a.wall[sx].needs_data || a.wall[sy].needs_data)) return;
        C s1[4], s2[4];
        wall_state(a, sx, (c & 2) ? ny - 1 : 0, s1);
        wall_state(a, sy, (c & 1) ? nx - 1 : 0, s2);
#pragma unroll
        for (int i = 0; i < 4; ++i) st[i] = C(0.5) * (s1[i] + s2[i]);
        wall_feq(a.k, st, feq);
        const int j = corner_link(c);
        a.corr[16LL * a.corr_stride + c] = feq[j] - feq[copp(j)];
    }
}

template <typename T, typename C>
__global__ void __launch_bounds__(128) wall_kernel(const StepArgs<T, C> a)
{
    wall_item(a, blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T, typename C>
__global__ void __launch_bounds__(128) batch_wall_kernel(const BatchDesc<T, C> *__restrict__ descs,
                                                        const int *__restrict__ lats, int parity)
{
    const StepArgs<T, C> &a = descs[lats[blockIdx.x]].a[parity];
    const int items = 2 * (a.nx + a.ny) + 4;
    for (int i = threadIdx.x; i < items; i += blockDim.x) wall_item(a, i);
}

// Value of link j of node (x, y) whose source lies beyond side `side` only.
template <typename T, typename C>
__device__ __forceinline__ C cross_wall(const StepArgs<T, C> &a, int side, int j, int x, int y)
{
    const int jb = copp(j);
    const WallArgs<C> &w = a.wall[side];
    const bool xwall = side <= EAST;
    const int pos = xwall ? y : x;
    const C add = w.needs_data ? a.corr[((long long)side * a.corr_stride + pos) * 4 + wall_slot(side, j)] : C(0);
    const bool normal = xwall ? cvy(j) == 0 : cvx(j) == 0;
    if (!normal) return ld(a, jb, x, y) + add;
    int xf = x, yf = y;
    if (xwall && (cvx(j) == 2 || cvx(j) == -2)) xf = side == WEST ? 1 - x : 2 * a.nx - 3 - x;
    if (!xwall && (cvy(j) == 2 || cvy(j) == -2)) yf = side == SOUTH ? 1 - y : 2 * a.ny - 3 - y;
    const C v = ld(a, jb, xf, yf);
    return (w.kind == WALL_MIXED ? -v : v) + add;
}

// Every link of one node resolved on its own (warps on the bottom/top rows).
template <typename T, typename C>
__device__ __noinline__ void gather_general(const StepArgs<T, C> &a, int x, int y, C f[Q])
{
    int sxd = -1, syd = -1;
    if (!a.per_x) sxd = x <= 1 ? WEST : (x >= a.nx - 2 ? EAST : -1);
    if (!a.per_y) syd = y <= 1 ? SOUTH : (y >= a.ny - 2 ? NORTH : -1);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        int sx = x - cvx(j), sy = y - cvy(j);
        bool ox = false, oy = false;
        if (sx < 0 || sx >= a.nx) {
            if (a.per_x) sx += sx < 0 ? a.nx : -a.nx;
            else ox = true;
        }
        if (sy < 0 || sy >= a.ny) {
            if (a.per_y) sy += sy < 0 ? a.ny : -a.ny;
            else oy = true;
        }
        if (!ox && !oy) {
            f[j] = ld(a, j, sx, sy);
        } else if (ox && oy) {
            const int c = (sxd == EAST ? 1 : 0) + (syd == NORTH ? 2 : 0);
            const C add = (a.wall[sxd].needs_data || a.wall[syd].needs_data) ? a.corr[16LL * a.corr_stride + c] : C(0);
            f[j] = ld(a, copp(j), x, y) + add;
        } else {
            f[j] = cross_wall(a, ox ? sxd : syd, j, x, y);
        }
    }
}

template <typename T, typename C>
__device__ __forceinline__ void store(const StepArgs<T, C> &a, int x, int y, const C f[Q])
{
    T *p = a.fout + (long long)y * a.pitch + x;
#pragma unroll
    for (int j = 0; j < Q; ++j) p[(long long)j * a.plane] = T(f[j]);
}

// ------------------------------------------------------------- the step

// One thread: R consecutive rows y0..y0+R-1 of column x.  A warp whose rows
// are all at least two rows away from the bottom and top edges loads its 13
// pulls with the source column clamped into the lattice (uniform code, always
// in bounds); lanes within two columns of the left or right edge then replace
// the links that cross that edge (periodic wrap, or the wall rule with the
// precomputed correction).  Warps on the bottom or top rows resolve every node
// with gather_general through `slot`, this thread's shared-memory row.
template <typename T, typename C, bool Force, int R>
__device__ __forceinline__ void process_column(const StepArgs<T, C> &a, int x, int y0, C *slot)
{
    const int nx = a.nx, ny = a.ny;
    const bool yin = y0 >= 2 && y0 + R <= ny - 2;
    if (__all_sync(0xffffffffu, yin)) {
        C f[R][Q];
        const T *base = a.fin + (long long)y0 * a.pitch;
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const int xs = min(max(x - cvx(j), 0), nx - 1);
                f[r][j] = C(__ldg(base + (long long)j * a.plane + (long long)(r - cvy(j)) * a.pitch + xs));
            }
        }
        if (x >= nx) return;
        if (x < 2 || x >= nx - 2) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    if (cvx(j) == 0) continue;
                    const int sx = x - cvx(j);
                    if (sx >= 0 && sx < nx) continue;
                    if (a.per_x)
                        f[r][j] = ld(a, j, sx < 0 ? sx + nx : sx - nx, y0 + r - cvy(j));
                    else
                        f[r][j] = cross_wall(a, sx < 0 ? WEST : EAST, j, x, y0 + r);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            collide<Force>(f[r], a.k);
            store(a, x, y0 + r, f[r]);
        }
    } else if (x < nx) {
        for (int r = 0; r < R; ++r) {
            const int y = y0 + r;
            if (y >= ny) break;
            C f[Q];
            gather_general(a, x, y, slot);
#pragma unroll
            for (int j = 0; j < Q; ++j) f[j] = slot[j];
            collide<Force>(f, a.k);
            store(a, x, y, f);
        }
    }
}

// One lattice: block 32 x 4 threads, each thread R rows of one column.
template <typename T, typename C, bool Force, int R>
__global__ void __launch_bounds__(128) step_kernel(const StepArgs<T, C> a)
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
cudaError_t launch_walls(const StepArgs<T, C> &a, cudaStream_t s)
{
    if (!a.any_wall_data) return cudaSuccess;
    const int items = 2 * (a.nx + a.ny) + 4;
    wall_kernel<T, C><<<(items + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t launch_batch_walls(const BatchDesc<T, C> *descs, const int *lats, int nlats, int parity, cudaStream_t s)
{
    if (nlats <= 0) return cudaSuccess;
    batch_wall_kernel<T, C><<<nlats, 128, 0, s>>>(descs, lats, parity);
    return cudaGetLastError();
}

template <typename T, typename C>
cudaError_t launch_step(const StepArgs<T, C> &a, bool force, cudaStream_t s)
{
    constexpr int R = sizeof(T) == 8 ? 1 : 2;
    constexpr int BY = 4;
    cudaError_t e = launch_walls(a, s);
    if (e != cudaSuccess) return e;
    dim3 block(32, BY);
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

template cudaError_t launch_walls<double, double>(const StepArgs<double, double> &, cudaStream_t);
template cudaError_t launch_walls<float, float>(const StepArgs<float, float> &, cudaStream_t);
template cudaError_t launch_batch_walls<double, double>(const BatchDesc<double, double> *, const int *, int, int,
                                                        cudaStream_t);
template cudaError_t launch_batch_walls<float, float>(const BatchDesc<float, float> *, const int *, int, int,
                                                      cudaStream_t);
template cudaError_t launch_step<double, double>(const StepArgs<double, double> &, bool, cudaStream_t);
template cudaError_t launch_step<float, float>(const StepArgs<float, float> &, bool, cudaStream_t);
template cudaError_t launch_batch<double, double>(const BatchDesc<double, double> *, const int2 *, int, int, int, int,
                                                  int, int, cudaStream_t);
template cudaError_t launch_batch<float, float>(const BatchDesc<float, float> *, const int2 *, int, int, int, int, int,
                                                int, cudaStream_t);

} // namespace lbm13
