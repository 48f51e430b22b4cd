// lbm13_step.cu -- the fused time step: pull-streaming over the 13 links,
// wall rules at the domain edges and the MRT collision, one pass over HBM.
//
// Storage: structure of arrays, population plane j at f + j * plane, row y at
// + y * pitch, x contiguous; pitch is a multiple of 32 elements so every row of
// every plane starts on a 128-byte (float) or 256-byte (double) boundary.  Two
// buffers alternate: the kernel reads the post-collision state f*(t) from
// `fin` and writes f*(t+1) to `fout`.
//
// Streaming is a pull: node x gathers population j from x - v_j.  A warp covers
// 32 consecutive x of one row, so each of its 13 loads per node is one
// coalesced 128/256-byte row segment, shifted by -v_x (0, +-1 or +-2 elements;
// the neighbouring warp reads the other half of the straddled sector, so DRAM
// traffic stays at one read per population); stores are aligned.
//
// Warps whose 32 x R nodes all have their 13 sources inside the lattice (no
// periodic wrap, no wall) take the branch-free path.  The others resolve every
// link on its own: periodic wrap, or the wall rule of the side it crosses:
//   halfway walls, half a link outside the first and last node; a population
//   leaving x_f with velocity -v_j crosses the wall and comes back with v_j
//   to x_f + (2a - 1)(-v_j), a the crossed fraction of the link: the same node
//   for |v_n| = 1 and for the diagonals, the other of the two wall rows for
//   the distance-2 links;
//   bounce-back    f_j(x) = f*_jbar(x_f) + 2 f_eq,odd_j(wall)       (Sec. 9; moving walls)
//   anti-bounce-back f_j(x) = -f*_jbar(x_f) + 2 f_eq,even_j(wall)   (Sec. 7, Eq. d2q13-cl-abb)
// with anti-bounce-back on the links normal to a velocity+temperature wall and
// bounce-back on its diagonal links and on every link of an adiabatic wall.
// The wall state is rho_w = 1.5 rho(first node) - 0.5 rho(second node) (the
// extrapolation of Sec. 7), u_w the wall velocity, and E_w from the wall
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

// Wall state at position `pos` along side `s`: st = (drho_w, dE_w, ux_w, uy_w).
template <typename T, typename C>
__device__ __noinline__ void wall_state(const StepArgs<T, C> &a, int s, int pos, C st[4])
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
    const C drho = C(1.5) * mass_dev(g0) - C(0.5) * mass_dev(g1);
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

// Every link of one node resolved on its own (edge warps).  wx, wy: deviation
// equilibria of the x-side and y-side wall at this node (zero for a wall at
// rest without temperature data, whose corrections vanish); wc: the corner's.
template <typename T, typename C>
__device__ __noinline__ void gather_general(const StepArgs<T, C> &a, int x, int y, C f[Q])
{
    int sxd = -1, syd = -1;
    if (!a.per_x) sxd = x <= 1 ? WEST : (x >= a.nx - 2 ? EAST : -1);
    if (!a.per_y) syd = y <= 1 ? SOUTH : (y >= a.ny - 2 ? NORTH : -1);
    const bool need_x = sxd >= 0 && a.wall[sxd].needs_data;
    const bool need_y = syd >= 0 && a.wall[syd].needs_data;
    const bool corner = sxd >= 0 && syd >= 0 && (need_x || need_y);
    C wx[Q], wy[Q], wc[Q], stx[4], sty[4];
#pragma unroll
    for (int j = 0; j < Q; ++j) wx[j] = wy[j] = wc[j] = C(0);
    if (need_x || corner) wall_state(a, sxd, y, stx);
    if (need_y || corner) wall_state(a, syd, x, sty);
    if (need_x) wall_feq(a.k, stx, wx);
    if (need_y) wall_feq(a.k, sty, wy);
    if (corner) {
        C st[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) st[i] = C(0.5) * (stx[i] + sty[i]);
        wall_feq(a.k, st, wc);
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int jb = copp(j);
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
            f[j] = ld(a, jb, x, y) + (wc[j] - wc[jb]);
        } else if (ox) {
            if (cvy(j) != 0) {
                f[j] = ld(a, jb, x, y) + (wx[j] - wx[jb]);
            } else {
                const int xf = (cvx(j) == 2 || cvx(j) == -2) ? (sxd == WEST ? 1 - x : 2 * a.nx - 3 - x) : x;
                if (a.wall[sxd].kind == WALL_MIXED)
                    f[j] = -ld(a, jb, xf, y) + (wx[j] + wx[jb]);
                else
                    f[j] = ld(a, jb, xf, y) + (wx[j] - wx[jb]);
            }
        } else {
            if (cvx(j) != 0) {
                f[j] = ld(a, jb, x, y) + (wy[j] - wy[jb]);
            } else {
                const int yf = (cvy(j) == 2 || cvy(j) == -2) ? (syd == SOUTH ? 1 - y : 2 * a.ny - 3 - y) : y;
                if (a.wall[syd].kind == WALL_MIXED)
                    f[j] = -ld(a, jb, x, yf) + (wy[j] + wy[jb]);
                else
                    f[j] = ld(a, jb, x, yf) + (wy[j] - wy[jb]);
            }
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

// Block: 32 x BY threads; each thread owns R consecutive rows of one column.
template <typename T, typename C, bool Force, int R>
__global__ void __launch_bounds__(128) step_kernel(const StepArgs<T, C> a)
{
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y0 = (blockIdx.y * blockDim.y + threadIdx.y) * R;
    const bool interior = x >= 2 && x < a.nx - 2 && y0 >= 2 && y0 + R <= a.ny - 2;
    if (__all_sync(0xffffffffu, interior)) {
        C f[R][Q];
        const T *base = a.fin + (long long)y0 * a.pitch + x;
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int j = 0; j < Q; ++j)
                f[r][j] = C(__ldg(base + (long long)j * a.plane + (long long)(r - cvy(j)) * a.pitch - cvx(j)));
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            collide<Force>(f[r], a.k);
            store(a, x, y0 + r, f[r]);
        }
    } else if (x < a.nx) {
        for (int r = 0; r < R; ++r) {
            const int y = y0 + r;
            if (y >= a.ny) break;
            C f[Q];
            gather_general(a, x, y, f);
            collide<Force>(f, a.k);
            store(a, x, y, f);
        }
    }
}

} // namespace

template <typename T, typename C>
cudaError_t launch_step(const StepArgs<T, C> &a, bool force, cudaStream_t s)
{
    constexpr int R = sizeof(T) == 8 ? 1 : 2;
    constexpr int BY = 4;
    dim3 block(32, BY);
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
