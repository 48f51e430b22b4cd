// lbm13_stepdev.cuh -- device code of one time step shared by the per-step
// kernels (lbm13_step.cu) and the persistent multi-step kernel (lbm13_multi.cu):
// the wall state and corrections of a wall position, the resolution of links
// that cross an edge, and the fused pull + collide + store of a column.
//
// The including file defines LBM13_LDG(p), the load used for populations and
// wall corrections: the read-only path (__ldg) where a launch only reads what
// earlier launches wrote, an L2-coherent load (__ldcg) where one launch reads
// what its other blocks wrote before a grid barrier.  The arithmetic is the
// same in both, so both give bit-identical results.
#pragma once

#include "lbm13_internal.h"

#ifndef LBM13_LDG
#error "define LBM13_LDG(p) before including lbm13_stepdev.cuh"
#endif

namespace lbm13 {

namespace {

template <typename T, typename C>
__device__ __forceinline__ C ld(const StepArgs<T, C> &a, int j, int x, int y)
{
    return C(LBM13_LDG(a.fin + (long long)j * a.plane + (long long)y * a.pitch + x));
}

// ------------------------------------------------------ boundary links

// Wall state at position `pos` along side `s`: st = (drho_w, dE_w).
template <typename T, typename C>
__device__ void wall_state(const StepArgs<T, C> &a, int s, int pos, C st[2])
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
        // distance-2 link from both nodes): rho_w = out / (e_unit + 2 e_two),
        // e the even parts at unit density (zf_ea, zf_eb)
        const int ja = s == WEST ? 3 : s == EAST ? 1 : s == SOUTH ? 4 : 2;
        const int jb = s == WEST ? 11 : s == EAST ? 9 : s == SOUTH ? 12 : 10;
        const C dout = g0[ja] + g0[jb] + g1[jb];
        drho = (dout - w.zf_ea - C(2) * w.zf_eb) / (w.wsum + w.zf_ea + C(2) * w.zf_eb);
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
}

// a0 + a1 x + a2 y + a3 x^2 + a4 x y (a wall correction from the wall state).
template <typename C>
__device__ __forceinline__ C wall_poly(const C p[5], C x, C y)
{
    return p[0] + x * (p[1] + x * p[3] + y * p[4]) + y * p[2];
}

// One wall position (or corner) of one lattice: items below 2 ny are the
// west/east positions, then 2 nx south/north positions, then the 4 corners.
// The corrections (2 f_eq,odd of the entering link for bounce-back, 2
// f_eq,even for anti-bounce-back, at the wall state) are evaluated from their
// exact quadratic form in the wall state's (drho, dE).
template <typename T, typename C>
__device__ void wall_item(const StepArgs<T, C> &a, int item)
{
    const int nx = a.nx, ny = a.ny;
    C st[2];
    if (item < 2 * ny + 2 * nx) {
        const int s = item < 2 * ny ? (item < ny ? WEST : EAST) : (item - 2 * ny < nx ? SOUTH : NORTH);
        const int pos = item < 2 * ny ? item % ny : (item - 2 * ny) % nx;
        const WallArgs<C> &w = a.wall[s];
        if (w.kind == PERIODIC || !w.needs_data) return;
        wall_state(a, s, pos, st);
        C *out = a.corr + ((long long)s * a.corr_stride + pos) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) out[i] = wall_poly(w.poly[i], st[0], st[1]);
    } else if (item < 2 * ny + 2 * nx + 4) {
        const int c = item - 2 * ny - 2 * nx;
        const int sx = (c & 1) ? EAST : WEST, sy = (c & 2) ? NORTH : SOUTH;
        if (a.per_x || a.per_y || !(a.wall[sx].needs_data || a.wall[sy].needs_data)) return;
        C s1[2], s2[2];
        wall_state(a, sx, (c & 2) ? ny - 1 : 0, s1);
        wall_state(a, sy, (c & 1) ? nx - 1 : 0, s2);
        a.corr[16LL * a.corr_stride + c] =
            wall_poly(a.corner_poly[c], C(0.5) * (s1[0] + s2[0]), C(0.5) * (s1[1] + s2[1]));
    }
}

// Value of link j of node (x, y) whose source lies beyond side `side` only.
template <typename T, typename C>
__device__ __forceinline__ C cross_wall(const StepArgs<T, C> &a, int side, int j, int x, int y)
{
    const int jb = copp(j);
    const WallArgs<C> &w = a.wall[side];
    const bool xwall = side <= EAST;
    const int pos = xwall ? y : x;
    const C add = w.needs_data ? LBM13_LDG(a.corr + ((long long)side * a.corr_stride + pos) * 4 + wall_slot(side, j))
                               : C(0);
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
    // Branch-free: every link's source offset, sign and correction are chosen
    // with selects, so the 13 population loads (and the corrections) are
    // independent and in flight together.
    const int nx = a.nx, ny = a.ny;
    const bool px = a.per_x != 0, py = a.per_y != 0;
    const bool west = x <= 1, south = y <= 1;
    const int kind_x = west ? a.wall[WEST].kind : a.wall[EAST].kind;
    const int kind_y = south ? a.wall[SOUTH].kind : a.wall[NORTH].kind;
    const bool nd_x = (west ? a.wall[WEST].needs_data : a.wall[EAST].needs_data) != 0;
    const bool nd_y = (south ? a.wall[SOUTH].needs_data : a.wall[NORTH].needs_data) != 0;
    const long long st = a.corr_stride;
    const long long row_x = ((long long)(west ? WEST : EAST) * st + y) * 4;
    const long long row_y = ((long long)(south ? SOUTH : NORTH) * st + x) * 4;
    const long long corner = 16LL * st + (west ? 0 : 1) + (south ? 0 : 2);
    C v[Q], ad[Q];
    unsigned cross = 0u, neg = 0u;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        int sx = x - cvx(j), sy = y - cvy(j);
        const bool bx = sx < 0 || sx >= nx, by = sy < 0 || sy >= ny;
        const bool ox = bx && !px, oy = by && !py;
        sx += sx < 0 ? nx : (sx >= nx ? -nx : 0);
        sy += sy < 0 ? ny : (sy >= ny ? -ny : 0);
        const bool c = ox || oy, both = ox && oy;
        int xs = c ? x : sx, ys = c ? y : sy;
        if (cvy(j) == 0 && (cvx(j) == 2 || cvx(j) == -2) && ox) xs = west ? 1 - x : 2 * nx - 3 - x;
        if (cvx(j) == 0 && (cvy(j) == 2 || cvy(j) == -2) && oy) ys = south ? 1 - y : 2 * ny - 3 - y;
        const int js = c ? copp(j) : j;
        const bool n = (ox && !oy && cvy(j) == 0 && kind_x == WALL_MIXED) ||
                       (oy && !ox && cvx(j) == 0 && kind_y == WALL_MIXED);
        const bool has = both ? (nd_x || nd_y) : (ox ? nd_x : (oy ? nd_y : false));
        const int slot_x = west ? wall_slot(WEST, j) : wall_slot(EAST, j);
        const int slot_y = south ? wall_slot(SOUTH, j) : wall_slot(NORTH, j);
        const long long coff = both ? corner : (ox ? row_x + slot_x : row_y + slot_y);
        v[j] = C(LBM13_LDG(a.fin + (long long)js * a.plane + (long long)ys * a.pitch + xs));
        ad[j] = has ? C(LBM13_LDG(a.corr + coff)) : C(0);
        cross |= (c ? 1u : 0u) << j;
        neg |= (n ? 1u : 0u) << j;
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const C w = ((neg >> j) & 1u) ? -v[j] : v[j];
        f[j] = ((cross >> j) & 1u) ? w + ad[j] : v[j];
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
                f[r][j] = C(LBM13_LDG(base + (long long)j * a.plane + (long long)(r - cvy(j)) * a.pitch + xs));
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

} // namespace

} // namespace lbm13
