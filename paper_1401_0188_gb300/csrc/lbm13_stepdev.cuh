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

// Debug builds (LBM13_DEBUG) check every population access against the
// lattice (plane below 13, row below ny, column below nx): an access outside
// it is counted in *a.bad and redirected to the buffer's first element, so it
// neither faults nor corrupts; release builds pass the pointer through.
template <typename T, typename C, typename P>
__device__ __forceinline__ P *chk(const StepArgs<T, C> &a, P *base, P *p)
{
#ifdef LBM13_DEBUG
    const long long i = p - base;
    bool out = i < 0;
    if (!out) {
        const long long j = i / a.plane, rem = i - j * a.plane;
        const long long y = rem / a.pitch, x = rem - y * a.pitch;
        out = j >= Q || y >= a.ny || x >= a.nx;
    }
    if (out) {
        atomicAdd(a.bad, 1ull);
        return base;
    }
#endif
    return p;
}

template <typename T, typename C>
__device__ __forceinline__ C ld(const StepArgs<T, C> &a, int j, int x, int y)
{
    return C(LBM13_LDG(chk(a, a.fin, a.fin + (long long)j * a.plane + (long long)y * a.pitch + x)));
}

// How the wall and edge code reads population j of node (x, y): from the
// input buffer, with the wall-state code called out of line (GlobalSrc: the
// step kernels, where edge nodes are a few lanes of a warp), or compiled into
// the caller (GlobalInlineSrc: a kernel whose threads step edge nodes only,
// so that every load of a node, the wall state's included, can be in flight
// at once).  The values and the arithmetic are the same either way.
template <typename T, typename C>
struct GlobalSrc {
    static constexpr bool kInline = false;
    __device__ __forceinline__ C operator()(const StepArgs<T, C> &a, int j, int x, int y) const
    {
        return ld(a, j, x, y);
    }
};
template <typename T, typename C>
struct GlobalInlineSrc {
    static constexpr bool kInline = true;
    __device__ __forceinline__ C operator()(const StepArgs<T, C> &a, int j, int x, int y) const
    {
        return ld(a, j, x, y);
    }
};

// ------------------------------------------------------ boundary links

// Wall state (drho_w, dE_w): deviations of the wall's density and energy from
// the rest state.
template <typename C>
struct WallState {
    C rho, E;
};

// The two nodes next to side s at position pos along it: (x0, y0) on the
// wall row or column, (x1, y1) one further in.
template <typename T, typename C>
__device__ __forceinline__ void wall_nodes(const StepArgs<T, C> &a, int s, int pos, int &x0, int &y0, int &x1,
                                           int &y1)
{
    if (s == WEST) { x0 = 0; x1 = 1; y0 = y1 = pos; }
    else if (s == EAST) { x0 = a.nx - 1; x1 = a.nx - 2; y0 = y1 = pos; }
    else if (s == SOUTH) { y0 = 0; y1 = 1; x0 = x1 = pos; }
    else { y0 = a.ny - 1; y1 = a.ny - 2; x0 = x1 = pos; }
}

// The outgoing normal links of side s: the unit link and the distance-2 link.
__device__ __forceinline__ int out_unit(int s) { return s == WEST ? 3 : s == EAST ? 1 : s == SOUTH ? 4 : 2; }
__device__ __forceinline__ int out_two(int s) { return s == WEST ? 11 : s == EAST ? 9 : s == SOUTH ? 12 : 10; }

// Wall state of a temperature wall whose density makes the net normal mass
// flux zero.  Every even moment of the wall equilibrium is proportional to
// rho_w, so the anti-bounce-back links return 2 rho_w e_j; rho_w balances the
// outgoing normal populations (the unit link from the first node, the
// distance-2 link from both nodes): rho_w = out / (e_unit + 2 e_two), e the
// even parts at unit density (zf_ea, zf_eb).  dout = deviation of those three
// populations, summed first node unit, first node distance-2, second node
// distance-2.
template <typename C>
__device__ __forceinline__ WallState<C> zero_flux_state(const WallArgs<C> &w, C dout)
{
    const C drho = (dout - w.zf_ea - C(2) * w.zf_eb) / (w.wsum + w.zf_ea + C(2) * w.zf_eb);
    const C rho = C(1) + drho;
    return {drho, drho * w.base + w.eT + C(13) * rho * (w.ux * w.ux + w.uy * w.uy)};
}

// Wall state at position `pos` along side `s`.
template <typename T, typename C, typename S>
__device__ __forceinline__ WallState<C> wall_state_body(const StepArgs<T, C> &a, int s, int pos, S src)
{
    const WallArgs<C> &w = a.wall[s];
    int x0, y0, x1, y1;
    wall_nodes(a, s, pos, x0, y0, x1, y1);
    if (w.kind == WALL_MIXED && w.mass_flux) {
        const int ja = out_unit(s), jb = out_two(s);
        return zero_flux_state(w, src(a, ja, x0, y0) + src(a, jb, x0, y0) + src(a, jb, x1, y1));
    }
    C g0[Q], g1[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        g0[j] = src(a, j, x0, y0);
        g1[j] = src(a, j, x1, y1);
    }
    const C drho = C(1.5) * mass_dev(g0) - C(0.5) * mass_dev(g1);
    const C rho = C(1) + drho;
    C dE;
    if (w.kind == WALL_MIXED)
        dE = drho * w.base + w.eT + C(13) * rho * (w.ux * w.ux + w.uy * w.uy);
    else
        dE = C(1.5) * energy_dev(g0) - C(0.5) * energy_dev(g1);
    return {drho, dE};
}

// Out of line: only the nodes next to a wall that needs data evaluate it;
// returned by value so that the caller keeps it in registers (no stack frame).
template <typename T, typename C>
__device__ __noinline__ WallState<C> wall_state(const StepArgs<T, C> &a, int s, int pos)
{
    return wall_state_body(a, s, pos, GlobalSrc<T, C>());
}

template <typename T, typename C, typename S>
__device__ __forceinline__ WallState<C> wall_state_of(const StepArgs<T, C> &a, int s, int pos, S src)
{
    if constexpr (S::kInline)
        return wall_state_body(a, s, pos, src);
    else
        return wall_state(a, s, pos);
}

// a0 + a1 x + a2 y + a3 x^2 + a4 x y (a wall correction from the wall state).
template <typename C>
__device__ __forceinline__ C wall_poly(const C p[5], C x, C y)
{
    return p[0] + x * (p[1] + x * p[3] + y * p[4]) + y * p[2];
}

// Value of link j of node (x, y) whose source lies beyond side `side` only;
// st is that side's wall state at the node's position (used when the wall
// needs data).
template <typename T, typename C>
__device__ __forceinline__ C cross_wall(const StepArgs<T, C> &a, int side, int j, int x, int y, WallState<C> st)
{
    const int jb = copp(j);
    const WallArgs<C> &w = a.wall[side];
    const bool xwall = side <= EAST;
    const C add = w.needs_data ? wall_poly(w.poly[wall_slot(side, j)], st.rho, st.E) : C(0);
    const bool normal = xwall ? cvy(j) == 0 : cvx(j) == 0;
    if (!normal) return ld(a, jb, x, y) + add;
    int xf = x, yf = y;
    if (xwall && (cvx(j) == 2 || cvx(j) == -2)) xf = side == WEST ? 1 - x : 2 * a.nx - 3 - x;
    if (!xwall && (cvy(j) == 2 || cvy(j) == -2)) yf = side == SOUTH ? 1 - y : 2 * a.ny - 3 - y;
    const C v = ld(a, jb, xf, yf);
    return (w.kind == WALL_MIXED ? -v : v) + add;
}

// Every link of one node resolved on its own (warps on the bottom/top rows).
template <typename T, typename C, typename S>
__device__ __forceinline__ void gather_body(const StepArgs<T, C> &a, int x, int y, C f[Q], S src)
{
    // Branch-free: every link's source offset and sign are chosen with
    // selects, so the 13 population loads are independent and in flight
    // together.
    const int nx = a.nx, ny = a.ny;
    const bool px = a.per_x != 0, py = a.per_y != 0;
    const bool west = x <= 1, south = y <= 1;
    const int sx_side = west ? WEST : EAST, sy_side = south ? SOUTH : NORTH;
    const int kind_x = a.wall[sx_side].kind, kind_y = a.wall[sy_side].kind;
    const bool nd_x = a.wall[sx_side].needs_data != 0, nd_y = a.wall[sy_side].needs_data != 0;
    // the wall states at this node's position, before the pulls so that
    // they are not live across the calls: a wall's own state where it needs
    // data (a corner node's diagonal takes each crossed wall's correction at
    // that wall's own state, so no other state is needed)
    const bool near_x = !px && (x <= 1 || x >= nx - 2), near_y = !py && (y <= 1 || y >= ny - 2);
    WallState<C> stx = {C(0), C(0)}, sty = {C(0), C(0)};
    if (near_x && nd_x) stx = wall_state_of(a, sx_side, y, src);
    if (near_y && nd_y) sty = wall_state_of(a, sy_side, x, src);
    C v[Q];
    unsigned cross = 0u, neg = 0u, crx = 0u, cry = 0u;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        int sx = x - cvx(j), sy = y - cvy(j);
        const bool bx = sx < 0 || sx >= nx, by = sy < 0 || sy >= ny;
        const bool ox = bx && !px, oy = by && !py;
        sx += sx < 0 ? nx : (sx >= nx ? -nx : 0);
        sy += sy < 0 ? ny : (sy >= ny ? -ny : 0);
        const bool c = ox || oy;
        int xs = c ? x : sx, ys = c ? y : sy;
        if (cvy(j) == 0 && (cvx(j) == 2 || cvx(j) == -2) && ox) xs = west ? 1 - x : 2 * nx - 3 - x;
        if (cvx(j) == 0 && (cvy(j) == 2 || cvy(j) == -2) && oy) ys = south ? 1 - y : 2 * ny - 3 - y;
        const int js = c ? copp(j) : j;
        const bool n = (ox && !oy && cvy(j) == 0 && kind_x == WALL_MIXED) ||
                       (oy && !ox && cvx(j) == 0 && kind_y == WALL_MIXED);
        v[j] = src(a, js, xs, ys);
        cross |= (c ? 1u : 0u) << j;
        neg |= (n ? 1u : 0u) << j;
        crx |= (ox ? 1u : 0u) << j;
        cry |= (oy ? 1u : 0u) << j;
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const bool ox = (crx >> j) & 1u, oy = (cry >> j) & 1u;
        // the correction of each wall the link crosses, at that wall's state:
        // a corner diagonal crosses both and takes both (with the node's two
        // single-wall diagonals they carry no net mass, as on a flat wall)
        C ad = C(0);
        if (ox && nd_x) ad = wall_poly(a.wall[sx_side].poly[west ? wall_slot(WEST, j) : wall_slot(EAST, j)], stx.rho, stx.E);
        if (oy && nd_y)
            ad += wall_poly(a.wall[sy_side].poly[south ? wall_slot(SOUTH, j) : wall_slot(NORTH, j)], sty.rho, sty.E);
        const C w = ((neg >> j) & 1u) ? -v[j] : v[j];
        f[j] = ((cross >> j) & 1u) ? w + ad : v[j];
    }
}

template <typename T, typename C>
__device__ __noinline__ void gather_general(const StepArgs<T, C> &a, int x, int y, C f[Q])
{
    gather_body(a, x, y, f, GlobalSrc<T, C>());
}

template <typename T, typename C>
__device__ __forceinline__ void store(const StepArgs<T, C> &a, int x, int y, const C f[Q])
{
    T *p = a.fout + (long long)y * a.pitch + x;
#pragma unroll
    for (int j = 0; j < Q; ++j) *chk(a, a.fout, p + (long long)j * a.plane) = T(f[j]);
}

// ------------------------------------------------------------- the step

// One thread: R consecutive rows y0..y0+R-1 of column x.  A warp whose rows
// are all at least two rows away from the bottom and top edges loads its 13
// pulls with the source column clamped into the lattice (uniform code, always
// in bounds); lanes within two columns of the left or right edge then replace
// the links that cross that edge (periodic wrap, or the wall rule with the
// correction evaluated from the wall state at the node's row).  Warps on the bottom or top rows resolve every node
// with gather_general through `slot`, this thread's shared-memory row.
template <typename T, typename C, bool Force, int R>
__device__ __forceinline__ void process_column(const StepArgs<T, C> &a, int x, int y0, C *slot)
{
    const int nx = a.nx, ny = a.ny;
    const bool yin = y0 >= 2 && y0 + R <= ny - 2;
    if (__all_sync(0xffffffffu, yin)) {
        // Lanes next to an x wall that needs data need its state at their
        // rows.  At a zero-flux temperature wall it takes three populations:
        // their loads are issued here and summed after the pulls, so they
        // share the pulls' round trip.  Other walls evaluate it out of line
        // first (nothing else is live yet).
        const bool xedge = x < nx && (x < 2 || x >= nx - 2) && !a.per_x;
        const int side = x < 2 ? WEST : EAST;
        const bool wdata = xedge && a.wall[side].needs_data;
        const bool zf = a.wall[side].kind == WALL_MIXED && a.wall[side].mass_flux;
        WallState<C> st[R];
        C zo[R][3];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            st[r] = {C(0), C(0)};
            zo[r][0] = zo[r][1] = zo[r][2] = C(0);
            if (wdata) {
                if (zf) {
                    int x0, y0w, x1, y1w;
                    wall_nodes(a, side, y0 + r, x0, y0w, x1, y1w);
                    zo[r][0] = ld(a, out_unit(side), x0, y0w);
                    zo[r][1] = ld(a, out_two(side), x0, y0w);
                    zo[r][2] = ld(a, out_two(side), x1, y1w);
                } else {
                    st[r] = wall_state(a, side, y0 + r);
                }
            }
        }
        C f[R][Q];
        const T *base = a.fin + (long long)y0 * a.pitch;
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const int xs = min(max(x - cvx(j), 0), nx - 1);
                f[r][j] = C(LBM13_LDG(chk(a, a.fin, base + (long long)j * a.plane + (long long)(r - cvy(j)) * a.pitch + xs)));
            }
        }
        if (x >= nx) return;
        if (x < 2 || x >= nx - 2) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (wdata && zf) st[r] = zero_flux_state(a.wall[side], zo[r][0] + zo[r][1] + zo[r][2]);
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    if (cvx(j) == 0) continue;
                    const int sx = x - cvx(j);
                    if (sx >= 0 && sx < nx) continue;
                    if (a.per_x)
                        f[r][j] = ld(a, j, sx < 0 ? sx + nx : sx - nx, y0 + r - cvy(j));
                    else
                        f[r][j] = cross_wall(a, side, j, x, y0 + r, st[r]);
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
            // halo rows of a y-slab are written by the exchange, never stepped
            if ((y < 2 && a.wall[SOUTH].kind == HALO) || (y >= ny - 2 && a.wall[NORTH].kind == HALO)) continue;
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
