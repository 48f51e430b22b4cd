// lbm13_internal.h -- structures passed from the C-ABI host code to the kernel
// launchers.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "lbm13_math.cuh"
#include "../../include/lbm13.h"

namespace lbm13 {

enum Side { WEST = 0, EAST = 1, SOUTH = 2, NORTH = 3 };
enum WallKind { PERIODIC = 0, WALL_BB = 1, WALL_MIXED = 2, HALO = 3 };

// One side of the lattice as the kernels see it.
template <typename C>
struct WallArgs {
    int kind;        // WallKind
    int needs_data;  // 1 when the wall's equilibrium enters (mixed wall, or moving wall)
    C ux, uy;        // wall velocity (tangential only)
    C base;          // 26 T_w - 28      (rho_w (26 T_w - 28) is E_w without kinetic part)
    C eT;            // 26 T_w - 28 - E0 = 26 (T_w - T0)
    int mass_flux;   // temperature wall whose density makes the net normal mass flux zero
    C wsum;          // w_unit + 2 w_two: rest populations of one unit and one distance-2 axis link
    C zf_ea, zf_eb;  // zero-flux density: even parts of the wall equilibrium at unit density,
                     // unit and distance-2 normal links
    // The correction of each entering link (slot i) as an exact polynomial in
    // the wall state's deviations (drho, dE): poly[i] = (a0, a1, a2, a3, a4) of
    // a0 + a1 drho + a2 dE + a3 drho^2 + a4 drho dE (every equilibrium moment
    // is at most quadratic in rho and E once j = rho u).
    C poly[4][5];
};

// Links that enter the lattice across each side, four per side, in a fixed
// order (the slot of a wall correction):
//   west (1, 5, 8, 9), east (3, 6, 7, 11), south (2, 5, 6, 10), north (4, 7, 8, 12).
LBM13_HD constexpr int wall_link(int side, int i)
{
    return side == 0 ? (i == 0 ? 1 : i == 1 ? 5 : i == 2 ? 8 : 9)
         : side == 1 ? (i == 0 ? 3 : i == 1 ? 6 : i == 2 ? 7 : 11)
         : side == 2 ? (i == 0 ? 2 : i == 1 ? 5 : i == 2 ? 6 : 10)
                     : (i == 0 ? 4 : i == 1 ? 7 : i == 2 ? 8 : 12);
}
LBM13_HD constexpr int wall_slot(int side, int j)
{
    return wall_link(side, 0) == j ? 0 : wall_link(side, 1) == j ? 1 : wall_link(side, 2) == j ? 2
         : wall_link(side, 3) == j ? 3 : -1;
}

template <typename T, typename C>
struct alignas(16) StepArgs {
    const T *__restrict__ fin;
    T *__restrict__ fout;
    int nx, ny;
    int per_x, per_y;
    long long pitch;  // elements per row
    long long plane;  // elements per population plane (ny * pitch)
    Coef<C> k;
    WallArgs<C> wall[4];
#ifdef LBM13_DEBUG
    unsigned long long *bad;  // debug builds: population accesses found outside the lattice
#endif
};

// One lattice of a batched launch: its arguments for both buffer parities
// (a[p].fin is the buffer read when the step's parity is p).
template <typename T, typename C>
struct BatchDesc {
    StepArgs<T, C> a[2];
    int force;    // nonzero when g != 0
    int tiles_x;  // ceil(nx / 32)
};

// Grid barrier words of a persistent launch (device memory, zeroed before use,
// each on its own 128-byte line: kSyncBytes in all) and the bound on every wait.
constexpr int kSyncBytes = 512;
struct GridSync {
    unsigned *count;   // arrivals at the current barrier
    unsigned *gen;     // barrier generation
    unsigned *error;   // nonzero once a wait ran out
    unsigned long long timeout_ns;
};

// Persistent multi-step launch of one lattice (lbm13_multi.cu): the largest
// co-resident grid for its tiles (0 when cooperative launch is unavailable),
// and nsteps steps alternating a0 (current parity) and a1 in one launch.
template <typename T, typename C>
int multi_grid(int nx, int ny, bool force);
template <typename T, typename C>
cudaError_t launch_multi(const StepArgs<T, C> &a0, const StepArgs<T, C> &a1, bool force, int nsteps, int grid,
                         const GridSync &g, cudaStream_t s);
// `rounds` grid barriers over `grid` blocks that wait for expect_blocks
// arrivals (expect_blocks > grid makes every wait run out).
cudaError_t launch_barrier_check(int grid, unsigned expect_blocks, int rounds, const GridSync &g, cudaStream_t s);

// Linear stability (lbm13_linear.cu, host): the largest |z| - 1 over the
// eigenvalues z of the linearised step about (rho, j, E) = (1, (ux, uy),
// E0 + 13 |u|^2) for the n x n wave vectors of [-pi, pi]^2.  D = the derived
// constants of lbm13_derive.  LBM13_EINVAL if an eigenvalue iteration fails.
int linear_growth(const lbm13_params &p, const double *D, double ux, double uy, int n, double *growth);
// The same scan for `count` cases at once on the GPU (stream s; synchronises
// it): parameter set p[c] with derived constants D + c * LBM13_DERIVED_COUNT
// about u = (ux[c], uy[c]); host out growth[count].  LBM13_EINVAL if an
// eigenvalue iteration fails, LBM13_ECUDA on a CUDA error.
int linear_growth_batch(const lbm13_params *p, const double *D, const double *ux, const double *uy, int count, int n,
                        double *growth, cudaStream_t s);

// Rest moments used by the read-outs (double precision).
struct Rest {
    double E0, eps0, vpi0;
};

// Arguments of the read-out and reduction kernels (always double).
template <typename T>
struct ReadArgs {
    const T *__restrict__ f;
    int nx, ny;
    long long pitch, plane;
    Rest rest;
    double gx, gy, rho_ref;
    double heat;  // energy source q: T is read half-way, (p* - q/2)/rho
};

// Streaming multiprocessors of the current device (queried once per device;
// 1 if the query fails, so that callers still size a valid grid).
int device_sm_count();

// Launchers (return the cudaError_t of the launch).
template <typename T, typename C>
cudaError_t launch_step(const StepArgs<T, C> &a, bool force, cudaStream_t s);

// Tile shapes (rows per thread R, warps per block BY) of the batched kernel.
bool batch_shape_supported(int R, int BY);

// Batched step over a work list of (lattice, (tile row << 16) | tile column),
// tiles of 32 columns x groups * BY * R rows.
template <typename T, typename C>
cudaError_t launch_batch(const BatchDesc<T, C> *descs, const int2 *work, int ntiles, int parity, int R, int BY,
                         int groups, int grid, cudaStream_t s);

// y-slab halo rows (HALO sides): pack the two rows next to the halo rows of
// side `side` (SOUTH or NORTH), the four populations that cross it, into
// out[2][4][nx]; unpack writes in[2][4][nx] into the halo rows of `side`.
template <typename T>
cudaError_t launch_halo(T *f, int nx, int ny, long long pitch, long long plane, int side, bool pack, T *buf,
                        cudaStream_t s);

template <typename T>
cudaError_t launch_init(T *f, int nx, int ny, long long pitch, long long plane, const Coef<double> &k,
                        const double *rho, const double *ux, const double *uy, const double *Tf, cudaStream_t s);

template <typename T>
cudaError_t launch_moments(const ReadArgs<T> &a, double *out, unsigned mask, cudaStream_t s);

// Reduction work space (device), laid out by the host.
struct ReduceBufs {
    double *fields;    // [3][ny][nx]: ux, uy, T
    double *snap;      // [3][ny][nx]: snapshot of the previous call
    double *partials;  // [nblocks][kPartials]
    double *stats;     // [16]: means after pass 1, results after pass 2
    int nblocks;
};

struct ReduceConf {
    int have_snap;
    long long K;        // steps since the snapshot
    long long step;
    int nusselt;        // west and east are temperature walls with dT != 0
    double dT, Tref, kappa;  // T_west - T_east, their mean, nu / Pr
    int asym_walls;     // west and east are temperature walls: asymmetry of T about Tasym
    double Tasym;       // (otherwise about the mean T)
};

constexpr int kReduceThreads = 256;
constexpr int kPartials = 16;
constexpr int kProj = 24;  // Fourier projections: 6 fields x 2 harmonics x (cos, sin)

int reduce_blocks(int nx, int ny);

// Fourier projections of one lattice: project_kernel over nblocks blocks into
// partials[nblocks][kProj], then out_dev[kProj] in block order.
template <typename T>
cudaError_t launch_project(const ReadArgs<T> &a, int kx, int ky, double *partials, int nblocks, double *out_dev,
                           cudaStream_t s);

template <typename T>
cudaError_t launch_reduce(const ReadArgs<T> &a, const ReduceBufs &b, const ReduceConf &c, double *out_dev,
                          cudaStream_t s);

// Read-only view of a lattice handle (population buffer, layout, rest
// constants, stream), for entry points that live outside lbm13_api.cu.
struct StateView {
    const void *f;
    int nx, ny, precision, device;
    long long pitch, plane;
    double E0, gx, gy, rho_ref, heat;
    cudaStream_t stream;
};

} // namespace lbm13

struct lbm13_lattice;
// Fills *v from a handle; returns false for a NULL handle.
bool lbm13_state_view(const lbm13_lattice *h, lbm13::StateView *v);
