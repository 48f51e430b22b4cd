// lbm13_internal.h -- structures passed from the C-ABI host code to the kernel
// launchers.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "lbm13_math.cuh"

namespace lbm13 {

enum Side { WEST = 0, EAST = 1, SOUTH = 2, NORTH = 3 };
enum WallKind { PERIODIC = 0, WALL_BB = 1, WALL_MIXED = 2 };

// One side of the lattice as the kernels see it.
template <typename C>
struct WallArgs {
    int kind;        // WallKind
    int needs_data;  // 1 when the wall's equilibrium enters (mixed wall, or moving wall)
    C ux, uy;        // wall velocity (tangential only)
    C base;          // 26 T_w - 28      (rho_w (26 T_w - 28) is E_w without kinetic part)
    C eT;            // 26 T_w - 28 - E0 = 26 (T_w - T0)
};

template <typename T, typename C>
struct StepArgs {
    const T *__restrict__ fin;
    T *__restrict__ fout;
    int nx, ny;
    int per_x, per_y;
    long long pitch;  // elements per row
    long long plane;  // elements per population plane (ny * pitch)
    Coef<C> k;
    WallArgs<C> wall[4];
};

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
};

// Launchers (return the cudaError_t of the launch).
template <typename T, typename C>
cudaError_t launch_step(const StepArgs<T, C> &a, bool force, cudaStream_t s);

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

int reduce_blocks(int nx, int ny);

template <typename T>
cudaError_t launch_reduce(const ReadArgs<T> &a, const ReduceBufs &b, const ReduceConf &c, double *out_dev,
                          cudaStream_t s);

// Read-only view of a lattice handle (population buffer, layout, rest
// constants, stream), for entry points that live outside lbm13_api.cu.
struct StateView {
    const void *f;
    int nx, ny, precision, device;
    long long pitch, plane;
    double E0, gx, gy, rho_ref;
    cudaStream_t stream;
};

} // namespace lbm13

struct lbm13_lattice;
// Fills *v from a handle; returns false for a NULL handle.
bool lbm13_state_view(const lbm13_lattice *h, lbm13::StateView *v);
