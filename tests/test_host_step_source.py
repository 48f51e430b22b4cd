"""The source of the step kernels' per-node code, checked on the host against
the oracle without a GPU.

A step kernel thread runs process_column (csrc/lbm13_stepdev.cuh) on one to
four rows of a column: the 13 pulls, the links that cross an x edge
(periodic wrap or the wall rules of cross_wall), or, on the two bottom and
two top rows, every link through gather_body (periodic wrap, bounce-back and
anti-bounce-back walls, the distance-2 links, corners), then collide and store
(csrc/lbm13_math.cuh).  Those functions are plain C++ apart from their CUDA
qualifiers, so this test compiles them with the host compiler (the
qualifiers ignored, a scalar load for the device load, the warp vote taken
over one lane), sets up the lattice constants with the same host code
lbm13_create uses (csrc/lbm13_coef.h), steps whole lattices with them and
compares the populations with the oracle's.

This is a check of the kernel source's logic, not a way to run the library:
the library has no CPU path and refuses to run without CUDA.  The GPU parity
tests check the compiled kernels themselves."""
import ctypes as C
import os
import shutil
import subprocess
import zlib

import numpy as np
import pytest

from oracle import oracle as O
from paper_1401_0188_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1401_0188_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
Q = 13

SRC = r"""
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>
// host stand-ins for the CUDA-only pieces the per-node functions name
#ifndef __noinline__
#define __noinline__ __attribute__((noinline))
#endif
using std::max;
using std::min;
static inline bool __all_sync(unsigned, bool b) { return b; }
#define LBM13_LDG(p) (*(p))
#include "lbm13_coef.h"
#include "lbm13_stepdev.cuh"
using namespace lbm13;

// mode 0: every node through gather_body, collide and store; mode R > 0:
// columns of R rows through process_column, the step kernels' per-thread
// code (the warp vote over one lane: each column picks its own path)
template <typename T, bool Force>
static void sweep(const StepArgs<T, T> &a, int mode)
{
    T slot[Q];
    if (mode == 0) {
        for (int y = 0; y < a.ny; ++y)
            for (int x = 0; x < a.nx; ++x) {
                T f[Q];
                gather_body(a, x, y, f, GlobalSrc<T, T>());
                collide<Force>(f, a.k);
                store(a, x, y, f);
            }
        return;
    }
    for (int y0 = 0; y0 < a.ny; y0 += mode)
        for (int x = 0; x < a.nx; ++x) {
            if (mode == 1) process_column<T, T, Force, 1>(a, x, y0, slot);
            else process_column<T, T, Force, 2>(a, x, y0, slot);
        }
}

template <typename T>
static void run(const lbm13_params &p, const double *D, const lbm13_boundary &b, int nx, int ny, int steps,
                int mode, const double *f0, double *f1)
{
    Coef<double> kd;
    collision_coef(p, D, b, kd);
    Coef<T> k;
    collision_coef(p, D, b, k);
    WallArgs<T> w[4];
    wall_coef(p, D, b, kd, w);
    const long long pitch = (nx + 31) / 32 * 32, plane = (long long)ny * pitch;
    std::vector<T> buf[2] = {std::vector<T>(Q * plane, T(0)), std::vector<T>(Q * plane, T(0))};
    const double *wr = D + 22;  // rest populations
    const long long n = (long long)nx * ny;
    for (int j = 0; j < Q; ++j)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) buf[0][j * plane + y * pitch + x] = T(f0[j * n + y * nx + x] - wr[j]);
    const bool force = b.gx != 0.0 || b.gy != 0.0 || b.heat != 0.0;
    int cur = 0;
    for (int s = 0; s < steps; ++s) {
        StepArgs<T, T> a;
        std::memset(&a, 0, sizeof a);
        a.fin = buf[cur].data();
        a.fout = buf[cur ^ 1].data();
        a.nx = nx;
        a.ny = ny;
        a.per_x = b.west.kind == PERIODIC;
        a.per_y = b.south.kind == PERIODIC;
        a.pitch = pitch;
        a.plane = plane;
        a.k = k;
        for (int i = 0; i < 4; ++i) a.wall[i] = w[i];
        if (force) sweep<T, true>(a, mode);
        else sweep<T, false>(a, mode);
        cur ^= 1;
    }
    for (int j = 0; j < Q; ++j)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) f1[j * n + y * nx + x] = double(buf[cur][j * plane + y * pitch + x]) + wr[j];
}

extern "C" void host_steps(const lbm13_params *p, const double *D, const lbm13_boundary *b, int nx, int ny,
                           int fp32, int steps, int mode, const double *f0, double *f1)
{
    if (fp32) run<float>(*p, D, *b, nx, ny, steps, mode, f0, f1);
    else run<double>(*p, D, *b, nx, ny, steps, mode, f0, f1);
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("hoststep")
    src, so = d / "host_step.cpp", d / "host_step.so"
    src.write_text(SRC)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-w", "-I", CSRC, "-I", CUDA_INC,
                           str(src), "-o", str(so)])
    L = C.CDLL(str(so))
    dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
    L.host_steps.argtypes = [C.c_void_p, dp, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, dp, dp]
    return L


def _cases(T0):
    hot, cold = T0 + 0.005, T0 - 0.005
    B, M = W.WALL_BB, W.WALL_MIXED
    return {
        "cavity": (30, 26, W.cavity(T0, 0.01, 2e-4)),
        "lid_driven": (20, 18, W.boundary(west=W.wall(B), east=W.wall(B), south=W.wall(B), north=W.wall(B, 0.03))),
        "all_mixed_moving": (23, 19, W.boundary(west=W.wall(M, -0.01, hot), east=W.wall(M, 0.015, cold),
                                                south=W.wall(M, 0.02, T0), north=W.wall(M, -0.01, hot),
                                                gx=1e-5, gy=-2e-5, rho_ref=1.0)),
        "all_mixed_zero_flux": (23, 19, W.boundary(west=W.wall(M, -0.01, hot), east=W.wall(M, 0.015, cold),
                                                   south=W.wall(M, 0.02, T0), north=W.wall(M, -0.01, hot),
                                                   gx=1e-5, gy=-2e-5, rho_ref=1.0, wall_density=1)),
        "x_walls_periodic_y": (21, 17, W.boundary(west=W.wall(M, 0.01, hot), east=W.wall(B, -0.02), gy=1e-5)),
        "heated_slab": (24, 8, W.heated_slab(T0, 1e-5, 0.02)),
        "periodic_forced_heated": (17, 13, W.boundary(gx=2e-5, gy=-1e-5, heat=2e-6)),
        "tiny_walls": (4, 4, W.boundary(west=W.wall(M, 0.0, hot), east=W.wall(M, 0.0, cold), south=W.wall(B, 0.02),
                                        north=W.wall(M, 0.0, T0))),
        "tiny_periodic": (2, 3, W.boundary()),
    }


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("case", list(_cases(0.576)))
def test_kernel_step_source_matches_the_oracle(lib, case, fp32, mode):
    """100 steps from perturbed populations, every node through the edge
    gather (mode 0) or through the per-thread column code with one or two
    rows per thread (modes 1, 2): FP64 within 1e-12 of the oracle (round-off
    of the different operation order), FP32 deviation storage within 1e-7."""
    from paper_1401_0188_gb300 import build, lbm13
    build.build()
    p = O.pstar(0.05, 0.71)
    st, D = lbm13.lbm13_derive(p)
    assert st == 0
    T0 = (p["E0"] + 28.0) / 26.0
    nx, ny, bnd = _cases(T0)[case]
    o = O.Lattice(nx, ny, p, bnd)
    f0 = W.perturbed_populations(o.constants()["w"], nx, ny, 1e-3, seed=zlib.crc32(case.encode()))
    o.set_raw(f0)
    steps = 100
    f1 = np.zeros_like(f0)
    Pp, Bb = lbm13.make_params(p), lbm13.make_boundary(bnd)
    lib.host_steps(C.addressof(Pp), np.ascontiguousarray(D), C.addressof(Bb), nx, ny, fp32, steps, mode,
                   np.ascontiguousarray(f0), f1)
    o.step(steps)
    d = np.abs(f1 - o.get_raw()).max()
    assert d < (1e-7 if fp32 else 1e-12), d
    assert np.abs(f1 - f0).max() > 1e-5  # the state moved
