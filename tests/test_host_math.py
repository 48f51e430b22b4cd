"""The kernels' per-node code on the host, without a GPU: the velocity and
wall-link tables, the factorised moment transforms and the collision of
csrc/lbm13_math.cuh (host and device functions, which the library's host code
also uses), with the collision constants lbm13_create computes
(csrc/lbm13_coef.h), are compiled with the host compiler and checked against
the paper's velocity set (tests/golden/velocities.txt, Sec. 1 and Sec. 2), the
oracle's dense moment matrix M of Eq. (d2q13-polynomes) and its inverse
M^T D^-1, and the oracle's collision.

This checks the source of the arithmetic the step kernels run (pair sums and
differences instead of 2 x 169 products); the GPU parity tests check the
compiled kernels end to end."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1401_0188_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
Q = 13
FIELDS = ("rho", "E", "eps", "vpi", "jx", "jy", "qx", "qy", "rx", "ry", "XX", "XY", "XXe")

SRC = r"""
#include "lbm13_internal.h"
#include "lbm13_coef.h"
using namespace lbm13;
// one collision of the step kernels' code, on deviations df = f - w
template <typename C>
void collide_dev(const lbm13_params *p, const double *D, const lbm13_boundary *b, const double *df, double *out)
{
    Coef<C> k;
    collision_coef(*p, D, *b, k);
    C f[Q];
    for (int j = 0; j < Q; ++j) f[j] = C(df[j]);
    if (b->gx != 0.0 || b->gy != 0.0 || b->heat != 0.0) collide<true>(f, k);
    else collide<false>(f, k);
    for (int j = 0; j < Q; ++j) out[j] = double(f[j]);
}
extern "C" void host_wall_polys(const lbm13_params *p, const double *D, const lbm13_boundary *b, double *poly)
{
    Coef<double> kd;
    collision_coef(*p, D, *b, kd);
    WallArgs<double> w[4];
    wall_coef(*p, D, *b, kd, w);
    for (int s = 0; s < 4; ++s)
        for (int i = 0; i < 4; ++i)
            for (int m = 0; m < 5; ++m) poly[(s * 4 + i) * 5 + m] = w[s].poly[i][m];
}
extern "C" void host_collide(const lbm13_params *p, const double *D, const lbm13_boundary *b, const double *df,
                             int fp32, double *out)
{
    if (fp32) collide_dev<float>(p, D, b, df, out);
    else collide_dev<double>(p, D, b, df, out);
}
extern "C" void wall_tables(int *link, int *slot)
{
    for (int s = 0; s < 4; ++s) {
        for (int i = 0; i < 4; ++i) link[4 * s + i] = wall_link(s, i);
        for (int j = 0; j < Q; ++j) slot[Q * s + j] = wall_slot(s, j);
    }
}
extern "C" void tables(int *vx, int *vy, int *opp)
{
    for (int j = 0; j < Q; ++j) { vx[j] = cvx(j); vy[j] = cvy(j); opp[j] = copp(j); }
}
extern "C" void forward_moments(const double *f, double *m)
{
    Mom<double> r;
    forward(f, r);
    const double v[Q] = {r.rho, r.E, r.eps, r.vpi, r.jx, r.jy, r.qx, r.qy, r.rx, r.ry, r.XX, r.XY, r.XXe};
    for (int k = 0; k < Q; ++k) m[k] = v[k];
}
extern "C" void wall_moments(const double *f, double *out)
{
    out[0] = mass_dev(f);
    out[1] = energy_dev(f);
}
extern "C" void inverse_populations(const double *d, int with_rho, double *f)
{
    const Mom<double> r = {d[0], d[1], d[2], d[3], d[4], d[5], d[6], d[7], d[8], d[9], d[10], d[11], d[12]};
    for (int j = 0; j < Q; ++j) f[j] = 0.0;
    if (with_rho) inverse_add<true>(r, f);
    else inverse_add<false>(r, f);
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("hostmath")
    src, so = d / "host_math.cpp", d / "host_math.so"
    src.write_text(SRC)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-w", "-I", CSRC, "-I", CUDA_INC,
                           str(src), "-o", str(so)])
    L = C.CDLL(str(so))
    ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
    dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
    L.tables.argtypes = [ip, ip, ip]
    L.forward_moments.argtypes = [dp, dp]
    L.inverse_populations.argtypes = [dp, C.c_int, dp]
    L.wall_moments.argtypes = [dp, dp]
    L.wall_tables.argtypes = [ip, ip]
    L.host_collide.argtypes = [C.c_void_p, dp, C.c_void_p, dp, C.c_int, dp]
    L.host_wall_polys.argtypes = [C.c_void_p, dp, C.c_void_p, dp]
    return L


def _golden_velocities():
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "velocities.txt"))
            if l.strip() and not l.startswith("#")]
    return np.array([[int(r[1]), int(r[2])] for r in rows])


def test_velocity_tables_follow_the_paper(lib):
    vx, vy, opp = (np.zeros(Q, dtype=np.int32) for _ in range(3))
    lib.tables(vx, vy, opp)
    v = _golden_velocities()
    assert np.array_equal(vx, v[:, 0]) and np.array_equal(vy, v[:, 1])
    assert np.array_equal(vx[opp], -vx) and np.array_equal(vy[opp], -vy)


def test_factorised_forward_transform_is_M(lib):
    M, _, _ = O.basis()
    f = np.random.default_rng(11).standard_normal((64, Q))
    for row in f:
        m = np.zeros(Q)
        lib.forward_moments(np.ascontiguousarray(row), m)
        assert np.allclose(m, M @ row, rtol=0, atol=1e-12), dict(zip(FIELDS, m - M @ row))


@pytest.mark.parametrize("with_rho", [1, 0])
def test_factorised_inverse_is_M_transposed_over_D(lib, with_rho):
    """inverse_add adds sum_k M_kj d_k for increments d_k already divided by
    D_k, so forward(inverse(m / D)) returns m; without the rho row the density
    increment is left out (the collision never changes rho)."""
    M, D, Minv = O.basis()
    m = np.random.default_rng(12).standard_normal((64, Q))
    for row in m:
        f = np.zeros(Q)
        lib.inverse_populations(np.ascontiguousarray(row / D), with_rho, f)
        want = M.T @ (row / D) if with_rho else M.T @ (row / D) - M[0] * row[0] / D[0]
        assert np.allclose(f, want, rtol=0, atol=1e-12)
        if with_rho:
            assert np.allclose(f, Minv @ row, rtol=0, atol=1e-12)


def test_wall_state_moments_are_the_rho_and_E_rows(lib):
    """The two moments a wall state is extrapolated from (Sec. 7) are the rho
    and E rows of M."""
    M, _, _ = O.basis()
    for row in np.random.default_rng(13).standard_normal((32, Q)):
        out = np.zeros(2)
        lib.wall_moments(np.ascontiguousarray(row), out)
        assert np.allclose(out, M[:2] @ row, rtol=0, atol=1e-12)


def test_each_side_lists_the_links_that_enter_across_it(lib):
    """A wall's corrections are kept per entering link (Sec. 7): west, east,
    south, north each list exactly the four velocities that point into the
    lattice across that side, and the slot lookup inverts the list."""
    link, slot = np.zeros(16, dtype=np.int32), np.zeros(4 * Q, dtype=np.int32)
    lib.wall_tables(link, slot)
    v = _golden_velocities()
    inward = [v[:, 0] > 0, v[:, 0] < 0, v[:, 1] > 0, v[:, 1] < 0]  # west, east, south, north
    for side in range(4):
        assert sorted(link[4 * side:4 * side + 4]) == sorted(np.flatnonzero(inward[side]))
        for j in range(Q):
            want = list(link[4 * side:4 * side + 4]).index(j) if inward[side][j] else -1
            assert slot[Q * side + j] == want


@pytest.mark.parametrize("case", ["plain", "force", "buoyancy_and_source"])
@pytest.mark.parametrize("fp32", [0, 1])
def test_kernel_collision_equals_the_oracle(lib, case, fp32):
    """One collision (Sec. 2: moments, equilibria at j + F/2 and E + 13 q,
    relaxation, force and source, back to populations) by the kernels' code,
    with the constants lbm13_create computes (lbm13_derive, then the host's
    collision constants), against the oracle's dense 13 x 13 collision, on
    populations around equilibria of random (rho, u, T): FP64 to round-off
    (measured 2e-16), FP32 deviation storage within 1e-8 (measured 1.6e-9)."""
    from paper_1401_0188_gb300 import build, lbm13
    build.build()
    p = O.pstar(0.05, 0.71)
    st, D = lbm13.lbm13_derive(p)
    assert st == 0
    bnd = {"plain": O.boundary(), "force": O.boundary(gx=3e-4, gy=-2e-4, rho_ref=0.0),
           "buoyancy_and_source": O.boundary(gy=-1e-3, rho_ref=1.0, heat=2e-5)}[case]
    lat = O.Lattice(2, 2, p, bnd)
    w = lat.constants()["w"]
    T0 = lat.constants()["T0"]
    rng = np.random.default_rng(14)
    P, B = lbm13.make_params(p), lbm13.make_boundary(bnd)
    worst = 0.0
    for _ in range(32):
        one = O.Lattice(2, 2, p, bnd)
        one.set_equilibrium(1 + 0.02 * rng.standard_normal(), 0.03 * rng.standard_normal(),
                            0.03 * rng.standard_normal(), T0 + 0.01 * rng.standard_normal())
        f = one.get_raw()[:, 0, 0] * (1 + 1e-2 * rng.standard_normal(Q))
        out = np.zeros(Q)
        lib.host_collide(C.addressof(P), np.ascontiguousarray(D), C.addressof(B), np.ascontiguousarray(f - w), fp32, out)
        worst = max(worst, np.abs(out + w - lat.collide_node(f)).max())
    assert worst < (1e-8 if fp32 else 1e-14), worst


def test_wall_corrections_are_the_oracle_equilibrium_parts(lib):
    """Sec. 7's walls, as the kernels apply them: each entering link gains a
    correction that is a quadratic polynomial in the wall state's deviations
    (drho_w, dE_w), fitted on the host (csrc/lbm13_coef.h).  At any wall state
    it must equal the oracle's equilibrium at that state: the odd part
    f_eq,j - f_eq,-j on bounce-back links (R14) and the even part
    f_eq,j + f_eq,-j on the normal links of a temperature wall (R11, anti-
    bounce-back), as deviations from the rest populations, with the wall's
    own velocity (R12's density and the temperature wall's energy enter only
    through that state)."""
    from paper_1401_0188_gb300 import build, lbm13
    build.build()
    p = O.pstar(0.05, 0.71)
    st, D = lbm13.lbm13_derive(p)
    assert st == 0
    T0 = (p["E0"] + 28.0) / 26.0
    B, M = O.WALL_BB, O.WALL_MIXED
    bnd = O.boundary(west=O.wall(M, 0.02, T0 + 0.01), east=O.wall(B, -0.03), south=O.wall(M, -0.01, T0 - 0.01),
                     north=O.wall(B, 0.025))
    poly = np.zeros(80)
    Pp, Bb = lbm13.make_params(p), lbm13.make_boundary(bnd)
    lib.host_wall_polys(C.addressof(Pp), np.ascontiguousarray(D), C.addressof(Bb), poly)
    poly = poly.reshape(4, 4, 5)
    link, slot = np.zeros(16, dtype=np.int32), np.zeros(4 * Q, dtype=np.int32)
    lib.wall_tables(link, slot)
    vx, vy = O.velocities()
    opp = [int(np.flatnonzero((vx == -vx[j]) & (vy == -vy[j]))[0]) for j in range(Q)]
    eq = O.Lattice(2, 2, p)
    w = eq.constants()["w"]
    rng = np.random.default_rng(15)
    sides = [bnd["west"], bnd["east"], bnd["south"], bnd["north"]]
    for s, side in enumerate(sides):
        u = (0.0, side["u_t"]) if s < 2 else (side["u_t"], 0.0)
        for _ in range(6):
            rho_w = 1 + 0.05 * rng.standard_normal()
            T_w = T0 + 0.02 * rng.standard_normal()
            eq.set_equilibrium(rho_w, u[0], u[1], T_w)
            feq = eq.get_raw()[:, 0, 0] - w
            dE = rho_w * (26 * T_w - 28) + 13 * rho_w * (u[0] ** 2 + u[1] ** 2) - p["E0"]
            for i in range(4):
                j = link[4 * s + i]
                normal = vy[j] == 0 if s < 2 else vx[j] == 0
                want = feq[j] + feq[opp[j]] if (side["kind"] == M and normal) else feq[j] - feq[opp[j]]
                a = poly[s, i]
                x, y = rho_w - 1, dE
                got = a[0] + x * (a[1] + x * a[3] + y * a[4]) + y * a[2]
                assert got == pytest.approx(want, abs=1e-14), (s, j)
