"""ctypes wrapper of the FP64 CPU oracle (lbm13_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check of the
package entry module and by bench.py's CPU-baseline leg.  It shares no code
with the CUDA path and never imports the product package.

The solver follows the paper's Sec. 2 (stencil, moment basis, equilibria,
derived constants), Sec. 5 and Sec. 8 (forcing), Sec. 7 (mixed bounce-back /
anti-bounce-back walls) and Sec. 10 (Nusselt number, centro-asymmetry); the
readings it takes where the paper is silent are listed in the C file's header.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

Q = 13
PARAM_FIELDS = ("E0", "c1", "k2", "c_epsE", "c_vpi_rho", "c_vpi_E", "Pr", "nu",
                "s_eps", "s_vpi", "s_r", "s_XXe")
PERIODIC, WALL_BB, WALL_MIXED = 0, 1, 2


class _Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in PARAM_FIELDS]


class _Wall(C.Structure):
    _fields_ = [("kind", C.c_int), ("u_t", C.c_double), ("T", C.c_double)]


class _Boundary(C.Structure):
    _fields_ = [("west", _Wall), ("east", _Wall), ("south", _Wall), ("north", _Wall),
                ("gx", C.c_double), ("gy", C.c_double), ("rho_ref", C.c_double), ("wall_density", C.c_int),
                ("heat", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        # LBM13_ORACLE_LIB: an alternative build of lbm13_oracle.c (the
        # mutation tests load copies with a planted mistake)
        path = os.environ.get("LBM13_ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, C.c_int, C.POINTER(_Params), C.POINTER(_Boundary), C.c_int]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_constants.argtypes = [C.c_void_p, dp]
        L.orc_set_equilibrium.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.orc_set_raw.argtypes = [C.c_void_p, dp]
        L.orc_get_raw.argtypes = [C.c_void_p, dp]
        L.orc_step.argtypes = [C.c_void_p, C.c_long]
        L.orc_step.restype = C.c_int
        L.orc_time.argtypes = [C.c_void_p]
        L.orc_time.restype = C.c_long
        L.orc_moments.argtypes = [C.c_void_p, dp]
        L.orc_macro.argtypes = [C.c_void_p, dp]
        L.orc_residual.argtypes = [C.c_void_p, dp]
        L.orc_project.argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
        L.orc_collide_node.argtypes = [C.c_void_p, dp, dp]
        L.orc_basis.argtypes = [dp, dp, dp, C.c_int]
        L.orc_velocities.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.orc_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def basis(printed_q_sign=False):
    """(M, D, Minv) of Eq. (d2q13-polynomes); printed_q_sign uses q = x(3 + r^2)."""
    M = np.zeros((Q, Q))
    D = np.zeros(Q)
    Minv = np.zeros((Q, Q))
    lib().orc_basis(_dp(M), _dp(D), _dp(Minv), 1 if printed_q_sign else 0)
    return M, D, Minv


def velocities():
    vx = (C.c_int * Q)()
    vy = (C.c_int * Q)()
    lib().orc_velocities(vx, vy)
    return np.array(list(vx)), np.array(list(vy))


def max_threads():
    return lib().orc_max_threads()


def wall(kind=PERIODIC, u_t=0.0, T=0.0):
    return {"kind": kind, "u_t": u_t, "T": T}


def boundary(west=None, east=None, south=None, north=None, gx=0.0, gy=0.0, rho_ref=0.0, wall_density=0, heat=0.0):
    """Sides, body force F = (rho - rho_ref) g, wall density rule (R12 / R12')
    and the energy source q per node and step (R18, Sec. 9)."""
    w = lambda d: d if d is not None else wall()
    return {"west": w(west), "east": w(east), "south": w(south), "north": w(north),
            "gx": gx, "gy": gy, "rho_ref": rho_ref, "wall_density": wall_density, "heat": heat}


def _mk_boundary(b):
    mk = lambda d: _Wall(int(d["kind"]), float(d.get("u_t", 0.0)), float(d.get("T", 0.0)))
    return _Boundary(mk(b["west"]), mk(b["east"]), mk(b["south"]), mk(b["north"]),
                     float(b.get("gx", 0.0)), float(b.get("gy", 0.0)), float(b.get("rho_ref", 0.0)),
                     int(b.get("wall_density", 0)), float(b.get("heat", 0.0)))


class Lattice:
    """One lattice of the oracle; state = post-collision f*(t), [13][ny][nx]."""

    def __init__(self, nx, ny, params, bnd=None, nthreads=1):
        self.nx, self.ny = int(nx), int(ny)
        self.params = dict(params)
        self.bnd = bnd if bnd is not None else boundary()
        p = _Params(*[float(params[n]) for n in PARAM_FIELDS])
        b = _mk_boundary(self.bnd)
        self._h = lib().orc_create(self.nx, self.ny, C.byref(p), C.byref(b), int(nthreads))
        if not self._h:
            raise ValueError("oracle rejected the lattice (sizes, boundary pairing or rates)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def constants(self):
        out = np.zeros(64)
        lib().orc_constants(self._h, _dp(out))
        names = ("A", "B", "h1", "k1", "h2", "c2", "c_erho", "sigma_XX", "sigma_q")
        d = {n: out[i] for i, n in enumerate(names)}
        d["s"] = out[9:22].copy()
        d["w"] = out[22:35].copy()
        d["T0"] = out[35]
        return d

    def set_equilibrium(self, rho, ux, uy, T):
        shape = (self.ny, self.nx)
        arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shape))
                for a in (rho, ux, uy, T)]
        lib().orc_set_equilibrium(self._h, *[_dp(a) for a in arrs])

    def set_raw(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(Q, self.ny, self.nx)
        lib().orc_set_raw(self._h, _dp(f))

    def get_raw(self):
        f = np.zeros((Q, self.ny, self.nx))
        lib().orc_get_raw(self._h, _dp(f))
        return f

    def step(self, n=1):
        if lib().orc_step(self._h, int(n)) != 0:
            raise RuntimeError("oracle streaming left a slot unwritten")

    @property
    def t(self):
        return lib().orc_time(self._h)

    def moments(self):
        out = np.zeros((Q, self.ny, self.nx))
        lib().orc_moments(self._h, _dp(out))
        return out

    def macro(self):
        """(rho, ux, uy, T), each [ny][nx]."""
        out = np.zeros((4, self.ny, self.nx))
        lib().orc_macro(self._h, _dp(out))
        return out

    def residual(self):
        out = np.zeros(16)
        lib().orc_residual(self._h, _dp(out))
        return out

    def project(self, kx, ky=0):
        """Sec. 6 aggregates: [field][harmonic][cos, sin] for the fields
        (rho - 1, ux, uy, T - T0, E - E0, p - T0), harmonics k and 2k."""
        out = np.zeros(24)
        lib().orc_project(self._h, int(kx), int(ky), _dp(out))
        return out.reshape(6, 2, 2)

    def collide_node(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        fs = np.zeros(Q)
        lib().orc_collide_node(self._h, _dp(f), _dp(fs))
        return fs


def pstar(nu=0.05, Pr=0.71):
    """A linearly stable choice of the free parameters of Sec. 2.

    The paper prints no values (it picks them by scanning the dispersion
    relation).  This set fixes the rest populations at weights
    (0.53, 0.049, 0.0175, 0.051) (rest, unit axes, diagonals, distance-2 axes),
    which fixes E0, eps0 and varpi0 as moments of those weights; c1 = -1,
    k2 = 0.4, c_varpiE = 0.3, c_varpirho = varpi0 - c_varpiE E0, and c_epsE is
    solved so that the equilibrium eps at rest stays eps0 once c_erho follows
    Pr through Eq. (d2q13-sigma-qx).  Rates: s_eps 0.6, s_varpi 1.25, s_r 1.2,
    s_XXe 1.0.
    """
    M, _, _ = basis()
    w = np.array([0.53] + [0.049] * 4 + [0.0175] * 4 + [0.051] * 4)
    m0 = M @ w
    E0, eps0, vpi0 = m0[1], m0[2], m0[3]
    c1, k2, cvE = -1.0, 0.4, 0.3
    cvr = vpi0 - cvE * E0
    A = 13 * c1 + 95 + 2 * E0
    # eps_eq(rest) = c_erho + c_epsE E0 with c_erho from Eq. (d2q13-sigma-qx):
    # 140 + 28 c + A (B0 - 11492 c) / (22984 Pr) + c E0 = eps0, linear in c.
    B0 = 114404 + 51051 * c1 + 7854 * E0
    a0 = 140 + A * B0 / (22984 * Pr) - eps0
    a1 = 28 - A * 11492 / (22984 * Pr) + E0
    ceE = -a0 / a1
    return {"E0": E0, "c1": c1, "k2": k2, "c_epsE": ceE, "c_vpi_rho": cvr, "c_vpi_E": cvE,
            "Pr": Pr, "nu": nu, "s_eps": 0.6, "s_vpi": 1.25, "s_r": 1.2, "s_XXe": 1.0}
