"""Seeded synthetic inputs shaped like the paper's test cases.

This module holds no arithmetic of the scheme: it draws fields and noise and
describes boundary set-ups with plain numbers, so the same inputs feed the
CUDA path and, in the tests, the CPU oracle.
"""
import numpy as np

PERIODIC, WALL_BB, WALL_MIXED = 0, 1, 2

SEED_PARITY = 20260101


def shear_wave(nx, ny, amplitude=0.01):
    """Transverse shear wave u_x = A sin(2 pi y / ny), u_y = 0 (Sec. 6 family)."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    return amplitude * np.sin(2.0 * np.pi * y / ny), np.zeros((ny, nx))


def noise(shape, seed=SEED_PARITY):
    """Standard normal draws from numpy's PCG64 with the given seed."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(shape)


def perturbed_populations(base, nx, ny, rel=1e-4, seed=SEED_PARITY):
    """base[j] * (1 + rel * N(0,1)) per population and node, shape (13, ny, nx).

    `base` is any 13-vector of positive populations (e.g. the rest weights)."""
    z = noise((13, ny, nx), seed)
    return np.asarray(base, dtype=np.float64)[:, None, None] * (1.0 + rel * z)


def random_fields(nx, ny, T0, seed, du=0.02, drho=0.02, dT=0.02):
    """Smoothless random (rho, ux, uy, T) around (1, 0, 0, T0)."""
    g = np.random.Generator(np.random.PCG64(seed))
    rho = 1.0 + drho * g.standard_normal((ny, nx))
    ux = du * g.standard_normal((ny, nx))
    uy = du * g.standard_normal((ny, nx))
    T = T0 + dT * g.standard_normal((ny, nx))
    return rho, ux, uy, T


def wall(kind=PERIODIC, u_t=0.0, T=0.0):
    return {"kind": kind, "u_t": u_t, "T": T}


def boundary(west=None, east=None, south=None, north=None, gx=0.0, gy=0.0, rho_ref=0.0, wall_density=0, heat=0.0):
    """wall_density: 0 extrapolated density at temperature walls, 1 zero net
    mass flux; heat: energy source per node and step (Sec. 9)."""
    w = lambda d: d if d is not None else wall()
    return {"west": w(west), "east": w(east), "south": w(south), "north": w(north),
            "gx": gx, "gy": gy, "rho_ref": rho_ref, "wall_density": wall_density, "heat": heat}


def cavity(T0, dT, g, rho_ref=1.0, wall_density=0):
    """Differentially heated cavity (Sec. 10): hot west and cold east velocity+
    temperature walls at T0 +- dT/2, adiabatic south and north walls, buoyancy
    F = (rho - rho_ref) (0, -g)."""
    return boundary(west=wall(WALL_MIXED, 0.0, T0 + dT / 2), east=wall(WALL_MIXED, 0.0, T0 - dT / 2),
                    south=wall(WALL_BB), north=wall(WALL_BB), gx=0.0, gy=-abs(g), rho_ref=rho_ref,
                    wall_density=wall_density)


def heated_slab(T_w, heat, v_w=0.0, wall_density=1):
    """Adiabatic-wall test (Sec. 9): periodic in y, a velocity+temperature
    wall on the west (temperature T_w, tangential velocity v_w), an adiabatic
    bounce-back wall at rest on the east, and a uniform energy source `heat`
    per node and step.  The steady temperature is the half-parabola with zero
    slope at the adiabatic wall."""
    return boundary(west=wall(WALL_MIXED, v_w, T_w), east=wall(WALL_BB), wall_density=wall_density, heat=heat)


def couette(T0, U, dT, wall_density=0):
    """Couette channel (Sec. 7): periodic in x, lower wall at rest at T0 - dT/2,
    upper wall moving at U at T0 + dT/2, both velocity+temperature walls."""
    return boundary(south=wall(WALL_MIXED, 0.0, T0 - dT / 2), north=wall(WALL_MIXED, U, T0 + dT / 2),
                    wall_density=wall_density)


def poiseuille(g, T0=None, dT=0.0, wall_density=0):
    """Poiseuille channel (Sec. 8): periodic in x, walls at rest, body force
    rho g along x.  With T0 given, the walls are velocity+temperature walls at
    T0 -+ dT/2 (the Couette-type temperature profile of Sec. 8), which also
    carry off the viscous heat; without, adiabatic bounce-back walls."""
    if T0 is None:
        return boundary(south=wall(WALL_BB), north=wall(WALL_BB), gx=g, gy=0.0, rho_ref=0.0)
    return boundary(south=wall(WALL_MIXED, 0.0, T0 - dT / 2), north=wall(WALL_MIXED, 0.0, T0 + dT / 2),
                    gx=g, gy=0.0, rho_ref=0.0, wall_density=wall_density)
