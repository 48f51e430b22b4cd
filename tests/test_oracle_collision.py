"""Pins of the oracle's collision: exact conservation (Sec. 2: the collision
keeps rho, E, j_x, j_y), equilibrium as a fixed point, and the force step
(Sec. 5, Sec. 8) as uniform acceleration without heating."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import linear


def _defs():
    vx, vy = O.velocities()
    e = -28 + 13 * (vx ** 2 + vy ** 2)
    return vx, vy, e


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_collision_conserves_mass_momentum_energy(pstar, seed):
    rng = np.random.default_rng(seed)
    lat = O.Lattice(2, 2, pstar)
    vx, vy, e = _defs()
    f = linear.equilibrium_f(lat, 1.0 + 0.05 * rng.standard_normal(), 0.03 * rng.standard_normal(),
                             0.03 * rng.standard_normal(), 0.576 + 0.02 * rng.standard_normal())
    f = f * (1 + 0.05 * rng.standard_normal(13))
    fs = lat.collide_node(f)
    for w in (np.ones(13), vx, vy, e):
        assert abs(w @ fs - w @ f) < 1e-13 * max(1.0, abs(w @ f))
    assert np.abs(fs - f).max() > 1e-4  # it does relax


@pytest.mark.parametrize("rho,ux,uy,T", [(1.0, 0.0, 0.0, 0.576), (1.05, 0.04, -0.02, 0.6), (0.95, -0.01, 0.05, 0.55)])
def test_equilibrium_is_fixed_point(pstar, rho, ux, uy, T):
    lat = O.Lattice(2, 2, pstar)
    f = linear.equilibrium_f(lat, rho, ux, uy, T)
    assert np.abs(lat.collide_node(f) - f).max() < 1e-14


def test_equilibrium_has_requested_macroscopic_fields(pstar):
    lat = O.Lattice(4, 4, pstar)
    lat.set_equilibrium(1.02, 0.03, -0.01, 0.61)
    rho, ux, uy, T = lat.macro()
    assert np.allclose(rho, 1.02, rtol=0, atol=1e-14)
    assert np.allclose(ux, 0.03, atol=1e-14) and np.allclose(uy, -0.01, atol=1e-14)
    assert np.allclose(T, 0.61, atol=1e-13)


def test_uniform_force_accelerates_without_heating(pstar):
    """A uniform state under a uniform body force F = rho g: u grows by g each
    step, rho and T do not change (the force does work on the mean flow only)."""
    g = (2e-5, -1e-5)
    b = O.boundary(gx=g[0], gy=g[1], rho_ref=0.0)
    lat = O.Lattice(4, 4, pstar, b)
    lat.set_equilibrium(1.0, 0.0, 0.0, 0.576)
    r0, u0, v0, T0 = lat.macro()
    n = 50
    lat.step(n)
    r1, u1, v1, T1 = lat.macro()
    assert np.allclose(r1, r0, atol=1e-14)
    assert np.allclose(u1 - u0, n * g[0], rtol=1e-10, atol=0)
    assert np.allclose(v1 - v0, n * g[1], rtol=1e-10, atol=0)
    assert np.abs(T1 - T0).max() < 1e-12


def test_buoyancy_force_vanishes_at_reference_density(pstar):
    """F = (rho - rho_ref) g (Sec. 5): no force where rho = rho_ref."""
    b = O.boundary(gx=0.0, gy=-1e-4, rho_ref=1.0)
    lat = O.Lattice(4, 4, pstar, b)
    lat.set_equilibrium(1.0, 0.0, 0.0, 0.576)
    f0 = lat.get_raw()
    lat.step(10)
    assert np.abs(lat.get_raw() - f0).max() < 1e-15
