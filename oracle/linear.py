"""Linearised (von Neumann) analysis of the oracle's time step.

TEST INFRASTRUCTURE ONLY.  The paper chooses its free parameters by computing
the roots of the dispersion equation for wave vectors of magnitude 0 to 2 pi in
several directions (end of Sec. 2) and states what the four hydrodynamic modes
must do: advect with the background velocity, decay isotropically, carry the
Prandtl number (Eqs. (d2q13-diffusion), (d2q13-sigma-qx)) and, to first order,
obey the 3x3 system of Eq. (d2q13-equiv-edp-ordre-1).

The collision Jacobian is taken from the oracle's own C collision by central
finite differences about a uniform state, so these checks pin the compiled
oracle, not a retyped formula.  Streaming of a Fourier mode exp(i k.x) over
link j multiplies population j by exp(-i k.v_j) (pull form), so one time step
of the linearised scheme is G(k) = diag(exp(-i k.v_j)) J.
"""
import numpy as np

from . import oracle as O


def equilibrium_f(lat, rho, ux, uy, T):
    """f_eq of one node, through the oracle's own initialiser."""
    one = O.Lattice(2, 2, lat.params)
    one.set_equilibrium(rho, ux, uy, T)
    return one.get_raw()[:, 0, 0].copy()


def collision_jacobian(lat, rho=1.0, ux=0.0, uy=0.0, T=None, h=1e-6):
    """d f*/d f at the equilibrium of (rho, u, T), central differences."""
    if T is None:
        T = lat.constants()["T0"]
    f0 = equilibrium_f(lat, rho, ux, uy, T)
    J = np.zeros((O.Q, O.Q))
    for i in range(O.Q):
        e = np.zeros(O.Q)
        e[i] = h
        J[:, i] = (lat.collide_node(f0 + e) - lat.collide_node(f0 - e)) / (2 * h)
    return J, f0


def amplification(J, k):
    vx, vy = O.velocities()
    ph = np.exp(-1j * (vx * k[0] + vy * k[1]))
    return ph[:, None] * J


def hydrodynamic_modes(J, k, n=4):
    """The n eigenvalues of G(k) with the largest modulus (the slow, hydrodynamic
    ones at small |k|), with their eigenvectors, sorted by decreasing |z|."""
    z, V = np.linalg.eig(amplification(J, k))
    order = np.argsort(-np.abs(z))[:n]
    return z[order], V[:, order]


def max_modulus(J, n=33):
    """max |z| of G(k) over an n x n grid of k in [-pi, pi]^2."""
    ks = np.linspace(-np.pi, np.pi, n)
    best = 0.0
    for kx in ks:
        for ky in ks:
            best = max(best, np.abs(np.linalg.eigvals(amplification(J, (kx, ky)))).max())
    return best
