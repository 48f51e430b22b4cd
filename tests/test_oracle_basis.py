"""Pins of the oracle's stencil, moment basis and equilibria against what the
paper fixes (Sec. 1-2 and the first-order system of Sec. 6)."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_velocities():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "velocities.txt")) if l.strip() and not l.startswith("#")]
    return np.array([[int(r[1]), int(r[2])] for r in rows])


def _golden_first_order():
    d = {}
    for l in open(os.path.join(GOLDEN, "first_order_system.txt")):
        if l.strip() and not l.startswith("#"):
            k, v = l.split()
            d[k] = float(Fraction(v))
    return d


def test_velocity_set_matches_paper():
    v = _golden_velocities()
    vx, vy = O.velocities()
    assert np.array_equal(vx, v[:, 0]) and np.array_equal(vy, v[:, 1])


def test_basis_is_orthogonal_with_integer_entries():
    M, D, Minv = O.basis()
    assert np.array_equal(M, np.round(M))
    G = M @ M.T
    assert np.abs(G - np.diag(np.diag(G))).max() == 0.0
    assert np.allclose(np.diag(G), D)
    assert np.abs(M @ Minv - np.eye(13)).max() < 1e-13


def test_printed_q_sign_is_not_orthogonal():
    """Erratum (reading R1): with q_x = x(3 + x^2 + y^2) as printed, q_x and j_x
    overlap by 84; with -3 they are orthogonal."""
    Mp, _, _ = O.basis(printed_q_sign=True)
    assert Mp[4] @ Mp[6] == 84.0 and Mp[5] @ Mp[7] == 84.0
    M, _, _ = O.basis()
    assert M[4] @ M[6] == 0.0


def test_conserved_rows_are_mass_momentum_energy():
    """rho = sum f, j = sum v f (Eq. d2q9-conserve); E = sum (-28 + 13|v|^2) f,
    the E polynomial of Eq. (d2q13-polynomes)."""
    v = _golden_velocities()
    M, _, _ = O.basis()
    assert np.array_equal(M[0], np.ones(13))
    assert np.array_equal(M[4], v[:, 0]) and np.array_equal(M[5], v[:, 1])
    assert np.array_equal(M[1], -28 + 13 * (v ** 2).sum(1))


@pytest.mark.parametrize("rho,T", [(1.0, 0.576), (1.1, 0.5), (0.9, 0.7)])
def test_rest_momentum_flux_matches_first_order_system(pstar, rho, T):
    """At rest, sum v_x^2 f_eq = (14/13) rho + E/26 (Eq. d2q13-equiv-edp-ordre-1)."""
    from oracle import linear
    g = _golden_first_order()
    lat = O.Lattice(2, 2, pstar)
    v = _golden_velocities()
    f = linear.equilibrium_f(lat, rho, 0.0, 0.0, T)
    E = (-28 + 13 * (v ** 2).sum(1)) @ f
    pxx = (v[:, 0] ** 2) @ f
    assert pxx == pytest.approx(g["momentum_rho_coefficient"] * rho + g["momentum_E_coefficient"] * E, rel=1e-13)


@pytest.mark.parametrize("c1,E0", [(-1.0, -13.024), (-1.2, -13.5), (-0.9, -13.2)])
def test_energy_flux_matches_first_order_system(pstar, c1, E0):
    """To first order in j at rho = 1, E = E0 the energy flux
    sum v_x (-28 + 13|v|^2) f_eq equals (1/2)(39 + 13 c1 + 2 E0) j_x
    (Eq. d2q13-equiv-edp-ordre-1).  This fixes the sign of q (R1) and h1, k1."""
    from oracle import linear
    g = _golden_first_order()
    p = dict(pstar, c1=c1, E0=E0)
    lat = O.Lattice(2, 2, p)
    v = _golden_velocities()
    T0 = (E0 + 28) / 26
    u = 1e-6
    f = linear.equilibrium_f(lat, 1.0, u, 0.0, T0)
    e = -28 + 13 * (v ** 2).sum(1)
    flux = (v[:, 0] * e) @ f
    expect = (g["energy_flux_constant"] + g["energy_flux_c1"] * c1 + g["energy_flux_E0"] * E0) * u
    assert flux == pytest.approx(expect, rel=1e-7)


def test_rest_weights_are_positive_and_sum_to_one(pstar):
    c = O.Lattice(2, 2, pstar).constants()
    assert c["w"].sum() == pytest.approx(1.0, abs=1e-14)
    assert (c["w"] > 0).all()
    assert c["T0"] == pytest.approx((pstar["E0"] + 28) / 26)


def test_rates_in_stable_range_and_rejected_outside(pstar):
    c = O.Lattice(2, 2, pstar).constants()
    s = c["s"][[2, 3, 6, 7, 8, 9, 10, 11, 12]]
    assert ((s > 0) & (s < 2)).all()
    with pytest.raises(ValueError):
        O.Lattice(2, 2, dict(pstar, s_eps=2.5))
    with pytest.raises(ValueError):
        O.Lattice(2, 2, dict(pstar, nu=-0.2))
