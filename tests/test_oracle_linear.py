"""Pins of the oracle's linearised behaviour against Sec. 2 and Sec. 6: the
hydrodynamic modes carry the input viscosity and Prandtl number (readings R4,
R5), decay isotropically (Eq. d2q13-sigma-qx), advect with the background flow
(Eq. d2q13-diffusion), propagate sound at the speed of the printed first-order
system (Eq. d2q13-equiv-edp-ordre-1), and the chosen parameters are linearly
stable (end of Sec. 2)."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from oracle import linear

KK = 0.02  # small wave number: O(k^2) dispersion stays below 1e-3 relative


def _golden():
    d = {}
    for l in open(os.path.join(os.path.dirname(__file__), "golden", "first_order_system.txt")):
        if l.strip() and not l.startswith("#"):
            k, v = l.split()
            d[k] = float(Fraction(v))
    return d


@pytest.fixture(scope="module")
def rest(pstar):
    lat = O.Lattice(2, 2, pstar)
    J, _ = linear.collision_jacobian(lat)
    return lat, J


def _modes(J, theta, U=(0.0, 0.0)):
    k = (KK * np.cos(theta), KK * np.sin(theta))
    z, V = linear.hydrodynamic_modes(J, k)
    lz = np.log(z)
    kU = k[0] * U[0] + k[1] * U[1]
    return lz, V, kU


def _split(lz, kU):
    """(non-propagating pair sorted by decay, acoustic pair)."""
    prop = np.abs(lz.imag + kU) > 0.1 * KK
    still = sorted(lz[~prop], key=lambda c: -c.real)
    return still, lz[prop]


@pytest.mark.parametrize("theta", [0.0, np.pi / 8, np.pi / 4])
def test_shear_mode_decays_at_input_viscosity(pstar, rest, theta):
    _, J = rest
    lz, _, kU = _modes(J, theta)
    (shear, diff), _ = _split(lz, kU)
    assert -shear.real / KK ** 2 == pytest.approx(pstar["nu"], rel=2e-4)


@pytest.mark.parametrize("theta", [0.0, np.pi / 8, np.pi / 4])
def test_diffusive_mode_carries_prandtl_number(pstar, rest, theta):
    _, J = rest
    lz, _, kU = _modes(J, theta)
    (shear, diff), _ = _split(lz, kU)
    kappa = -diff.real / KK ** 2
    assert pstar["nu"] / kappa == pytest.approx(pstar["Pr"], rel=1e-3)


@pytest.mark.parametrize("theta", [0.0, np.pi / 8, np.pi / 4])
def test_sound_speed_matches_first_order_system(pstar, rest, theta):
    g = _golden()
    _, J = rest
    lz, _, kU = _modes(J, theta)
    _, ac = _split(lz, kU)
    cs2 = g["momentum_rho_coefficient"] + g["momentum_E_coefficient"] * (
        g["energy_flux_constant"] + g["energy_flux_c1"] * pstar["c1"] + g["energy_flux_E0"] * pstar["E0"])
    assert np.abs(ac.imag / KK) == pytest.approx([np.sqrt(cs2)] * 2, rel=2e-4)


def test_acoustic_damping_is_isotropic(rest):
    _, J = rest
    damp = []
    for th in (0.0, np.pi / 8, np.pi / 4):
        lz, _, kU = _modes(J, th)
        _, ac = _split(lz, kU)
        damp.append(-ac.real.mean() / KK ** 2)
    assert max(damp) / min(damp) - 1 < 1e-3


@pytest.mark.parametrize("U", [(0.02, 0.0), (0.014, 0.014), (0.0, -0.02)])
def test_modes_advect_with_background_flow(pstar, U):
    """Galilean constraints of Eq. (d2q13-diffusion): all four hydrodynamic
    modes are Doppler shifted by k.U."""
    lat = O.Lattice(2, 2, pstar)
    J, _ = linear.collision_jacobian(lat, 1.0, U[0], U[1])
    spd = np.hypot(*U)
    for th in (0.0, np.pi / 8, np.pi / 4):
        lz, _, kU = _modes(J, th, U)
        still, ac = _split(lz, kU)
        for m in still:
            assert abs(m.imag + kU) < 1e-2 * KK * spd
        assert abs(ac.imag.mean() + kU) < 1e-2 * KK * spd


def test_viscosity_independent_of_parallel_flow(pstar):
    lat = O.Lattice(2, 2, pstar)
    J, _ = linear.collision_jacobian(lat, 1.0, 0.02, 0.0)
    lz, _, kU = _modes(J, 0.0, (0.02, 0.0))
    (shear, diff), _ = _split(lz, kU)
    assert -shear.real / KK ** 2 == pytest.approx(pstar["nu"], rel=1e-2)


def test_diffusive_mode_at_rest_is_constant_pressure(pstar, rest):
    """Sec. 6: without advection the diffusive mode is (rho, j, E) = (1, 0, -28)."""
    g = _golden()
    _, J = rest
    M, _, _ = O.basis()
    lz, V, kU = _modes(J, 0.0)
    (shear, diff), _ = _split(lz, kU)
    i = int(np.argmin(np.abs(lz - diff)))
    m = M @ V[:, i]
    assert (m[1] / m[0]).real == pytest.approx(g["diffusive_mode_E_over_rho"], rel=1e-4)
    assert abs(m[4] / m[0]) < 1e-2 and abs(m[5] / m[0]) < 1e-2


@pytest.mark.parametrize("V", [0.0, 0.03, 0.06])
def test_momentum_flux_with_transverse_velocity(pstar, V):
    """Sec. 6, Eq. (d2q13-equiv-edp-ordre-1) with a transverse velocity V: the
    momentum-flux row is (14/13 + V^2/2) d rho + (1/26) d E (transverse momentum
    held), whose null vector is E = -(28 + 13 V^2) rho."""
    g = _golden()
    lat = O.Lattice(2, 2, pstar)
    vx, vy = O.velocities()
    e_of = -28 + 13 * (vx ** 2 + vy ** 2)

    def pxx(rho, E, jt):
        uy = jt / rho
        T = ((E + 28 * rho) / rho - 13 * uy * uy) / 26
        f = linear.equilibrium_f(lat, rho, 0.0, uy, T)
        assert e_of @ f == pytest.approx(E, abs=1e-12)
        return (vx ** 2) @ f

    E0 = pstar["E0"] + 13 * V * V
    h = 1e-5
    d_rho = (pxx(1 + h, E0, V) - pxx(1 - h, E0, V)) / (2 * h)
    d_E = (pxx(1, E0 + h, V) - pxx(1, E0 - h, V)) / (2 * h)
    assert d_rho == pytest.approx(g["momentum_rho_coefficient"] + V * V / 2, rel=1e-8)
    assert d_E == pytest.approx(g["momentum_E_coefficient"], rel=1e-8)
    assert -d_rho / d_E == pytest.approx(g["diffusive_mode_E_over_rho"] + g["diffusive_mode_transverse_V2"] * V * V, rel=1e-8)


@pytest.mark.parametrize("U", [(0.0, 0.0), (0.02, 0.0), (0.014, 0.014)])
def test_parameter_set_is_linearly_stable(pstar, U):
    lat = O.Lattice(2, 2, pstar)
    J, _ = linear.collision_jacobian(lat, 1.0, U[0], U[1])
    assert linear.max_modulus(J, n=25) <= 1 + 1e-9


def test_each_moment_relaxes_at_its_own_rate(pstar, rest):
    """Sec. 2, the multiple-relaxation-time collision: a perturbation along one
    non-conserved moment of the basis (the population vector whose moments are
    that unit moment alone) leaves rho, E and j unchanged, so the equilibria do
    not move, and one collision multiplies it by 1 - s_k.  The rates are those
    of the parameter list (s_eps, s_varpi, s_r, s_XXe as given), s_q and s_XX
    from 1/(sigma + 1/2) (sigma_XX from nu, R4; sigma_q the derived constant of
    Eq. (d2q13-sigma-qx)), and R3 (each y partner takes its x moment's rate)."""
    lat, J = rest
    _, _, Minv = O.basis()
    c = lat.constants()
    s_q = 1.0 / (c["sigma_q"] + 0.5)
    s_XX = 1.0 / (c["sigma_XX"] + 0.5)
    assert c["sigma_XX"] == pytest.approx(104.0 * pstar["nu"] / c["A"], rel=1e-14)
    rates = {2: pstar["s_eps"], 3: pstar["s_vpi"], 6: s_q, 7: s_q, 8: pstar["s_r"], 9: pstar["s_r"],
             10: s_XX, 11: s_XX, 12: pstar["s_XXe"]}
    for k, s in rates.items():
        v = Minv[:, k]
        assert np.allclose(J @ v, (1.0 - s) * v, rtol=0, atol=1e-8 * np.abs(v).max()), k
