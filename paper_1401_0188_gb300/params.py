"""Free-parameter sets for the D2Q13 scheme (host side).

Sec. 2 leaves E0, c1, k2, c_epsE, c_varpirho, c_varpiE and the rates s_XX,
s_r, s_eps, s_varpi, s_XXe free, chosen by scanning the dispersion relation;
the paper prints no values.  `pstar` is one linearly stable choice: rest
populations at weights (0.53, 0.049, 0.0175, 0.051) for the rest particle, the
unit axes, the diagonals and the distance-2 axes (which fixes E0, eps0, varpi0
as their moments), c1 = -1, k2 = 0.4, c_varpiE = 0.3,
c_varpirho = varpi0 - c_varpiE E0, rates s_eps 0.6, s_varpi 1.25, s_r 1.2,
s_XXe 1.0, and c_epsE solved so that eps_eq at rest stays eps0 once c_erho
follows the Prandtl number (Eq. d2q13-sigma-qx).
"""

# Values of the E, eps and varpi polynomials of Eq. (d2q13-polynomes) on the
# four velocity shells |v|^2 = 0, 1, 2, 4 (four velocities each but the first).
_SHELL_E = (-28.0, -15.0, -2.0, 24.0)
_SHELL_EPS = (140.0, -2.0, -67.0, 34.0)
_SHELL_VPI = (-12.0, 8.0, -6.0, 1.0)
_WEIGHTS = (0.53, 0.049, 0.0175, 0.051)


def _shell_moment(row):
    return row[0] * _WEIGHTS[0] + 4.0 * sum(r * w for r, w in zip(row[1:], _WEIGHTS[1:]))


def pstar(nu=0.05, Pr=0.71):
    E0 = _shell_moment(_SHELL_E)
    eps0 = _shell_moment(_SHELL_EPS)
    vpi0 = _shell_moment(_SHELL_VPI)
    c1, k2, cvE = -1.0, 0.4, 0.3
    A = 13.0 * c1 + 95.0 + 2.0 * E0
    # c_erho(c) + c E0 = eps0 with c_erho = 140 + 28 c + A (B0 - 11492 c) / (22984 Pr)
    B0 = 114404.0 + 51051.0 * c1 + 7854.0 * E0
    const = 140.0 + A * B0 / (22984.0 * Pr) - eps0
    slope = 28.0 - A * 11492.0 / (22984.0 * Pr) + E0
    ceE = -const / slope
    return {"E0": E0, "c1": c1, "k2": k2, "c_epsE": ceE, "c_vpi_rho": vpi0 - cvE * E0, "c_vpi_E": cvE,
            "Pr": Pr, "nu": nu, "s_eps": 0.6, "s_vpi": 1.25, "s_r": 1.2, "s_XXe": 1.0}


def rest_temperature(params):
    """T0 = (E0 + 28) / 26: the temperature p / rho of the rest state."""
    return (params["E0"] + 28.0) / 26.0


# Free-parameter sets found by stability.search (Nelder-Mead on the linear
# stability scan at background speeds up to 0.03), as raw search vectors
# (x0, x1, x2, x3, c1, k2, c_varpiE, s_eps, s_varpi, s_r, s_XXe); see
# stability.make_params for the mapping.  Scanned stable (max |z| <= 1 + 1e-9
# on a 21 x 21 k-grid, |U| <= 0.03):
#   SET_LOW_NU   nu in [0.003, 0.1] for Pr in [0.5, 0.71] (searched at nu 0.003, Pr 0.71);
#   SET_HIGH_PR  nu in [0.01, 0.35] for Pr in [0.5, 1.0]  (searched at nu 0.005, Pr 1.0);
#   SET_GAP      nu in [0.005, 0.03] for Pr in [0.5, 0.95] (searched at nu 0.004, Pr 0.95).
# pstar itself is stable for nu >= 0.03 at Pr <= 0.9 and unstable for Pr >= 0.93.
SET_LOW_NU = (0.5105925173414232, 0.36284305707154935, 0.15375698786144854, 0.19957761259165652,
              -0.8246361124294435, 0.45127975266252085, 0.042829871476437284, 0.30139798738512336,
              0.6571556784798335, 0.4287662694105171, 1.4000349991716017)
SET_HIGH_PR = (0.5380898546127793, 0.16261587889116952, 0.11007573675017865, 0.20438685516974286,
               -0.9009122586041832, 0.5225617224127665, 0.05449435477260242, 0.4203578356399446,
               0.7999481655065166, 0.7180603877966116, 1.4786106341856398)

SET_GAP = (0.514685701857462, 0.17842478563835837, 0.12038160750190877, 0.20614735400913026,
           -0.9404624029864772, 0.49908866373015703, 0.05020697851061984, 0.4543578998715883,
           0.7805796117579609, 0.659693290434811, 1.5179765139129429)


# A set with physical viscous heating: c1 follows E0 through
# stability.heating_c1, so sigma_q gamma = nu (stability.viscous_heating_factor
# = 1 for every nu and Pr; pstar gives -0.53 and the sets above 0.88 to 1.18).
# Searched at nu 0.05, Pr 0.71 with physical_heating; scanned stable for nu in
# [0.005, 0.35] at Pr in [0.5, 0.71], [0.005, 0.2] at Pr 0.9 and
# [0.005, 0.05] at Pr 0.95.
SET_HEAT = (0.501485, 0.176529, 0.121983, 0.211432, -0.955121, 0.508922, 0.051073, 0.454721, 0.783621,
            0.656364, 1.479079)


def _heat_set_stable(nu, Pr):
    if not (0.5 <= Pr <= 0.95 and nu >= 0.005):
        return False
    return nu <= (0.35 if Pr <= 0.71 else 0.2 if Pr <= 0.9 else 0.05)


_SEARCHED = {}


def _gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except ImportError:
        return False


def select(nu, Pr, physical_heating=True, search="auto"):
    """A free-parameter set that is linearly stable at (nu, Pr) for background
    speeds up to 0.03; with physical_heating (the default) the SET_HEAT family
    wherever it is stable, else the sets above.  Outside their ranges, with
    search = "auto" and a CUDA device (or search = True), the sets are searched
    on demand by stability.search_batched (the batched GPU scan of the end of
    Sec. 2) and the result kept for the process; ValueError when that finds no
    stable set, or without a search."""
    from . import stability
    if physical_heating and _heat_set_stable(nu, Pr):
        return stability.make_params(SET_HEAT, nu, Pr, physical_heating=True)
    if nu >= 0.01 and 0.5 <= Pr <= 1.0:
        return stability.make_params(SET_HIGH_PR, nu, Pr)
    if 0.003 <= nu <= 0.1 and 0.5 <= Pr <= 0.71:
        return stability.make_params(SET_LOW_NU, nu, Pr)
    if 0.005 <= nu <= 0.03 and 0.5 <= Pr <= 0.95:
        return stability.make_params(SET_GAP, nu, Pr)
    if search is True or (search == "auto" and _gpu_available()):
        key = (round(nu, 12), round(Pr, 12), bool(physical_heating))
        if key not in _SEARCHED:
            p, g, _ = stability.search_batched(nu, Pr, physical_heating=physical_heating)
            _SEARCHED[key] = p if g <= 1e-11 else None
        if _SEARCHED[key] is not None:
            return dict(_SEARCHED[key])
    raise ValueError(f"no stable parameter set known for nu = {nu}, Pr = {Pr}")


def stable_viscosity(nu, Pr):
    """The smallest viscosity >= nu for which select() has a set."""
    if 0.5 <= Pr <= 0.71:
        return max(nu, 0.003)
    if Pr <= 0.95:
        return max(nu, 0.005)
    return max(nu, 0.01)
