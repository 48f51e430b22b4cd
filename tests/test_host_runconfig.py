"""JSON run descriptions (no GPU): parsing into parameters, walls, forcing
and initial fields, and the C structs the library takes."""
import json

import pytest

from paper_1401_0188_gb300 import lbm13, params as P, runconfig as R, workloads as W


def test_cavity_description():
    desc = json.loads('''{"nx": 64, "ny": 48, "precision": "fp64",
        "params": {"nu": 0.05, "Pr": 0.71},
        "walls": {"west": {"kind": "mixed", "T_offset": 0.005}, "east": {"kind": "mixed", "T_offset": -0.005},
                  "south": {"kind": "bb"}, "north": {"kind": "bb", "u": 0.02}},
        "force": {"gy": -1e-4, "rho_ref": 1.0}, "wall_density": "zero_flux",
        "init": {"T_offset": 0.001}, "steady": {"tol": 1e-8}}''')
    nx, ny, p, bnd, prec = R.setup(desc)
    T0 = P.rest_temperature(p)
    assert (nx, ny, prec) == (64, 48, lbm13.FP64)
    assert p == P.pstar(0.05, 0.71)
    assert bnd["west"] == W.wall(W.WALL_MIXED, 0.0, T0 + 0.005)
    assert bnd["east"] == W.wall(W.WALL_MIXED, 0.0, T0 - 0.005)
    # an adiabatic wall's temperature is not used
    assert (bnd["south"]["kind"], bnd["south"]["u_t"]) == (W.WALL_BB, 0.0)
    assert (bnd["north"]["kind"], bnd["north"]["u_t"]) == (W.WALL_BB, 0.02)
    assert (bnd["gy"], bnd["rho_ref"], bnd["wall_density"]) == (-1e-4, 1.0, 1)
    b = lbm13.make_boundary(bnd)
    assert b.west.kind == W.WALL_MIXED and b.north.u_t == pytest.approx(0.02) and b.wall_density == 1
    rho, ux, uy, T = R.initial_fields(desc, nx, ny, T0)
    assert (rho, ux, uy) == (1.0, 0.0, 0.0) and T == pytest.approx(T0 + 0.001)


def test_periodic_defaults_and_explicit_parameters():
    p = P.pstar(0.02, 0.6)
    nx, ny, q, bnd, prec = R.setup({"nx": 32, "ny": 16, "params": dict(p), "init": {"shear_wave": 0.01}})
    assert q == pytest.approx(p) and prec == lbm13.FP32_DEVIATION
    assert all(bnd[s]["kind"] == W.PERIODIC for s in ("west", "east", "south", "north"))
    _, ux, _, _ = R.initial_fields({"init": {"shear_wave": 0.01}}, nx, ny, 0.5)
    assert ux.shape == (16, 32) and abs(ux).max() == pytest.approx(0.01, rel=1e-2)


def test_bad_descriptions_are_rejected():
    with pytest.raises(KeyError):
        R.setup({"nx": 8, "ny": 8, "walls": {"west": {"kind": "slippery"}}})
    with pytest.raises(ValueError):
        R.setup({"nx": 8, "ny": 8, "wall_density": "sticky"})
    with pytest.raises(ValueError):
        R.setup({"nx": 8, "ny": 8, "params": {"set": "best"}})
