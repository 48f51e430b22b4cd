"""Differentially heated square cavity (de Vahl Davis test, Sec. 10) on the
CUDA time step: parameter set-up from (L, Ra, Pr) and a run to steady state.

Set-up readings (the paper gives no lattice values):
- Rayleigh number Ra = g beta dT L^3 / (nu kappa) (Sec. 1, Eq. intro-rayleigh)
  with kappa = nu / Pr and, for the gas the D2Q13 scheme models, beta = 1/T0
  (at constant pressure rho ~ 1/T), T0 the rest temperature (E0 + 28)/26.
- Viscosity from a target free-fall speed U_ff = sqrt(g beta dT L):
  nu = U_ff L sqrt(Pr / Ra), clamped to [nu_min, nu_max]; then g follows Ra.
- Walls: hot west and cold east velocity+temperature walls at T0 +- dT/2,
  adiabatic south and north walls, buoyancy F = -g (rho - 1) y-hat.  The
  temperature walls take the zero-net-mass-flux density by default: with the
  extrapolated density of Sec. 7 mass leaks through them (~1e-8 per step per
  node) and, since the scheme's transport coefficients are calibrated at
  rho = 1, the solution drifts and never reaches a steady residual.
"""
import math
import time

from . import lbm13, params as P, workloads as W


def setup(L, Ra, Pr, dT=0.01, U_ff=0.05, nu_min=0.01, nu_max=0.35, param_fn=None, wall_density=1):
    """Returns (params, boundary, info) for an L x L cavity."""
    nu = min(max(U_ff * L * math.sqrt(Pr / Ra), nu_min), nu_max)
    p = (param_fn or P.pstar)(nu, Pr)
    T0 = P.rest_temperature(p)
    kappa = nu / Pr
    beta = 1.0 / T0
    g = Ra * nu * kappa / (beta * dT * L ** 3)
    bnd = W.cavity(T0, dT, g, rho_ref=1.0, wall_density=wall_density)
    info = {"L": L, "Ra": Ra, "Pr": Pr, "dT": dT, "nu": nu, "kappa": kappa, "g": g, "T0": T0,
            "U_ff": math.sqrt(g * beta * dT * L)}
    return p, bnd, info


def run_to_steady(lat, tol=1e-8, check_every=1000, max_steps=2_000_000, on_check=None):
    """Step until the residual (r of lbm13_residual) falls to `tol`, checking
    every `check_every` steps.  Returns a dict with the last read-outs."""
    lat.residual()
    t0 = time.perf_counter()
    hist = []
    out = None
    while lat.t < max_steps:
        lat.step(check_every)
        out = lat.residual()
        hist.append((lat.t, out[0]))
        if on_check:
            on_check(lat.t, out)
        if out[0] <= tol:
            break
    wall = time.perf_counter() - t0
    return {"steps": int(lat.t), "residual": float(out[0]), "converged": bool(out[0] <= tol),
            "Nu": float(out[8]), "S_u": float(out[9]), "S_T": float(out[10]), "umax": float(out[11]),
            "wall_s": wall, "history": hist}


def solve(L, Ra, Pr=0.71, precision=lbm13.FP64, tol=1e-8, check_every=1000, max_steps=2_000_000, **kw):
    p, bnd, info = setup(L, Ra, Pr, **kw)
    lat = lbm13.Lattice(L, L, p, bnd, precision=precision)
    lat.set_state(1.0, 0.0, 0.0, info["T0"])
    res = run_to_steady(lat, tol, check_every, max_steps)
    res.update(info)
    res["precision"] = "fp64" if precision == lbm13.FP64 else "fp32-deviation"
    res["fields"] = lat.macro()
    lat.close()
    return res


