"""Runs described by a JSON file: one lattice, its parameters, walls,
forcing and initial state, stepped for a fixed count or to a steady state,
with one JSON line of read-outs per report.

    python -m paper_1401_0188_gb300.runconfig run.json

A description (every key but "nx" and "ny" optional):

    {"nx": 256, "ny": 256, "precision": "fp32" | "fp64",
     "params": {"nu": 0.05, "Pr": 0.71, "set": "pstar" | "select"}
               or the twelve free parameters of lbm13_params by name,
     "walls": {"west": {"kind": "mixed", "u": 0.0, "T": 0.581}, "east": ...,
               "south": {"kind": "bb"}, "north": {"kind": "bb", "u": 0.02}},
               (omitted sides are periodic; "T_offset" instead of "T" is
               relative to the rest temperature)
     "force": {"gx": 0.0, "gy": -1e-4, "rho_ref": 1.0}, "heat": 0.0,
     "wall_density": "extrapolated" | "zero_flux",
     "init": {"rho": 1.0, "ux": 0.0, "uy": 0.0, "T_offset": 0.0,
              "shear_wave": 0.01},
     "steps": 10000   or   "steady": {"tol": 1e-8, "check_every": 1000,
                                      "max_steps": 2000000},
     "report_every": 1000}

Each report line holds the step, the residual, the conserved totals, the
Nusselt number and asymmetry read-outs, and the updates per second since
the previous line; the last line adds the run's wall time.
"""
import json
import sys
import time

from . import lbm13, params as P, workloads as W

_KINDS = {"periodic": W.PERIODIC, "bb": W.WALL_BB, "mixed": W.WALL_MIXED}
_PRECISIONS = {"fp32": lbm13.FP32_DEVIATION, "fp64": lbm13.FP64}


def parameters(desc):
    """The free-parameter set a description names."""
    p = desc.get("params", {})
    if all(k in p for k in lbm13.PARAM_FIELDS):
        return {k: float(p[k]) for k in lbm13.PARAM_FIELDS}
    nu, Pr = float(p.get("nu", 0.05)), float(p.get("Pr", 0.71))
    choice = p.get("set", "pstar")
    if choice == "pstar":
        return P.pstar(nu, Pr)
    if choice == "select":
        return P.select(nu, Pr)
    raise ValueError(f"params.set must be 'pstar' or 'select', not {choice!r}")


def setup(desc):
    """(nx, ny, params, boundary dict, precision) of a description."""
    nx, ny = int(desc["nx"]), int(desc["ny"])
    prec = _PRECISIONS[desc.get("precision", "fp32")]
    p = parameters(desc)
    T0 = P.rest_temperature(p)
    walls = {}
    for side in ("west", "east", "south", "north"):
        w = desc.get("walls", {}).get(side)
        if w is None:
            walls[side] = W.wall()
            continue
        kind = _KINDS[w.get("kind", "bb")]
        T = float(w["T"]) if "T" in w else T0 + float(w.get("T_offset", 0.0))
        walls[side] = W.wall(kind, float(w.get("u", 0.0)), T)
    force = desc.get("force", {})
    density = desc.get("wall_density", "extrapolated")
    if density not in ("extrapolated", "zero_flux"):
        raise ValueError("wall_density must be 'extrapolated' or 'zero_flux'")
    bnd = W.boundary(**walls, gx=float(force.get("gx", 0.0)), gy=float(force.get("gy", 0.0)),
                     rho_ref=float(force.get("rho_ref", 0.0)), wall_density=1 if density == "zero_flux" else 0,
                     heat=float(desc.get("heat", 0.0)))
    return nx, ny, p, bnd, prec


def initial_fields(desc, nx, ny, T0):
    init = desc.get("init", {})
    rho = float(init.get("rho", 1.0))
    ux, uy = float(init.get("ux", 0.0)), float(init.get("uy", 0.0))
    T = T0 + float(init.get("T_offset", 0.0))
    if "shear_wave" in init:
        wx, _ = W.shear_wave(nx, ny, float(init["shear_wave"]))
        ux = ux + wx
    return rho, ux, uy, T


def _line(lat, res, steps, dt, **extra):
    out = {"t": int(lat.t), "residual": float(res[0]), "Nu": float(res[8]), "S_u": float(res[9]),
           "S_T": float(res[10]), "umax": float(res[11]), "MLUPS": lat.nx * lat.ny * steps / dt / 1e6 if dt > 0 else None}
    out.update(extra)
    return out


def run(desc, emit=print):
    """Step the described lattice; emit one JSON line per report."""
    nx, ny, p, bnd, prec = setup(desc)
    lat = lbm13.Lattice(nx, ny, p, bnd, precision=prec)
    lat.set_state(*initial_fields(desc, nx, ny, P.rest_temperature(p)))
    lat.residual()
    every = int(desc.get("report_every", 1000))
    steady = desc.get("steady")
    total = int(desc.get("steps", 0))
    max_steps = int(steady.get("max_steps", 2_000_000)) if steady else total
    tol = float(steady.get("tol", 1e-8)) if steady else None
    if steady:
        every = int(steady.get("check_every", every))
    t_start = time.perf_counter()
    res = None
    while lat.t < max_steps:
        n = min(every, max_steps - lat.t)
        t0 = time.perf_counter()
        lat.step(n)
        res = lat.residual()
        emit(json.dumps(_line(lat, res, n, time.perf_counter() - t0)))
        if tol is not None and res[0] <= tol:
            break
    wall = time.perf_counter() - t_start
    last = _line(lat, res if res is not None else lat.residual(), 0, 0.0, wall_s=wall,
                 converged=bool(tol is not None and res is not None and res[0] <= tol))
    emit(json.dumps(last))
    lat.close()
    return last


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    if len(argv) != 1:
        print(__doc__)
        return 2
    with open(argv[0]) as f:
        run(json.load(f))
    return 0


if __name__ == "__main__":
    sys.exit(main())
