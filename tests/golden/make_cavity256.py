"""Writes cavity256_oracle.json: the differentially heated cavity of Sec. 10
on a 256 x 256 lattice, run by the FP64 CPU oracle to a steady residual, at
Ra = 1e3, 1e4 and 1e5 (Pr = 0.71, the Prandtl number of Table 1).

Set-up (the paper prints no lattice values; these are the readings the
library's cavity set-up takes, restated here so that this script calls the
oracle and the seeded input module only):
  - parameters: the oracle's `pstar` set at nu = U_ff L sqrt(Pr / Ra) with
    U_ff = 0.05, clamped to [0.01, 0.35];
  - Ra = g beta dT L^3 / (nu kappa), kappa = nu / Pr, beta = 1 / T0 (a gas at
    constant pressure), dT = 0.01, so g = Ra nu kappa / (beta dT L^3);
  - walls: hot west / cold east velocity+temperature walls at T0 +- dT/2 with
    the zero-net-mass-flux wall density (reading R12'), adiabatic south and
    north walls, buoyancy F = -g (rho - 1) y-hat;
  - start at rest (rho = 1, u = 0, T = T0); every 1000 steps the residual of
    reading R17; stop at residual <= 1e-8.
Stored per Rayleigh number: the parameters and boundary as used, the step
count, residual, Nusselt number, asymmetries, max |u|, mean T, and u_x, u_y,
T at 36 sampled nodes.  Run: python tests/golden/make_cavity256.py (about an
hour on 8 cores).
"""
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1401_0188_gb300 import workloads as W  # noqa: E402

L = 256
PR = 0.71
DT = 0.01
U_FF = 0.05
TOL = 1e-8
CHECK = 1000
SAMPLE = [8, 51, 102, 153, 204, 247]  # rows and columns of the sampled nodes
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cavity256_oracle.json")


def setup(Ra):
    nu = min(max(U_FF * L * math.sqrt(PR / Ra), 0.01), 0.35)
    p = O.pstar(nu, PR)
    T0 = (p["E0"] + 28.0) / 26.0
    kappa = nu / PR
    g = Ra * nu * kappa * T0 / (DT * L ** 3)
    bnd = W.cavity(T0, DT, g, rho_ref=1.0, wall_density=1)
    return p, bnd, T0


def run(Ra, nthreads):
    p, bnd, T0 = setup(Ra)
    o = O.Lattice(L, L, p, bnd, nthreads=nthreads)
    o.set_equilibrium(1.0, 0.0, 0.0, T0)
    o.residual()
    t0 = time.time()
    r = None
    while o.t < 3_000_000:
        o.step(CHECK)
        r = o.residual()
        if r[0] <= TOL:
            break
    macro = o.macro()  # rho, ux, uy, T
    samples = [[int(y), int(x), float(macro[1, y, x]), float(macro[2, y, x]), float(macro[3, y, x])]
               for y in SAMPLE for x in SAMPLE]
    return {"Ra": Ra, "params": {k: float(v) for k, v in p.items()}, "boundary": bnd, "T0": T0,
            "steps": int(o.t), "residual": float(r[0]), "Nu": float(r[8]), "S_u": float(r[9]),
            "S_T": float(r[10]), "umax": float(r[11]), "Tmean": float(r[15]),
            "samples_y_x_ux_uy_T": samples, "oracle_seconds": time.time() - t0, "threads": nthreads}


def main():
    nthreads = os.cpu_count() or 1
    out = {"what": "Sec. 10 differentially heated cavity, 256 x 256, FP64 oracle to residual 1e-8",
           "cite": "Sec. 10 (de Vahl Davis cavity, Table 1 Rayleigh numbers; Pr = 0.71)",
           "L": L, "Pr": PR, "dT": DT, "tol": TOL, "check_every": CHECK, "runs": []}
    for Ra in (1e3, 1e4, 1e5):
        res = run(Ra, nthreads)
        out["runs"].append(res)
        print(json.dumps({k: res[k] for k in ("Ra", "steps", "residual", "Nu", "S_u", "oracle_seconds")}),
              flush=True)
        with open(OUT, "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
