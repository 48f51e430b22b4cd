"""Validation runs of the CUDA time step on the paper's test cases.

  python -m paper_1401_0188_gb300.validate cavity  [--L 256] [--Ra 1e3 1e4 1e5] [--tol 1e-8]
  python -m paper_1401_0188_gb300.validate channels [--nx 1024] [--ny 128]

`cavity`: the differentially heated cavity of Sec. 10 in FP64 and in
FP32-deviation storage, each run until the residual reaches `tol`; prints per
run Nu, the centro-asymmetry S_u, S_T, max |u|, steps and time, then the FP32
error against FP64 per result.
`channels`: the Couette flow of Sec. 7 (moving heated upper wall) and the
Poiseuille flow of Sec. 8 (body force), compared with their closed forms.
One JSON object per line.
"""
import argparse
import json
import math

import numpy as np

from . import cavity, lbm13, params as P, workloads as W


def run_cavity(L, Ras, Pr, tol, check_every, max_steps):
    for Ra in Ras:
        res = {}
        for prec in (lbm13.FP64, lbm13.FP32_DEVIATION):
            r = cavity.solve(L, Ra, Pr, precision=prec, tol=tol, check_every=check_every, max_steps=max_steps)
            fields = r.pop("fields")
            r.pop("history")
            res[r["precision"]] = (r, fields)
            print(json.dumps({"case": "cavity", **r}), flush=True)
        (a, fa), (b, fb) = res["fp64"], res["fp32-deviation"]
        err = {"case": "cavity_fp32_error", "L": L, "Ra": Ra,
               "Nu": abs(b["Nu"] - a["Nu"]), "S_u": abs(b["S_u"] - a["S_u"]), "S_T": abs(b["S_T"] - a["S_T"]),
               "u_max_abs": float(max(np.abs(fb[1] - fa[1]).max(), np.abs(fb[2] - fa[2]).max())),
               "T_max_abs": float(np.abs(fb[3] - fa[3]).max()), "rho_max_abs": float(np.abs(fb[0] - fa[0]).max())}
        print(json.dumps(err), flush=True)


def run_channels(nx, ny, steps_factor):
    p = P.pstar(0.05, 0.71)
    T0 = P.rest_temperature(p)
    nu = p["nu"]
    eta = np.arange(ny) + 0.5
    steps = int(steps_factor * ny * ny / nu)
    for prec in (lbm13.FP64, lbm13.FP32_DEVIATION):
        name = "fp64" if prec == lbm13.FP64 else "fp32-deviation"
        # Poiseuille (Sec. 8): walls at rest holding T0, body force rho g along x
        g = 1e-6
        lat = lbm13.Lattice(nx, ny, p, W.poiseuille(g, T0=T0, dT=0.0, wall_density=1), precision=prec)
        lat.set_state(1.0, 0.0, 0.0, T0)
        lat.step(steps)
        u = lat.macro()[1]
        exact = g * eta * (ny - eta) / (2 * nu)
        prof = u.mean(axis=1)
        print(json.dumps({"case": "poiseuille", "precision": name, "nx": nx, "ny": ny, "steps": steps, "g": g,
                          "u_max": float(prof.max()), "u_max_exact": float(exact.max()),
                          "rel_L2": float(np.linalg.norm(prof - exact) / np.linalg.norm(exact)),
                          "x_variation": float(np.abs(u - prof[:, None]).max()),
                          "T_mean": float(lat.macro()[3].mean())}), flush=True)
        lat.close()
        # Couette: lower wall at rest at T0 - dT/2, upper wall at U and T0 + dT/2
        U, dT = 0.05, 0.01
        lat = lbm13.Lattice(nx, ny, p, W.couette(T0, U, dT, wall_density=1), precision=prec)
        lat.set_state(1.0, 0.0, 0.0, T0)
        lat.step(steps)
        m = lat.macro()
        ux = m[1].mean(axis=1)
        T = m[3].mean(axis=1)
        exact_u = U * eta / ny
        exact_T = T0 - dT / 2 + dT * eta / ny
        print(json.dumps({"case": "couette", "precision": name, "nx": nx, "ny": ny, "steps": steps, "U": U, "dT": dT,
                          "u_rel_L2": float(np.linalg.norm(ux - exact_u) / np.linalg.norm(exact_u)),
                          "T_dev_max_over_dT": float(np.abs(T - exact_T).max() / dT),
                          "uy_max": float(np.abs(m[2]).max()), "rho_mean": float(m[0].mean())}), flush=True)
        lat.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("cavity")
    c.add_argument("--L", type=int, default=256)
    c.add_argument("--Ra", type=float, nargs="+", default=[1e3, 1e4, 1e5])
    c.add_argument("--Pr", type=float, default=0.71)
    c.add_argument("--tol", type=float, default=1e-8)
    c.add_argument("--check-every", type=int, default=1000)
    c.add_argument("--max-steps", type=int, default=3_000_000)
    h = sub.add_parser("channels")
    h.add_argument("--nx", type=int, default=1024)
    h.add_argument("--ny", type=int, default=128)
    h.add_argument("--steps-factor", type=float, default=3.0)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    if a.cmd == "cavity":
        run_cavity(a.L, a.Ra, a.Pr, a.tol, a.check_every, a.max_steps)
    else:
        run_channels(a.nx, a.ny, a.steps_factor)


if __name__ == "__main__":
    main()
