"""Validation runs of the CUDA time step on the paper's test cases.

  python -m paper_1401_0188_gb300.validate cavity  [--L 256] [--Ra 1e3 1e4 1e5] [--tol 1e-8]
  python -m paper_1401_0188_gb300.validate channels [--nx 1024] [--ny 128]
  python -m paper_1401_0188_gb300.validate waves [--precision both]
  python -m paper_1401_0188_gb300.validate serving [--requests 64 --rate 200 --side-max 512 --ra-max 1e6]

`cavity`: the differentially heated cavity of Sec. 10 in FP64 and in
FP32-deviation storage, each run until the residual reaches `tol`; prints per
run Nu, the centro-asymmetry S_u, S_T, max |u|, steps and time, then the FP32
error against FP64 per result.
`channels`: the Couette flow of Sec. 7 (moving heated upper wall) and the
Poiseuille flow of Sec. 8 (body force), compared with their closed forms.
`waves`: the thermal wave (Sec. 4), buoyancy wave (Sec. 5), transverse-wave
aggregates (Sec. 6) and heated slab (Sec. 9) against their closed forms.
`serving`: a Poisson trace of cavity and channel solves served with continuous
batching (p50/p99 time to steady state, throughput) and the Nusselt numbers of
its smallest cavities against plain FP64 runs.
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


def _row(nx, ny, fn):
    return fn(np.arange(nx)[None, :] * np.ones((ny, 1)))


def run_waves(precisions):
    """Sec. 4 thermal wave, Sec. 5 buoyancy wave (510 wide), Sec. 6 transverse
    wave aggregates and the Sec. 9 heated slab, against their closed forms, for
    pstar (viscous heating factor -0.53) and the physical-heating set."""
    from . import stability as S
    sets = {"pstar": P.pstar(0.05, 0.71), "heating": P.select(0.05, 0.71)}
    for prec in precisions:
        name = "fp64" if prec == lbm13.FP64 else "fp32-deviation"
        for sname, p in sets.items():
            T0 = P.rest_temperature(p)
            nu, D = p["nu"], p["nu"] / p["Pr"]
            phi = S.viscous_heating_factor(p)
            # Sec. 6: u_y = V cos kx on 1024 x 2; E~ rate over steps 4..16
            nx, V = 1024, 0.02
            k = 2 * math.pi / nx
            lat = lbm13.Lattice(nx, 2, p, W.boundary(), precision=prec)
            lat.set_state(1.0, 0.0, _row(nx, 2, lambda x: V * np.cos(2 * math.pi * x / nx)), T0)
            lat.step(4)
            a4 = lat.project(1)
            lat.step(12)
            a16 = lat.project(1)
            lat.step(1984)
            a2000 = lat.project(1)
            rate = (a16[4, 1, 0] - a4[4, 1, 0]) / 12
            N = 2 * nx
            print(json.dumps({"case": "transverse_wave", "precision": name, "params": sname, "phi": phi,
                              "E_rate": rate, "E_rate_first_order": -13 * phi * nu * k * k * V * V * N,
                              "E_rate_physical": -13 * nu * k * k * V * V * N,
                              "Vy_decay": math.log(a2000[2, 0, 0] / a16[2, 0, 0]) / 1984, "nu_k2": -nu * k * k}),
                  flush=True)
            lat.close()
            # Sec. 4: T = T0 + dT cos kx at constant pressure on 256 x 2
            nx, dT = 256, 1e-4
            k = 2 * math.pi / nx
            Tf = _row(nx, 2, lambda x: T0 + dT * np.cos(2 * math.pi * x / nx))
            lat = lbm13.Lattice(nx, 2, p, W.boundary(), precision=prec)
            lat.set_state(T0 / Tf, 0.0, 0.0, Tf)
            lat.step(200)
            a1 = lat.project(1)
            lat.step(8000)
            a2 = lat.project(1)
            print(json.dumps({"case": "thermal_wave", "precision": name, "params": sname,
                              "T_decay": math.log(a2[3, 0, 0] / a1[3, 0, 0]) / 8000, "D_k2": -D * k * k,
                              "rho_over_T_times_T0": float(a2[0, 0, 0] / a2[3, 0, 0] * T0)}), flush=True)
            lat.close()
            # Sec. 5: buoyancy on the temperature wave, 510 wide, periodic
            nx, dT, g = 510, 1e-3, 3e-5
            k = 2 * math.pi / nx
            Tf = _row(nx, 2, lambda x: T0 + dT * np.cos(2 * math.pi * x / nx))
            rho = T0 / Tf
            lat = lbm13.Lattice(nx, 2, p, W.boundary(gy=-g, rho_ref=float(rho.mean())), precision=prec)
            lat.set_state(rho, 0.0, 0.0, Tf)
            r0 = lat.project(1)[0, 0, 0]
            out = {"case": "buoyancy_wave", "precision": name, "params": sname, "nx": nx}
            for t in (2000, 20000, 100000):
                lat.step(t - lat.t)
                a = lat.project(1)
                exact = -g * r0 * (math.exp(-D * k * k * t) - math.exp(-nu * k * k * t)) / ((nu - D) * k * k)
                m = lat.macro()
                out[f"Vy_rel_err_t{t}"] = float(a[2, 0, 0] / exact - 1)
                out[f"ux_over_uy_t{t}"] = float(np.abs(m[1]).max() / np.abs(m[2]).max())
            print(json.dumps(out), flush=True)
            lat.close()
            # Sec. 9: heated slab, temperature wall at T0 (zero-flux density)
            # moving at v_w, adiabatic wall at rest; steady state
            for nx in (64, 128, 256):
                A = 13 * p["c1"] + 95 + 2 * p["E0"]
                h = A / 52
                q = 2e-3 * 2 * D * h / (T0 * nx * nx)
                xi = np.arange(nx) + 0.5
                exact = T0 + q * T0 / D / h * (nx * xi - xi ** 2 / 2)
                rises = {}
                for vw in (0.0, 0.02):
                    lat = lbm13.Lattice(nx, 4, p, W.heated_slab(T0, q, vw), precision=prec)
                    lat.set_state(1.0, 0.0, 0.0, T0)
                    lat.step(int(5 * nx * nx / D))
                    m = lat.macro()
                    rises[vw] = m[3].mean(axis=0) - T0
                    if vw == 0.0:
                        err = float(np.abs(m[3].mean(axis=0) - exact).max() / (exact.max() - T0))
                    else:
                        uy_err = float(np.abs(m[2].mean(axis=0) - vw * (1 - xi / nx)).max() / vw)
                    lat.close()
                extra = nu * (0.02 / nx) ** 2 / q
                phi_m = float((rises[0.02][nx // 2:].sum() / rises[0.0][nx // 2:].sum() - 1) / extra)
                print(json.dumps({"case": "heated_slab", "precision": name, "params": sname, "nx": nx, "q": q,
                                  "T_rel_err": err, "uy_rel_err": uy_err, "phi_measured": phi_m, "phi": phi}),
                      flush=True)


def run_serving(n, rate, side_min, side_max, ra_min, ra_max, tol, check_every, fp64_subset):
    """A Poisson trace of cavity and channel requests served with continuous
    batching (FP32-deviation), then the `fp64_subset` smallest cavity requests
    again in plain FP64, one lattice per launch, with the same stopping rule:
    the Nusselt-number difference states the served accuracy."""
    from . import serving as S
    reqs = S.poisson_trace(n, rate=rate, seed=5151, side_range=(side_min, side_max), ra_range=(ra_min, ra_max),
                           tol=tol)
    srv = S.Server(lbm13.FP32_DEVIATION, hbm_budget=120e9, max_slots=256, check_every=check_every, realtime=True)
    res, summary = srv.run(reqs)
    sides = [r.nx for r in res]
    print(json.dumps({"case": "serving", "requests": n, "rate_per_s": rate, "sides": [side_min, side_max],
                      "Ra": [ra_min, ra_max], "tol": tol, **summary,
                      "max_side_served": max(sides), "steps_max": max(r.steps for r in res)}), flush=True)
    cav = sorted([r for r in reqs if r.kind == "cavity"], key=lambda r: r.L)[:fp64_subset]
    base, _ = S.Server(lbm13.FP64, check_every=check_every, batched=False, realtime=False).run(cav)
    served = {r.rid: r for r in res}
    errs = [{"rid": b.rid, "L": b.nx, "Ra": b.Ra, "Nu_fp64": b.Nu, "Nu_fp32_served": served[b.rid].Nu,
             "abs_err": abs(served[b.rid].Nu - b.Nu)} for b in base]
    print(json.dumps({"case": "serving_nusselt_vs_fp64", "cavities": errs,
                      "max_abs_err": max(e["abs_err"] for e in errs)}), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("cavity")
    c.add_argument("--L", type=int, default=256)
    c.add_argument("--Ra", type=float, nargs="+", default=[1e3, 1e4, 1e5, 1e6])
    c.add_argument("--Pr", type=float, default=0.71)
    c.add_argument("--tol", type=float, default=1e-8)
    c.add_argument("--check-every", type=int, default=1000)
    c.add_argument("--max-steps", type=int, default=3_000_000)
    h = sub.add_parser("channels")
    h.add_argument("--nx", type=int, default=1024)
    h.add_argument("--ny", type=int, default=128)
    h.add_argument("--steps-factor", type=float, default=3.0)
    w = sub.add_parser("waves")
    w.add_argument("--precision", choices=["fp64", "fp32", "both"], default="both")
    v = sub.add_parser("serving")
    v.add_argument("--requests", type=int, default=64)
    v.add_argument("--rate", type=float, default=200.0)
    v.add_argument("--side-min", type=int, default=64)
    v.add_argument("--side-max", type=int, default=512)
    v.add_argument("--ra-min", type=float, default=1e3)
    v.add_argument("--ra-max", type=float, default=1e6)
    v.add_argument("--tol", type=float, default=1e-7)
    v.add_argument("--check-every", type=int, default=1000)
    v.add_argument("--fp64-subset", type=int, default=6)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    if a.cmd == "cavity":
        run_cavity(a.L, a.Ra, a.Pr, a.tol, a.check_every, a.max_steps)
    elif a.cmd == "channels":
        run_channels(a.nx, a.ny, a.steps_factor)
    elif a.cmd == "serving":
        run_serving(a.requests, a.rate, a.side_min, a.side_max, a.ra_min, a.ra_max, a.tol, a.check_every,
                    a.fp64_subset)
    else:
        precs = {"fp64": [lbm13.FP64], "fp32": [lbm13.FP32_DEVIATION],
                 "both": [lbm13.FP64, lbm13.FP32_DEVIATION]}[a.precision]
        run_waves(precs)


if __name__ == "__main__":
    main()
