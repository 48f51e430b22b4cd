"""Bounds-checked build (LBM13_DEBUG), the stand-in for a memory checker:
every population load and store of the step kernels is checked against its
lattice (plane, row and column in range) and counted when outside.  The
parity shapes (ragged, tiny, every wall kind, forcing, energy source) in both
storages, the persistent launch, paired steps of the periodic FP32 lattices,
and a plan stepped in every configuration (every tile shape including the
tensor-copy slabs and the ring-staged strips with their edge work items,
grids, orders, row groups) must make no access outside their lattices."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json
import numpy as np
import torch
from paper_1401_0188_gb300 import lbm13, params as P, workloads as W

p = P.pstar(0.05, 0.71)
T0 = P.rest_temperature(p)
M, B = W.WALL_MIXED, W.WALL_BB
hot, cold = T0 + 0.005, T0 - 0.005
cases = [
    (48, 40, W.cavity(T0, 0.01, 2e-4)), (37, 30, W.couette(T0, 0.05, 0.01)), (40, 33, W.poiseuille(1e-5)),
    (36, 36, W.boundary(west=W.wall(B), east=W.wall(B), south=W.wall(B), north=W.wall(B, 0.03))),
    (34, 29, W.boundary(west=W.wall(M, -0.01, hot), east=W.wall(M, 0.015, cold), south=W.wall(M, 0.02, T0),
                        north=W.wall(M, -0.01, hot))),
    (35, 33, W.boundary(west=W.wall(M, 0.01, hot), east=W.wall(B, -0.02))),
    (66, 20, W.boundary(west=W.wall(M, 0.0, hot), east=W.wall(M, 0.0, cold), south=W.wall(B, 0.03),
                        north=W.wall(B))),
    (45, 50, W.boundary(gx=2e-5, gy=-1e-5, rho_ref=0.0)),
    (4, 4, W.boundary(west=W.wall(M, 0.0, hot), east=W.wall(M, 0.0, cold), south=W.wall(B, 0.02),
                      north=W.wall(M, 0.0, T0))),
    (2, 3, W.boundary()), (100, 70, W.cavity(T0, 0.01, 1e-4)), (48, 40, W.cavity(T0, 0.01, 2e-4, wall_density=1)),
    (37, 30, W.couette(T0, 0.03, 0.01, wall_density=1)), (40, 24, W.heated_slab(T0, 1e-5, 0.02)),
    (130, 45, W.boundary(gx=1e-5, gy=-2e-5)), (200, 128, W.cavity(T0, 0.01, 1e-4, wall_density=1)),
    (1024, 8, W.boundary(south=W.wall(M, 0.01, hot), north=W.wall(B, -0.02), wall_density=1)),
    (600, 400, W.boundary(gx=1e-5, gy=-2e-5)),
]
lats = []
for prec in (lbm13.FP64, lbm13.FP32_DEVIATION):
    for nx, ny, bnd in cases:
        g = lbm13.Lattice(nx, ny, p, bnd, precision=prec)
        t = W.random_fields(nx, ny, T0, 7, du=0.01, drho=0.005, dT=0.003)
        g.set_state(*t)
        g.step(37)
        lats.append(g)
for g in lats[:6]:
    g.set_persistent(lbm13.PERSISTENT_ON)
    g.step(40)
fp32 = [g for g in lats if g.precision == lbm13.FP32_DEVIATION]
paired = 0
for g in fp32:
    # paired steps wherever the lattice takes them (periodic in x and y)
    g.set_pair_steps(lbm13.PAIR_ON)
    paired += g.step_launches(41) < 41
    g.step(41)
    g.set_pair_steps(lbm13.PAIR_AUTO)
plan = lbm13.Plan(fp32)
configs = 0
for R, BY in ((1, 4), (2, 4), (4, 4), (2, 2), (1, 8)):
    for ctas in (0, 8):
        for order in (0, 1, 2):
            for groups in (1, 3):
                plan.set_config(R, BY, ctas, order, groups)
                plan.step(2)
                configs += 1
for BY in (8, 4):  # ring-staged strips and their edge work items
    for order in (0, 2):
        for groups in (1, 3, 16):
            plan.set_config(0, BY, 0, order, groups)
            plan.step(2)
            configs += 1
plan.step(33)
plan.residual()
plan.close()
torch.cuda.synchronize()
print(json.dumps({"lattices": len(lats), "configs": configs, "paired": paired,
                  "violations": sum(g.debug_violations() for g in lats)}))
"""


@pytest.mark.gpu
def test_step_kernels_stay_inside_the_lattice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_0188_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, LBM13_DEBUG_BUILD="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["lattices"] == 36 and d["configs"] == 72 and d["paired"] >= 3
    assert d["violations"] == 0, d
