"""The second configuration at its own size: the Sec. 10 differentially heated
cavity on 256 x 256 at Ra = 1e3, 1e4, 1e5 (Pr = 0.71), run on the GPU against
the FP64 oracle's run of the same set-up to residual 1e-8
(tests/golden/cavity256_oracle.json, written by tests/golden/make_cavity256.py,
which calls the oracle only).

FP64: the same step count with the residual read at the same steps gives the
oracle's Nusselt number, asymmetries, max |u| and sampled fields.  FP32
deviation storage, run to its own residual of 1e-8, stays within the stated
bounds below of the oracle."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cavity256_oracle.json")
# stated bounds of FP32-deviation storage against the FP64 oracle at steady
# state (256^2 cavity, residual 1e-8)
FP32_BOUNDS = {"Nu": 1e-4, "S_u": 2e-5, "S_T": 2e-5, "u": 5e-6, "T": 5e-6}


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_0188_gb300 import build, lbm13
    build.build()
    lbm13.lib()
    return lbm13


def _run(L, g, run, precision, steps=None):
    lat = L.Lattice(g["L"], g["L"], run["params"], run["boundary"], precision=precision)
    lat.set_state(1.0, 0.0, 0.0, run["T0"])
    lat.residual()
    r = None
    while True:
        lat.step(g["check_every"])
        r = lat.residual()
        if (steps is not None and lat.t >= steps) or (steps is None and r[0] <= g["tol"]) or lat.t >= 3_000_000:
            break
    fields, t = lat.macro(), lat.t
    lat.close()
    return t, r, fields


def _samples(fields, run):
    out = []
    for y, x, ux, uy, T in run["samples_y_x_ux_uy_T"]:
        out.append((fields[1, y, x] - ux, fields[2, y, x] - uy, fields[3, y, x] - T))
    return np.array(out)


@pytest.mark.parametrize("i", [0, 1, 2])
def test_cavity256_fp64_matches_oracle(L, gold, i):
    run = gold["runs"][i]
    t, r, fields = _run(L, gold, run, L.FP64, steps=run["steps"])
    assert t == run["steps"]
    assert r[0] <= gold["tol"] * 1.001
    assert r[8] == pytest.approx(run["Nu"], rel=1e-9)
    assert r[9] == pytest.approx(run["S_u"], rel=1e-6, abs=1e-12)
    assert r[10] == pytest.approx(run["S_T"], rel=1e-6, abs=1e-12)
    assert r[11] == pytest.approx(run["umax"], rel=1e-9)
    assert np.abs(_samples(fields, run)).max() <= 1e-10


@pytest.mark.parametrize("i", [0, 1, 2])
def test_cavity256_fp32_deviation_within_stated_bounds(L, gold, i):
    run = gold["runs"][i]
    t, r, fields = _run(L, gold, run, L.FP32_DEVIATION)
    assert r[0] <= gold["tol"], "FP32-deviation storage reaches the residual of 1e-8"
    assert abs(r[8] - run["Nu"]) <= FP32_BOUNDS["Nu"]
    assert abs(r[9] - run["S_u"]) <= FP32_BOUNDS["S_u"]
    assert abs(r[10] - run["S_T"]) <= FP32_BOUNDS["S_T"]
    d = _samples(fields, run)
    assert np.abs(d[:, :2]).max() <= FP32_BOUNDS["u"]
    assert np.abs(d[:, 2]).max() <= FP32_BOUNDS["T"]
