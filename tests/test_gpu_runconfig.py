"""A JSON run description stepped end to end on the GPU: a small heated
cavity to a steady state, one JSON line per check."""
import json

import pytest


@pytest.mark.gpu
def test_description_runs_to_steady_state():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_0188_gb300 import build, runconfig as R
    build.build()
    desc = {"nx": 48, "ny": 40, "precision": "fp32", "params": {"nu": 0.1, "Pr": 0.71},
            "walls": {"west": {"kind": "mixed", "T_offset": 0.005}, "east": {"kind": "mixed", "T_offset": -0.005},
                      "south": {"kind": "bb"}, "north": {"kind": "bb"}},
            "force": {"gy": -2e-4, "rho_ref": 1.0}, "wall_density": "zero_flux",
            "steady": {"tol": 1e-6, "check_every": 500, "max_steps": 100000}}
    lines = []
    last = R.run(desc, emit=lines.append)
    rows = [json.loads(l) for l in lines]
    assert len(rows) >= 2 and rows[-1] == last
    assert last["converged"] and last["residual"] <= 1e-6
    assert [r["t"] for r in rows[:-1]] == [500 * (i + 1) for i in range(len(rows) - 1)]
    assert 0.99 < last["Nu"] < 3.0 and last["umax"] > 0
    assert all(r["MLUPS"] > 0 for r in rows[:-1])
