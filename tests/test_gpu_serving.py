"""Continuous-batching server: requests admitted by memory budget and slots,
stepped together, retired at their tolerance.  Each result is bit-identical
to the same request served alone; FP32-deviation serving agrees with the plain
FP64 one-lattice-per-launch path and with the oracle within stated bounds."""
import os

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu
NTH = max(1, os.cpu_count() or 1)

# Stated bound on the served FP32-deviation Nusselt number against FP64.
NU_FP32 = 2e-4


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_0188_gb300 import build, serving
    build.build()
    return serving


def _trace(S):
    return S.poisson_trace(6, rate=50.0, seed=5151, side_range=(32, 64), ra_range=(1e3, 1e4), tol=1e-6)


@pytest.fixture(scope="module")
def served(S):
    from paper_1401_0188_gb300 import lbm13
    reqs = _trace(S)
    budget = 2.5 * max(S.lattice_bytes(*S.request_setup(r)[:2], lbm13.FP32_DEVIATION) for r in reqs)
    srv = S.Server(lbm13.FP32_DEVIATION, hbm_budget=budget, max_slots=3, check_every=500, realtime=False)
    return reqs, srv.run(reqs)


def test_all_requests_converge_with_queueing(S, served):
    reqs, (res, summary) = served
    assert summary["requests"] == len(reqs) and summary["converged"] == len(reqs)
    assert all(r.admitted >= r.arrival for r in res)
    assert summary["p99_tts_s"] >= summary["p50_tts_s"] > 0
    # the budget holds at most two lattices: some requests waited in the queue
    assert any(r.admitted > r.arrival + 1e-3 for r in res)


def test_each_result_is_the_same_alone_and_in_the_mix(S, served):
    from paper_1401_0188_gb300 import lbm13
    reqs, (res, _) = served
    for req, r in zip(reqs, res):
        alone, _ = S.Server(lbm13.FP32_DEVIATION, check_every=500, realtime=False).run([req])
        a = alone[0]
        assert (a.steps, a.residual, a.Nu, a.S_u, a.S_T, a.umax, a.rho_total) == \
               (r.steps, r.residual, r.Nu, r.S_u, r.S_T, r.umax, r.rho_total), req


def test_fp32_serving_against_fp64_baseline_and_oracle(S, served):
    from paper_1401_0188_gb300 import lbm13
    reqs, (res, _) = served
    base, summary = S.Server(lbm13.FP64, check_every=500, batched=False, realtime=False).run(reqs)
    assert summary["converged"] == len(reqs)
    for a, b in zip(res, base):
        if a.kind == "cavity":
            assert abs(a.Nu - b.Nu) <= NU_FP32, (a.rid, a.Nu, b.Nu)
        assert abs(a.umax - b.umax) <= 1e-6
    # the smallest cavity against the FP64 oracle at the same step count
    cav = [r for r in base if r.kind == "cavity"]
    if cav:
        r = min(cav, key=lambda r: r.nx)
        req = reqs[r.rid]
        nx, ny, p, bnd = S.request_setup(req)
        o = O.Lattice(nx, ny, p, bnd, nthreads=NTH)
        o.set_equilibrium(1.0, 0.0, 0.0, (p["E0"] + 28) / 26)
        o.residual()
        o.step(r.steps)
        ro = o.residual()
        assert r.Nu == pytest.approx(ro[8], rel=1e-9)
