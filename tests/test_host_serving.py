"""The serving admission loop on the CPU, with a stand-in backend (no GPU):
admission by the device-memory budget and the slot count, retirement at the
residual tolerance or on divergence, queueing under a simulated clock, and a
result that does not depend on the mix of requests it was served with."""
import math

import numpy as np
import pytest

from paper_1401_0188_gb300 import lbm13, serving as S


class _Live:
    bytes = 0
    peak_bytes = 0
    count = 0
    peak_count = 0


class FakeLattice:
    """Converges as exp(-t / tau) with tau set by the lattice size; the Nusselt
    read-out depends on the request only; `diverge_at` makes it report
    non-finite populations from that step on."""

    diverge_at = {}

    def __init__(self, nx, ny, p, bnd, precision):
        self.nx, self.ny, self.t, self.last = nx, ny, 0, None
        self.bytes = S.lattice_bytes(nx, ny, precision)
        self.tau = 40.0 * max(nx, ny)
        self.key = (nx, ny, round(p["nu"], 12))
        _Live.bytes += self.bytes
        _Live.count += 1
        _Live.peak_bytes = max(_Live.peak_bytes, _Live.bytes)
        _Live.peak_count = max(_Live.peak_count, _Live.count)

    def set_state(self, *a):
        self.t = 0

    def step(self, n):
        self.t += n

    def residual(self, raise_on_divergence=True):
        out = np.zeros(16)
        out[13] = 0 if self.last is None else self.t - self.last
        out[0] = math.exp(-self.t / self.tau)
        out[8] = 1.0 + 1e-3 * self.nx + self.key[2]
        out[12] = 1.0 if self.t >= FakeLattice.diverge_at.get(self.key, 1 << 62) else 0.0
        self.last = self.t
        return out

    def close(self):
        _Live.bytes -= self.bytes
        _Live.count -= 1


class FakePlan:
    shapes = []   # (shape, nodes in the plan, plan) at every set_config

    made = 0

    def __init__(self, lattices):
        self.lattices = list(lattices)
        FakePlan.made += 1
        self.serial = FakePlan.made

    def set_config(self, *a):
        FakePlan.shapes.append((a, sum(g.nx * g.ny for g in self.lattices), self.serial))

    def add(self, lat):
        assert all(g is not lat for g in self.lattices)
        self.lattices.append(lat)

    def remove(self, lat):
        # the last lattice takes the removed one's row, as in lbm13_plan_remove
        i = next(k for k, g in enumerate(self.lattices) if g is lat)
        self.lattices[i] = self.lattices[-1]
        self.lattices.pop()

    def step(self, n):
        for g in self.lattices:
            g.step(n)

    def residual(self, raise_on_divergence=True):
        return np.array([g.residual() for g in self.lattices])

    def close(self):
        pass


class Backend:
    Lattice = FakeLattice
    Plan = FakePlan


@pytest.fixture(autouse=True)
def _reset():
    _Live.bytes = _Live.peak_bytes = _Live.count = _Live.peak_count = 0
    FakeLattice.diverge_at = {}
    FakePlan.shapes = []
    yield


def _trace(n=12):
    return S.poisson_trace(n, rate=50.0, seed=5151, side_range=(64, 192), ra_range=(1e3, 1e5), tol=1e-3)


@pytest.mark.parametrize("batched", [True, False])
def test_admission_respects_budget_and_slots(batched):
    reqs = _trace()
    sizes = [S.lattice_bytes(*S.request_setup(r)[:2], lbm13.FP32_DEVIATION) for r in reqs]
    budget = 2.2 * max(sizes)
    srv = S.Server(lbm13.FP32_DEVIATION, hbm_budget=budget, max_slots=3, check_every=100, realtime=False,
                   batched=batched, backend=Backend)
    res, summary = srv.run(reqs)
    assert summary["requests"] == len(reqs) == summary["converged"]
    assert _Live.peak_bytes <= budget and _Live.peak_count <= 3
    assert _Live.bytes == 0 and _Live.count == 0
    assert [r.rid for r in res] == sorted(r.rid for r in reqs)
    assert all(r.admitted >= r.arrival and r.finished >= r.admitted for r in res)
    assert any(r.admitted > r.arrival for r in res)          # some waited for memory
    # retired at the first check that meets the tolerance: steps = check_every * ceil(tau ln(1/tol) / check_every)
    for r in res:
        tau = 40.0 * max(r.nx, r.ny)
        assert r.steps == 100 * math.ceil(tau * math.log(1e3) / 100)
        assert r.residual <= 1e-3
    assert summary["p99_tts_s"] >= summary["p50_tts_s"] > 0


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = _trace(8)
    srv = S.Server(lbm13.FP32_DEVIATION, hbm_budget=1e12, max_slots=4, check_every=100, realtime=False,
                   backend=Backend)
    mixed, _ = srv.run(reqs)
    for req, m in zip(reqs, mixed):
        alone, _ = S.Server(lbm13.FP32_DEVIATION, check_every=100, realtime=False, backend=Backend).run([req])
        a = alone[0]
        assert (a.steps, a.residual, a.Nu, a.converged) == (m.steps, m.residual, m.Nu, m.converged)


def test_divergence_retires_the_request_unconverged():
    reqs = _trace(4)
    keys = []
    for r in reqs:
        nx, ny, p, _ = S.request_setup(r)
        keys.append((nx, ny, round(p["nu"], 12)))
    i = next(k for k in range(len(reqs)) if keys.count(keys[k]) == 1)
    FakeLattice.diverge_at[keys[i]] = 300
    res, summary = S.Server(lbm13.FP32_DEVIATION, check_every=100, realtime=False, backend=Backend).run(reqs)
    bad = [r for r in res if r.rid == reqs[i].rid][0]
    assert not bad.converged and bad.steps == 300
    assert summary["converged"] == len(reqs) - 1


def test_request_above_the_budget_is_refused():
    reqs = _trace(2)
    with pytest.raises(ValueError):
        S.Server(lbm13.FP32_DEVIATION, hbm_budget=1000.0, check_every=100, realtime=False, backend=Backend).run(reqs)


def test_plan_shape_follows_the_node_count():
    """With plan_config "auto" the served plan takes the ring-staged strips
    while it holds 2^20 nodes or more and the one-row tile below that, set
    again whenever admission or retirement crosses the threshold."""
    reqs = S.poisson_trace(10, rate=50.0, seed=7, side_range=(256, 1024), ra_range=(1e3, 1e5), tol=1e-3)
    srv = S.Server(lbm13.FP32_DEVIATION, hbm_budget=1e12, max_slots=8, check_every=100, realtime=False,
                   backend=Backend)
    res, summary = srv.run(reqs)
    assert summary["converged"] == len(reqs)
    shapes = FakePlan.shapes
    assert shapes and all(a == (S.Server.LARGE_PLAN if n >= S.Server.LARGE_PLAN_NODES else S.Server.SMALL_PLAN)
                          for a, n, _ in shapes)
    assert {a for a, _, _ in shapes} == {S.Server.LARGE_PLAN, S.Server.SMALL_PLAN}
    # a plan is set again only when its shape changes
    assert all(x[0] != y[0] for x, y in zip(shapes, shapes[1:]) if x[2] == y[2])
    # a fixed shape is set once per plan and never changed
    FakePlan.shapes = []
    S.Server(lbm13.FP32_DEVIATION, hbm_budget=1e12, max_slots=8, check_every=100, realtime=False,
             backend=Backend, plan_config=(1, 4, 0, 2, 1)).run(reqs)
    assert {a for a, _, _ in FakePlan.shapes} == {(1, 4, 0, 2, 1)}
    assert len({p for _, _, p in FakePlan.shapes}) == len(FakePlan.shapes)
