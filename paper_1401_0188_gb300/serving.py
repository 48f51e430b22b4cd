"""Continuous-batching solve server for cavity and channel requests.

Requests arrive over time (a seeded Poisson stream).  A request is admitted
when a slot is free and its lattice fits in the device-memory budget; from then
on its populations stay on the device and it is stepped together with every
other admitted request in one batched launch per time step (one plan over the
active lattices).  Rounds of `check_every` steps are launched asynchronously;
while a round runs on the GPU, requests that arrive are admitted on the host
and their lattices created and initialised on a second CUDA stream, so that
their set-up overlaps the round.  At the end of the round the FP64 residuals
of all active lattices are read back in one synchronisation; a request retires
when its residual reaches its tolerance (lbm13_plan_remove, freeing its slot
and memory for the queue) and the newly admitted lattices join the plan
(lbm13_plan_add) for the next round.  Admission and retirement take effect
only between rounds, so each request sees the same sequence of steps and
checks whether it runs alone or in a mix: its result does not depend on the
mix.

The baseline mode steps each lattice with its own launches in FP64 (the plain
one-lattice-per-launch path), with the same admission and checks.
"""
import math
import time
from dataclasses import dataclass

import numpy as np

from . import lbm13, params as P, workloads as W


@dataclass
class Request:
    rid: int
    kind: str          # "cavity" or "channel"
    L: int             # cavity side, or channel length (height L/4)
    Ra: float = 1e4    # cavity Rayleigh number
    Pr: float = 0.71
    tol: float = 1e-7
    arrival: float = 0.0   # seconds after the start of the run


@dataclass
class Result:
    rid: int
    kind: str
    nx: int
    ny: int
    Ra: float
    Pr: float
    arrival: float
    admitted: float
    finished: float
    steps: int
    converged: bool
    residual: float
    Nu: float
    S_u: float
    S_T: float
    umax: float
    rho_total: float
    tts: float          # time to steady state: finished - arrival (queueing included)


def request_setup(req):
    """(nx, ny, params, boundary) of a request."""
    if req.kind == "cavity":
        nu = 0.05 * req.L * math.sqrt(req.Pr / req.Ra)
        nu = min(P.stable_viscosity(nu, req.Pr), 0.35)
        p = P.select(nu, req.Pr)
        T0 = P.rest_temperature(p)
        kappa = nu / req.Pr
        g = req.Ra * nu * kappa * T0 / (0.01 * req.L ** 3)
        return req.L, req.L, p, W.cavity(T0, 0.01, g, rho_ref=1.0, wall_density=1)
    # Poiseuille channel with temperature walls (Sec. 8): u_max = 0.02 at nu = 0.1
    ny = max(16, req.L // 4)
    p = P.select(0.1, req.Pr)
    T0 = P.rest_temperature(p)
    g = 8 * 0.1 * 0.02 / ny ** 2
    return req.L, ny, p, W.poiseuille(g, T0=T0, dT=0.01, wall_density=1)


def lattice_bytes(nx, ny, precision):
    """Device bytes a request holds: two population buffers and the FP64
    reduction buffers (six fields plus per-block partial sums, an upper
    bound on the library's block count)."""
    elem = 8 if precision == lbm13.FP64 else 4
    pitch = (nx + 31) // 32 * 32
    return 2 * 13 * elem * pitch * ny + 8 * (6 * nx * ny + 1216 * 16 + 32)


def poisson_trace(n, rate, seed=5151, side_range=(64, 192), ra_range=(1e3, 1e5), Pr=0.71, tol=1e-7,
                  pr_range=None):
    """n requests, exponential inter-arrival times of mean 1/rate, alternating
    cavity/channel (50/50), side log-uniform in side_range rounded to a
    multiple of 32, Ra log-uniform in ra_range; Pr fixed, or uniform in
    pr_range when given.  Each request draws its values in turn, so the first
    k requests of a longer trace are the trace of k requests."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    t = 0.0
    for i in range(n):
        t += float(g.exponential(1.0 / rate))
        side = int(round(math.exp(g.uniform(math.log(side_range[0]), math.log(side_range[1]))) / 32) * 32)
        ra = math.exp(g.uniform(math.log(ra_range[0]), math.log(ra_range[1])))
        pr = float(g.uniform(*pr_range)) if pr_range is not None else Pr
        kind = "cavity" if i % 2 == 0 else "channel"
        out.append(Request(i, kind, max(32, side), ra, pr, tol, t))
    return out


@dataclass
class _Active:
    req: Request
    lat: object
    nx: int
    ny: int
    bytes: int
    admitted: float
    steps: int = 0


class Server:
    """`backend` provides Lattice and Plan (the CUDA binding by default; the
    CPU tests of the admission logic pass a stand-in).  With `overlap` (and
    the CUDA backend), new lattices are set up on a second stream while the
    current round runs."""

    # tile shapes of the served plan, (R, BY, ctas_per_sm, order, groups): the
    # one-row register tile while the plan is small, the 32-column ring-staged
    # strips of 16 four-row groups once it holds LARGE_PLAN_NODES nodes or more
    # (measured faster there, slower on a trace of lattices up to 192^2; on the
    # fifth configuration's first 16 requests p99 19.2 s with 16 groups, 20.8 s
    # with 8, the strips' best segment before their edge nodes became work
    # items of their own); both give bit-identical steps
    SMALL_PLAN = (1, 4, 0, 2, 1)
    LARGE_PLAN = (0, 4, 0, 0, 16)
    LARGE_PLAN_NODES = 1 << 20

    def __init__(self, precision=lbm13.FP32_DEVIATION, hbm_budget=120e9, max_slots=256, check_every=1000,
                 max_steps=2_000_000, batched=True, realtime=True, backend=lbm13, plan_config="auto",
                 overlap=True, poll_s=0.0002):
        # plan_config: (R, BY, ctas_per_sm, order, groups) of the batched step,
        # or "auto" (by the plan's node count, see SMALL_PLAN / LARGE_PLAN)
        self.plan_config = plan_config if plan_config == "auto" else tuple(plan_config)
        self.backend = backend
        self.precision = precision
        self.hbm_budget = hbm_budget
        self.max_slots = max_slots
        self.check_every = check_every
        self.max_steps = max_steps
        self.batched = batched
        self.realtime = realtime
        self.overlap = overlap
        self.poll_s = poll_s

    def run(self, requests):
        pending = sorted(requests, key=lambda r: r.arrival)
        active, results = [], []
        self._used = 0
        plan = None
        t0 = time.perf_counter()
        self._clock_offset = 0.0
        now = lambda: time.perf_counter() - t0 + self._clock_offset
        side = None
        if self.batched and self.overlap and self.backend is lbm13:
            import torch
            side = torch.cuda.Stream()
        lattice_steps = 0
        joining = []     # admitted during the current round: join the next one
        shape, changed = None, False   # the plan's tile shape; membership changed since set
        while pending or active or joining:
            # newly admitted lattices join the plan for this round
            changed = changed or bool(joining)
            for a in joining:
                if self.batched and plan is not None:
                    plan.add(a.lat)
                active.append(a)
            if self.batched and joining and plan is None:
                plan = self.backend.Plan([a.lat for a in active])
                shape = None
            joining = []
            if self.batched and plan is not None and (changed or shape is None):
                want = self._shape(active)
                if want != shape:
                    plan.set_config(*want)
                    shape = want
            changed = False
            if not active:
                joining = self._admit(pending, active, joining, now, side)
                if not joining:
                    wait = pending[0].arrival - now()
                    if wait > 0:
                        if self.realtime:
                            time.sleep(wait)
                        else:
                            self._clock_offset += wait
                continue
            if self.batched:
                plan.step(self.check_every)
                done_ev = self._record(plan)
                # admit arrivals while the round runs (set-up on the side stream)
                while True:
                    joining = self._admit(pending, active, joining, now, side)
                    if done_ev is None or not self.realtime or done_ev.query():
                        break
                    wait = pending[0].arrival - now() if pending else None
                    if wait is None or wait <= 0:
                        # nothing left to admit, or arrivals held back by the
                        # slots or the budget until a retirement: wait for the round
                        done_ev.synchronize()
                        break
                    time.sleep(min(self.poll_s, wait))
                res = plan.residual(raise_on_divergence=False)
            else:
                for a in active:
                    a.lat.step(self.check_every)
                res = np.array([a.lat.residual(raise_on_divergence=False) for a in active])
                joining = self._admit(pending, active, joining, now, side)
            lattice_steps += self.check_every * sum(a.nx * a.ny for a in active)
            keep = []
            for a, r in zip(list(plan.lattices if self.batched else [a.lat for a in active]), res):
                a = next(x for x in active if x.lat is a)
                a.steps += self.check_every
                done = (r[13] > 0 and r[0] <= a.req.tol) or a.steps >= self.max_steps or r[12] > 0
                if done:
                    t = now()
                    results.append(Result(a.req.rid, a.req.kind, a.nx, a.ny, a.req.Ra, a.req.Pr, a.req.arrival,
                                          a.admitted, t, a.steps, bool(r[13] > 0 and r[0] <= a.req.tol),
                                          float(r[0]), float(r[8]), float(r[9]), float(r[10]), float(r[11]),
                                          float(r[4]), t - a.req.arrival))
                    if self.batched:
                        if len(plan.lattices) > 1:
                            plan.remove(a.lat)
                        else:
                            plan.close()
                            plan = None
                        shape = None if plan is None else shape
                        changed = True
                    a.lat.close()
                    self._used -= a.bytes
                else:
                    keep.append(a)
            active = keep
        if plan is not None:
            plan.close()
        wall = now()
        tts = np.array([r.tts for r in results])
        summary = {"requests": len(results), "converged": int(sum(r.converged for r in results)),
                   "wall_s": wall, "p50_tts_s": float(np.percentile(tts, 50)), "p99_tts_s": float(np.percentile(tts, 99)),
                   "throughput_req_s": len(results) / wall, "MLUPS": lattice_steps / wall / 1e6,
                   "precision": "fp64" if self.precision == lbm13.FP64 else "fp32-deviation",
                   "batched": self.batched, "overlap": side is not None}
        return sorted(results, key=lambda r: r.rid), summary

    def _shape(self, active):
        if self.plan_config != "auto":
            return self.plan_config
        nodes = sum(a.nx * a.ny for a in active)
        return self.LARGE_PLAN if nodes >= self.LARGE_PLAN_NODES else self.SMALL_PLAN

    def _record(self, plan):
        """An event after the round just launched (None for stand-in plans)."""
        stream = getattr(plan, "stream", None)
        if stream is None or self.backend is not lbm13:
            return None
        import torch
        ev = torch.cuda.Event()
        ev.record(stream)
        return ev

    def _admit(self, pending, active, joining, now, side):
        """Admit the requests that have arrived, as slots and the budget allow;
        their lattices start at rest with a residual snapshot."""
        while pending and pending[0].arrival <= now() and len(active) + len(joining) < self.max_slots:
            nx, ny, p, bnd = request_setup(pending[0])
            b = lattice_bytes(nx, ny, self.precision)
            if self._used + b > self.hbm_budget:
                if not active and not joining:
                    raise ValueError(f"request {pending[0].rid} needs {b} bytes, above the budget")
                break
            req = pending.pop(0)
            if side is not None:
                lat = self.backend.Lattice(nx, ny, p, bnd, precision=self.precision, stream=side)
            else:
                lat = self.backend.Lattice(nx, ny, p, bnd, precision=self.precision)
            lat.set_state(None, None, None, None)  # rest: rho 1, u 0, T T0
            lat.residual()
            joining.append(_Active(req, lat, nx, ny, b, now()))
            self._used += b
        return joining


def batch_workload(n=256, seed=4242, sides=(64, 96, 128, 192, 256, 384, 512), ra_range=(1e3, 1e6),
                   pr_range=(0.5, 1.0)):
    """The batched workload: n cavities, side uniform from `sides`, Ra
    log-uniform, Pr uniform; each with a parameter set that scans stable at its
    viscosity (raised to the smallest stable one where needed)."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        L = int(g.choice(sides))
        ra = math.exp(g.uniform(math.log(ra_range[0]), math.log(ra_range[1])))
        pr = float(g.uniform(*pr_range))
        out.append(Request(i, "cavity", L, ra, pr))
    return out
