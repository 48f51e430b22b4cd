"""Batched stepping (plans): many uneven lattices in one launch per step give
results bit-identical to the same lattices stepped alone, for every tile
shape, grid size and tile order the autotuner can pick."""
import numpy as np
import pytest

from paper_1401_0188_gb300 import pstar as product_pstar
from paper_1401_0188_gb300 import slabs
from paper_1401_0188_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_0188_gb300 import build, lbm13
    build.build()
    lbm13.lib()
    return lbm13


def _specs():
    out = []
    for i, (nx, ny, kind, nu, Pr) in enumerate([
            (64, 64, "cavity", 0.05, 0.71), (96, 70, "cavity", 0.03, 0.6), (37, 30, "couette", 0.05, 0.71),
            (40, 33, "poiseuille", 0.08, 0.8), (130, 45, "periodic", 0.02, 0.5), (4, 4, "box", 0.05, 0.71),
            (200, 128, "cavity", 0.1, 0.9), (33, 257, "cavity", 0.04, 0.55), (48, 20, "slab", 0.05, 0.71),
            (96, 40, "slab_halos", 0.05, 0.71), (70, 36, "cavity_halo", 0.05, 0.71)]):
        p = product_pstar(nu, Pr)
        T0 = (p["E0"] + 28) / 26
        bnd = {"cavity": W.cavity(T0, 0.01, 1e-4), "couette": W.couette(T0, 0.02, 0.01),
               "poiseuille": W.poiseuille(1e-5), "periodic": W.boundary(gx=1e-5, gy=-2e-5),
               "box": W.boundary(west=W.wall(W.WALL_BB), east=W.wall(W.WALL_BB), south=W.wall(W.WALL_BB),
                                 north=W.wall(W.WALL_BB, 0.02)),
               "slab": W.heated_slab(T0, 2e-6, 0.01),
               # y-slabs of a decomposed lattice: halo rows on both sides, or
               # below a walled top (halo rows are never stepped)
               "slab_halos": slabs.slab_boundary(W.poiseuille(1e-5), True, True),
               "cavity_halo": slabs.slab_boundary(W.cavity(T0, 0.01, 1e-4), True, False)}[kind]
        out.append((nx, ny, p, bnd, W.random_fields(nx, ny, T0, seed=100 + i, du=0.01, drho=0.005, dT=0.003)))
    return out


def _twins(L, precision):
    """Two identical sets of lattices; lattice i is pre-stepped i % 3 times so
    buffer parities differ across the plan."""
    a, b = [], []
    for i, (nx, ny, p, bnd, fields) in enumerate(_specs()):
        for group in (a, b):
            g = L.Lattice(nx, ny, p, bnd, precision=precision)
            g.set_state(*fields)
            g.step(i % 3)
            group.append(g)
    return a, b


def _same(a, b):
    for x, y in zip(a, b):
        assert x.t == y.t
        assert x.save() == y.save()


@pytest.mark.parametrize("precision", [0, 1])
def test_plan_equals_lattices_stepped_alone(L, precision):
    a, b = _twins(L, precision)
    plan = L.Plan(a)
    plan.step(37)       # one 32-step graph + 5 single launches
    for g in b:
        g.step(37)
    _same(a, b)
    plan.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_every_configuration_is_bit_identical(L, precision):
    a, b = _twins(L, precision)
    plan = L.Plan(a)
    for R, BY in ((1, 4), (2, 4), (4, 4), (2, 2), (1, 8)):
        for ctas in (0, 1, 8):
            for order in (0, 1, 2):
                for groups in (1, 3, 16):
                    plan.set_config(R, BY, ctas, order, groups)
                    c = plan.config()
                    assert (c["R"], c["BY"], c["ctas_per_sm"], c["order"], c["groups"]) == (R, BY, ctas, order,
                                                                                              groups)
                    plan.step(3)
                    for g in b:
                        g.step(3)
    if precision == 1:
        # ring-staged strips: segments of 1 to 64 four-row groups (one group,
        # shorter and longer than the six-slot ring, and a whole lattice)
        for BY in (8, 4):  # strips of 64 and 32 columns
            for order in (0, 1, 2):
                for groups in (1, 2, 5, 6, 7, 16, 64):
                    plan.set_config(0, BY, 0, order, groups)
                    plan.step(3)
                    for g in b:
                        g.step(3)
    else:
        with pytest.raises(L.Lbm13Error):
            plan.set_config(0, 8, 0, 0, 16)
    _same(a, b)
    plan.close()


@pytest.mark.parametrize("precision,shape", [(0, (1, 4, 0, 2, 4)), (1, (1, 4, 0, 2, 4)), (1, (0, 8, 0, 2, 16)),
                                             (1, (0, 4, 0, 2, 16))])
def test_admit_and_retire_keep_lattices_bit_identical(L, precision, shape):
    """lbm13_plan_add / lbm13_plan_remove: lattices join one at a time (past
    the table's first capacity, at different buffer parities, one just
    re-initialised on its own stream), leave from the middle, the end and the
    front, and step alone afterwards; every lattice stays bit-identical to its
    twin stepped alone, and residual rows follow the plan's order."""
    import torch
    a, b = _twins(L, precision)
    side = torch.cuda.Stream()
    plan = L.Plan(a[:2])
    plan.set_config(*shape)
    inside = [0, 1]
    plan.step(5)
    for k in inside:
        b[k].step(5)
    for k in range(2, len(a)):
        if k == 5:
            # set up on another stream right before joining: the plan's launches
            # must wait for it
            a[k].set_stream(side)
            b[k].set_stream(side)
            fields = _specs()[k][4]
            a[k].set_state(*fields)
            b[k].set_state(*fields)
        plan.add(a[k])
        inside.append(k)
        plan.step(3)
        for j in inside:
            b[j].step(3)
    assert [id(g) for g in plan.lattices] == [id(a[k]) for k in inside]
    for victim in (4, len(a) - 1, 0):
        plan.remove(a[victim])
        inside.remove(victim)
        plan.step(33)  # one 32-step graph and one launch
        for j in inside:
            b[j].step(33)
        a[victim].step(2)  # alone again, on its own stream
        b[victim].step(2)
    r = plan.residual()
    assert [int(row[14]) for row in r] == [g.t for g in plan.lattices]
    torch.cuda.synchronize()
    _same(a, b)
    with pytest.raises(L.Lbm13Error):
        plan.add(plan.lattices[0])  # already in the plan
    with pytest.raises(L.Lbm13Error):
        plan.remove(a[0])  # not in the plan
    plan.close()


def test_ring_strips_on_large_and_periodic_lattices(L):
    """The ring-staged strips over lattices wider and taller than one strip
    segment (interior nodes from the staged chunks, edges from global loads),
    with walls, a body force and periodic sides, through 32-step graphs."""
    specs = []
    for i, (nx, ny, kind) in enumerate([(300, 260, "cavity"), (257, 131, "periodic"), (128, 640, "couette"),
                                        (64, 64, "cavity"), (520, 96, "poiseuille"), (70, 400, "periodic")]):
        p = product_pstar(0.05, 0.71)
        T0 = (p["E0"] + 28) / 26
        bnd = {"cavity": W.cavity(T0, 0.01, 1e-4), "couette": W.couette(T0, 0.02, 0.01),
               "poiseuille": W.poiseuille(1e-5), "periodic": W.boundary(gx=1e-5, gy=-2e-5)}[kind]
        specs.append((nx, ny, p, bnd, W.random_fields(nx, ny, T0, seed=300 + i, du=0.01, drho=0.005, dT=0.003)))
    a, b = [], []
    for i, (nx, ny, p, bnd, fields) in enumerate(specs):
        for group in (a, b):
            g = L.Lattice(nx, ny, p, bnd, precision=1)
            g.set_state(*fields)
            g.step(i % 2)
            group.append(g)
    plan = L.Plan(a)
    for BY in (8, 4):
        for groups in (3, 16, 32):
            plan.set_config(0, BY, 0, 2, groups)
            plan.step(35)
            for g in b:
                g.step(35)
            _same(a, b)
    plan.close()


@pytest.mark.parametrize("shape", [(4, 4, 1), (0, 8, 16), (0, 4, 16)])
def test_staged_tile_wait_is_bounded(L, shape):
    """The staged (tensor-copy) tiles -- slabs and ring-staged strips -- wait on
    mbarriers with a time limit: with the copies withheld every wait runs out,
    the error word is set and read back, and nothing is written; with the
    copies issued no wait runs out; the plan then steps on, bit-identical to
    lattices stepped alone."""
    a, b = _twins(L, 1)
    plan = L.Plan(a)
    plan.set_config(shape[0], shape[1], 0, 2, shape[2])
    before = [g.save() for g in a]
    assert plan.tma_check(0.02, withhold=True) is True
    assert [g.save() for g in a] == before
    assert plan.tma_check(0.5, withhold=False) is False
    plan.step(5)
    for g in b:
        g.step(5)
    _same(a, b)
    plan.close()


def test_tune_then_step(L):
    a, b = _twins(L, 1)
    plan = L.Plan(a)
    t0 = a[0].t
    best = plan.tune(2)
    c = plan.config()
    assert best > 0 and c["tried"] == 204  # 180 register/slab tiles + 24 ring-staged strips
    taken = a[0].t - t0
    assert taken == c["tried"] * 3
    plan.step(40)
    for g in b:
        g.step(taken + 40)
    _same(a, b)
    plan.close()


def test_plan_follows_steps_taken_outside(L):
    a, b = _twins(L, 0)
    plan = L.Plan(a)
    plan.step(5)
    a[2].step(1)          # parity of one lattice changes behind the plan's back
    a[5].set_state(*_specs()[5][4])
    b[5].set_state(*_specs()[5][4])
    plan.step(4)
    for i, g in enumerate(b):
        g.step(5 + 4 + (1 if i == 2 else 0) if i != 5 else 4)
    _same(a, b)
    plan.close()


def test_plan_rejects_bad_lattice_lists(L):
    p = product_pstar()
    x = L.Lattice(16, 16, p)
    y = L.Lattice(16, 16, p, precision=L.FP32_DEVIATION)
    with pytest.raises(L.Lbm13Error):
        L.Plan([x, y])
    with pytest.raises(L.Lbm13Error):
        L.Plan([x, x])
    plan = L.Plan([x])
    with pytest.raises(L.Lbm13Error):
        plan.set_config(3, 4, 8, 0)
    with pytest.raises(L.Lbm13Error):
        plan.set_config(1, 4, 8, 0, 0)
    with pytest.raises(L.Lbm13Error):
        plan.step(-1)
    plan.close()


def test_full_batched_workload(L):
    """The bench's batched workload at full size: 256 cavities (19.7 M nodes,
    sides 64..512, Ra 1e3..1e6, Pr 0.5..1.0, FP32-deviation) in the
    configuration the autotuner picks on GB300 (one row per thread, 4 warps, one
    block per tile, largest lattice first, 4 row groups).  After 6 steps from
    rest every lattice is bit-identical to the same lattice stepped alone, and
    the first 64 x 64 cavity agrees with the FP64 oracle within the FP32 bounds."""
    import os
    import torch
    from oracle import oracle as O
    from paper_1401_0188_gb300 import serving as S
    reqs = S.batch_workload(256)
    setups = [S.request_setup(r) for r in reqs]

    def make():
        out = []
        for nx, ny, p, bnd in setups:
            g = L.Lattice(nx, ny, p, bnd, precision=L.FP32_DEVIATION)
            g.set_state(1.0, 0.0, 0.0, (p["E0"] + 28) / 26)
            out.append(g)
        return out

    a = make()
    plan = L.Plan(a)
    plan.set_config(1, 4, 0, 2, 4)
    plan.step(6)
    plan_state = [g.save() for g in a]
    plan.close()
    for g in a:
        g.close()
    del a
    torch.cuda.empty_cache()
    b = make()
    for g in b:
        g.step(6)
    assert all(g.save() == s for g, s in zip(b, plan_state))
    i = next(k for k, (nx, ny, _, _) in enumerate(setups) if nx == 64)
    nx, ny, p, bnd = setups[i]
    o = O.Lattice(nx, ny, p, bnd, nthreads=max(1, os.cpu_count() or 1))
    o.set_equilibrium(1.0, 0.0, 0.0, (p["E0"] + 28) / 26)
    o.step(6)
    mo, mg = o.macro(), b[i].macro()
    assert np.abs(mo - mg).max() <= 1e-7
    for g in b:
        g.close()
