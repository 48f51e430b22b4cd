"""Persistent multi-step launches: many steps per cooperative launch with grid
barriers between the phases of a step.  They must give bit-identical states to
per-step launches for every wall kind, both storages, odd and even step
counts and runs longer than one launch; the barrier's bounded wait must run
out (and leave the context usable) when the barrier cannot complete."""
import zlib

import numpy as np
import pytest

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


def _T0(p):
    return (p["E0"] + 28.0) / 26.0


def _cases(T0):
    hot, cold = T0 + 0.005, T0 - 0.005
    B, M = W.WALL_BB, W.WALL_MIXED
    return {
        "periodic": (64, 40, W.boundary()),
        "periodic_forced_heated": (45, 50, W.boundary(gx=2e-5, gy=-1e-5, rho_ref=0.0, heat=2e-6)),
        "cavity": (48, 40, W.cavity(T0, 0.01, 2e-4)),
        "cavity_zero_flux": (100, 70, W.cavity(T0, 0.01, 1e-4, wall_density=1)),
        "couette": (37, 30, W.couette(T0, 0.03, 0.01)),
        "lid_driven": (36, 36, W.boundary(west=W.wall(B), east=W.wall(B), south=W.wall(B), north=W.wall(B, 0.03))),
        "all_mixed_moving": (34, 29, W.boundary(west=W.wall(M, -0.01, hot), east=W.wall(M, 0.015, cold),
                                                south=W.wall(M, 0.02, T0), north=W.wall(M, -0.01, hot),
                                                gx=1e-5, gy=-2e-5, rho_ref=1.0)),
        "heated_slab": (40, 24, W.heated_slab(T0, 1e-5, 0.02)),
        "tiny_walls": (4, 4, W.boundary(west=W.wall(M, 0.0, hot), east=W.wall(M, 0.0, cold),
                                        south=W.wall(B, 0.02), north=W.wall(M, 0.0, T0))),
        "wide": (300, 20, W.cavity(T0, 0.01, 1e-4)),
    }


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", list(_cases(0.576).keys()))
def test_persistent_equals_per_step_launches(L, pstar, case, precision):
    T0 = _T0(pstar)
    nx, ny, bnd = _cases(T0)[case]
    fields = W.random_fields(nx, ny, T0, seed=zlib.crc32(case.encode()) % 1000, du=0.01, drho=0.005, dT=0.003)
    a = L.Lattice(nx, ny, pstar, bnd, precision=precision)
    b = L.Lattice(nx, ny, pstar, bnd, precision=precision)
    a.set_persistent(L.PERSISTENT_ON)
    b.set_persistent(L.PERSISTENT_OFF)
    for g in (a, b):
        g.set_state(*fields)
    for n in (1, 37, 64, 3):
        a.step(n)
        b.step(n)
        assert a.t == b.t
        assert a.save() == b.save(), (case, n)
    assert a.info()["persistent_grid"] > 0
    ra, rb = a.residual(), b.residual()
    assert np.array_equal(ra, rb)


def test_persistent_runs_longer_than_one_launch(L, pstar):
    """2,100 steps: three launches of at most 1,024 steps, the last one odd."""
    T0 = _T0(pstar)
    bnd = W.cavity(T0, 0.01, 2e-4, wall_density=1)
    a = L.Lattice(64, 48, pstar, bnd, precision=L.FP32_DEVIATION)
    b = L.Lattice(64, 48, pstar, bnd, precision=L.FP32_DEVIATION)
    a.set_persistent(L.PERSISTENT_ON)
    b.set_persistent(L.PERSISTENT_OFF)
    for g in (a, b):
        g.set_state(1.0, 0.0, 0.0, T0)
    a.step(2100)
    b.step(2100)
    assert a.save() == b.save()


def test_modes(L, pstar):
    """AUTO (the default) steps launch by launch; ON takes the persistent
    launch (its grid size is reported once chosen); other modes are refused."""
    g = L.Lattice(256, 256, pstar, precision=L.FP32_DEVIATION)
    g.step(4)
    assert g.info()["persistent_grid"] == 0
    g.set_persistent(L.PERSISTENT_ON)
    g.step(4)
    assert g.info()["persistent_grid"] > 0
    with pytest.raises(L.Lbm13Error):
        g.set_persistent(7)


def test_barrier_wait_is_bounded(L, pstar):
    """A barrier over the whole grid completes; one that waits for a block
    that was never launched runs out after its timeout, reports it, and the
    context stays usable."""
    assert L.barrier_check(8, 0, 0.05) is False
    assert L.barrier_check(8, 1, 0.05) is True
    assert L.barrier_check(1, 3, 0.01) is True
    g = L.Lattice(32, 32, pstar)
    g.step(10)
    g.synchronize()
    assert g.t == 10
    with pytest.raises(L.Lbm13Error):
        L.barrier_check(8, 0, 5.0)
