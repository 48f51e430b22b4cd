"""Paired steps (two time steps per launch for FP32-deviation lattices periodic
in x and y): bit-identical to single steps for every lattice shape (tiles
clear of the periodic seam through the tensor copy, tiles across it through
wrapped loads, lattices smaller than one tile, ragged edges, and lattices
with more tiles than SMs, whose blocks alternate input buffers), with and
without a body force and an energy source, for odd and even step counts and
through the 32-step graphs; the bounded wait reports when its copy is
withheld; walled, slab and FP64 lattices keep one launch per step."""
import numpy as np
import pytest

from paper_1401_0188_gb300 import pstar as product_pstar
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


def _pair(L, nx, ny, bnd, seed):
    p = product_pstar(0.05, 0.71)
    T0 = (p["E0"] + 28) / 26
    fields = W.random_fields(nx, ny, T0, seed=seed, du=0.01, drho=0.005, dT=0.003)
    a = L.Lattice(nx, ny, p, bnd, precision=L.FP32_DEVIATION)
    b = L.Lattice(nx, ny, p, bnd, precision=L.FP32_DEVIATION)
    a.set_pair_steps(L.PAIR_ON)
    b.set_pair_steps(L.PAIR_OFF)
    a.set_state(*fields)
    b.set_state(*fields)
    return a, b


@pytest.mark.parametrize("nx,ny", [(256, 128), (200, 90), (40, 24), (24, 20), (8, 6), (64, 33), (33, 64), (600, 400),
                                   (1000, 310)])
@pytest.mark.parametrize("kind", ["plain", "force", "heat"])
def test_paired_steps_equal_single_steps(L, nx, ny, kind):
    bnd = {"plain": W.boundary(), "force": W.boundary(gx=1e-5, gy=-2e-5),
           "heat": W.boundary(gx=3e-6, heat=2e-6)}[kind]
    a, b = _pair(L, nx, ny, bnd, seed=nx * 7 + ny)
    assert a.step_launches(2) == 1 and a.step_launches(7) == 4 and a.step_launches(64) == 32
    assert b.step_launches(7) == 7
    for n in (2, 1, 7, 40, 67):
        a.step(n)
        b.step(n)
        assert a.t == b.t
        assert a.save() == b.save(), (nx, ny, kind, a.t)
    a.close()
    b.close()


def test_paired_wait_is_bounded(L):
    """The staged tiles' tensor-copy wait: withheld, every wait runs out, the
    error word is read back and nothing of the state changes; issued, no wait
    runs out; stepping then goes on bit-identical."""
    a, b = _pair(L, 256, 128, W.boundary(), seed=5)
    before = a.save()
    assert a.pair_check(0.02, withhold=True) is True
    assert a.save() == before
    assert a.pair_check(0.5, withhold=False) is False
    a.step(10)
    b.step(10)
    assert a.save() == b.save()
    a.close()
    b.close()


def test_walled_slab_and_fp64_lattices_step_singly(L):
    p = product_pstar(0.05, 0.71)
    T0 = (p["E0"] + 28) / 26
    from paper_1401_0188_gb300 import slabs
    for bnd, prec in ((W.cavity(T0, 0.01, 1e-4), L.FP32_DEVIATION), (W.poiseuille(1e-5), L.FP32_DEVIATION),
                      (slabs.slab_boundary(W.boundary(), True, True), L.FP32_DEVIATION), (W.boundary(), L.FP64)):
        g = L.Lattice(64, 40, p, bnd, precision=prec)
        g.set_pair_steps(L.PAIR_ON)
        assert g.step_launches(10) == 10
        g.close()
    # AUTO pairs from 2^20 nodes on
    g = L.Lattice(768, 768, p, W.boundary(), precision=L.FP32_DEVIATION)
    assert g.step_launches(10) == 10
    g.close()
    g = L.Lattice(1024, 1024, p, W.boundary(), precision=L.FP32_DEVIATION)
    assert g.step_launches(10) == 5
    g.close()
    g = L.Lattice(64, 40, p, W.boundary(), precision=L.FP32_DEVIATION)
    g.set_persistent(L.PERSISTENT_ON)
    assert g.step_launches(10) in (1, 10)  # one persistent launch where co-residency allows it
    with pytest.raises(L.Lbm13Error):
        g.set_pair_steps(7)
    g.close()
