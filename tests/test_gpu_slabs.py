"""y-slab decomposition on one device: a lattice split into K slabs with a
two-row halo exchange after every step (LBM13_HALO sides, lbm13_halo_pack /
lbm13_halo_unpack) gives bit-identical states to the undivided lattice, with
walls, forcing, periodic rings (including a ring of one slab) and both
storages; in FP64 it matches the oracle within 1e-10."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1401_0188_gb300 import pstar as product_pstar
from paper_1401_0188_gb300 import workloads as W

pytestmark = pytest.mark.gpu
NTH = max(1, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_0188_gb300 import build, lbm13
    build.build()
    lbm13.lib()
    return lbm13


def _case(kind, nx, ny, seed):
    p = product_pstar(0.05, 0.71)
    T0 = (p["E0"] + 28) / 26
    bnd = {"cavity": W.cavity(T0, 0.01, 1e-4, wall_density=1), "periodic": W.boundary(gx=1e-5, gy=-2e-5),
           "poiseuille": W.poiseuille(1e-5), "couette": W.couette(T0, 0.02, 0.01),
           "slab": W.heated_slab(T0, 2e-6, 0.01)}[kind]
    return p, bnd, W.random_fields(nx, ny, T0, seed=seed, du=0.01, drho=0.005, dT=0.003)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind,nx,ny,K", [("cavity", 64, 70, 2), ("cavity", 48, 61, 4), ("periodic", 48, 64, 3),
                                          ("periodic", 40, 24, 1), ("poiseuille", 40, 48, 2),
                                          ("couette", 36, 40, 3), ("slab", 40, 36, 3)])
def test_slabs_equal_the_undivided_lattice(L, precision, kind, nx, ny, K):
    from paper_1401_0188_gb300 import slabs
    p, bnd, fields = _case(kind, nx, ny, seed=700 + K)
    whole = L.Lattice(nx, ny, p, bnd, precision=precision)
    whole.set_state(*fields)
    split = slabs.SlabLattice(nx, ny, K, p, bnd, precision=precision)
    split.set_state(*fields)
    assert np.array_equal(split.raw_state(), whole.get_raw_state())
    for n in (1, 40):
        whole.step(n)
        split.step(n)
        assert split.t == whole.t
        assert np.array_equal(split.raw_state(), whole.get_raw_state()), (kind, K, whole.t)
    split.close()
    whole.close()


def test_slabs_match_the_oracle_fp64(L):
    """The 64 x 64 transverse shear wave of the first configuration with the
    seeded perturbation, in four slabs, 1000 steps: all 13 moments within 1e-10
    of the oracle."""
    from paper_1401_0188_gb300 import slabs
    p = product_pstar(0.05, 0.71)
    T0 = (p["E0"] + 28) / 26
    n = 64
    ux, uy = W.shear_wave(n, n, 0.01)
    split = slabs.SlabLattice(n, n, 4, p, W.boundary(), precision=L.FP64)
    split.set_state(1.0, ux, uy, T0)
    o = O.Lattice(n, n, p, O.boundary(), nthreads=NTH)
    o.set_equilibrium(1.0, ux, uy, T0)
    split.step(1000)
    o.step(1000)
    assert np.abs(split.moments() - o.moments()).max() <= 1e-10
    split.close()


def test_halo_arguments_are_checked(L):
    from paper_1401_0188_gb300 import slabs
    import torch
    p = product_pstar(0.05, 0.71)
    halo = {"kind": L.HALO, "u_t": 0.0, "T": 0.0}
    with pytest.raises(L.Lbm13Error):  # halo sides are south or north only
        L.Lattice(32, 32, p, dict(W.boundary(), west=halo, east=halo))
    with pytest.raises(L.Lbm13Error):  # four rows besides the two halo rows of each side
        L.Lattice(32, 7, p, slabs.slab_boundary(W.poiseuille(1e-5), True, True))
    g = L.Lattice(32, 12, p, slabs.slab_boundary(W.poiseuille(1e-5), True, False))
    buf = torch.empty(g.halo_bytes(), dtype=torch.uint8, device="cuda")
    assert g.halo_bytes() == 8 * 32 * 8
    g.halo_pack(L.HALO_SOUTH, buf)
    with pytest.raises(L.Lbm13Error):  # north is a wall, not a halo side
        g.halo_pack(L.HALO_NORTH, buf)
    g.close()
