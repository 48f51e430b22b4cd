"""lbm13_totals_noalloc: conserved totals for callers that cannot allocate.

A serving loop that has given its whole HBM budget to lattices through another
allocator, a latency-bound loop that cannot take the device-wide
synchronisation of cudaMalloc/cudaFree, or code inside an allocator callback
cannot let lbm13_residual allocate its reduction buffers.
lbm13_totals_noalloc gives them the same FP64 totals from a fixed file-scope
scratch array.  This file checks it through the C ABI against lbm13_residual,
on two calls in a row (the second reuses the scratch left by the first), at
the largest lattice the scratch holds (8192^2: every one of its 4096 rows in
use), and that a lattice one row larger is refused.  It is named so that
pytest collects it last.
"""
import ctypes as C

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


def _noalloc(L, lat):
    import torch
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    st = L.lib().lbm13_totals_noalloc(lat.handle, C.c_void_p(out.data_ptr()))
    assert st == 0, L.lib().lbm13_last_error(lat.handle)
    lat.synchronize()
    return out.cpu().numpy()


def _compare(res, tot, n, mom_scale=0.0):
    """Same sums in another block order: rounding differences only.  mom_scale
    bounds sum |j| over the lattice (momentum sums that cancel to ~0)."""
    assert tot[7] == n
    for k, i in enumerate((4, 5, 6, 7)):   # sum rho, jx, jy, E
        atol = 1e-12 + (1e-13 * mom_scale if k in (1, 2) else 0.0)
        assert tot[k] == pytest.approx(res[i], rel=1e-12, abs=atol), (k, tot[k], res[i])
    assert tot[4] == res[12]                # non-finite count
    assert tot[5] == res[11]                # max |u|
    assert tot[6] == pytest.approx(res[15], rel=1e-13)  # mean T


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_totals_match_residual_on_two_calls(L, pstar, precision):
    T0 = (pstar["E0"] + 28.0) / 26.0
    nx, ny = 300, 170
    lat = L.Lattice(nx, ny, pstar, W.cavity(T0, 0.01, 1e-4), precision=precision)
    lat.set_state(*W.random_fields(nx, ny, T0, seed=404, du=0.01, drho=0.005, dT=0.003))
    lat.step(25)
    _compare(lat.residual(), _noalloc(L, lat), nx * ny)
    lat.step(40)
    _compare(lat.residual(), _noalloc(L, lat), nx * ny)


def test_noalloc_totals_at_the_scratch_limit(L, pstar):
    import torch
    side = 8192  # 8192^2 = LBM13_NOALLOC_MAX_NODES: all 4096 scratch rows
    assert side * side == 67108864
    lat = L.Lattice(side, side, pstar, precision=L.FP32_DEVIATION)
    ux, uy = W.shear_wave(side, side)
    lat.set_state(1.0, ux, uy, None)
    lat.step(3)
    scale = 0.01 * side * side  # |u_x| <= 0.01
    _compare(lat.residual(), _noalloc(L, lat), side * side, scale)
    lat.step(2)
    _compare(lat.residual(), _noalloc(L, lat), side * side, scale)
    lat.close()
    torch.cuda.empty_cache()


def test_noalloc_refuses_lattices_beyond_its_scratch(L, pstar):
    import torch
    nx, ny = 8192, 8193  # one row more than LBM13_NOALLOC_MAX_NODES
    lat = L.Lattice(nx, ny, pstar, precision=L.FP32_DEVIATION)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert L.lib().lbm13_totals_noalloc(lat.handle, C.c_void_p(out.data_ptr())) == 1
    assert torch.count_nonzero(out).item() == 0
    lat.close()
    torch.cuda.empty_cache()
