"""The batched linear-stability scan on the GPU (lbm13_linear_growth_batch,
the dispersion-root procedure of the end of Sec. 2 for many cases at once):
it agrees with the library's host scan and with a scan of the oracle's
finite-difference Jacobian, for stable and unstable sets and moving
backgrounds; the population search built on it repairs an unstable starting
set; lbm13_create also scans at a moving wall's speed."""
import numpy as np
import pytest

from oracle import linear as OL
from oracle import oracle as O
from paper_1401_0188_gb300 import params, stability

pytestmark = pytest.mark.gpu

CASES = [(params.pstar(0.05, 0.71), (0.0, 0.0)), (params.pstar(0.05, 0.71), (0.03, 0.0)),
         (params.pstar(0.005, 0.71), (0.0, 0.0)), (params.pstar(0.05, 1.0), (0.0212, 0.0212)),
         (params.select(0.02, 0.5), (0.02, 0.01)), (params.select(0.3, 0.9), (0.0, 0.03)),
         (params.pstar(0.05, 0.71), (0.1, 0.0))]


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_0188_gb300 import build, lbm13
    build.build()
    lbm13.lib()
    return lbm13


@pytest.mark.parametrize("n", [1, 9, 17])
def test_batched_scan_equals_host_scan(L, n):
    g = L.linear_growth_batch([p for p, _ in CASES], [u for _, u in CASES], n)
    for (p, u), gi in zip(CASES, g):
        assert gi == pytest.approx(L.linear_growth(p, u[0], u[1], n), abs=1e-12)
    # on a grid beyond k = 0 the unstable cases show, the stable ones stay stable
    assert abs(g[0]) < 1e-12
    if n > 1:
        assert g[2] > 1e-6 and g[3] > 1e-3 and g[6] > 1e-3


def test_batched_scan_matches_oracle_jacobian(L):
    """max |z| - 1 over the k-grid from the eigenvalues of
    diag(exp(-i k.v)) J with J differentiated from the oracle's collision."""
    n = 9
    ks = np.linspace(-np.pi, np.pi, n)
    V = np.array(O.velocities()).T
    for p, u in CASES[:5]:
        J, _ = OL.collision_jacobian(O.Lattice(2, 2, p), 1.0, u[0], u[1])
        worst = -1.0
        for kx in ks:
            for ky in ks:
                A = np.exp(-1j * (V @ np.array([kx, ky])))[:, None] * J
                worst = max(worst, np.abs(np.linalg.eigvals(A)).max() - 1.0)
        assert L.linear_growth_batch([p], [u], n)[0] == pytest.approx(worst, abs=1e-7)


def test_search_repairs_an_unstable_start(L):
    """pstar is unstable at Pr = 0.97 (the merging of the thermal and viscous
    modes near Pr = 1); the GPU population search started from it alone
    returns a set that scans stable on a finer grid."""
    assert stability.max_growth(params.pstar(0.05, 0.97), ((0.0, 0.0),), 13) > 1e-6
    p, g, _ = stability.search_batched(0.05, 0.97, starts=[stability.PSTAR_RAW], population=48, generations=60)
    assert g <= 1e-11
    assert stability.max_growth(p, ((0.0, 0.0), (0.03, 0.0), (0.0212, 0.0212)), 21) < 1e-9


def test_create_scans_at_the_wall_speed(L):
    """A set stable at rest but unstable in a flow at 0.1 is accepted for a
    box at rest and refused when a wall moves at 0.1."""
    import ctypes
    from paper_1401_0188_gb300 import workloads as W
    p = params.pstar(0.05, 0.71)
    assert L.linear_growth(p, 0.0, 0.0, 9) < 1e-9 < L.linear_growth(p, 0.1, 0.0, 9)
    box = W.boundary(west=W.wall(W.WALL_BB), east=W.wall(W.WALL_BB), south=W.wall(W.WALL_BB),
                     north=W.wall(W.WALL_BB))
    L.Lattice(16, 16, p, box).close()
    lid = dict(box, north=W.wall(W.WALL_BB, 0.1))
    with pytest.raises(L.Lbm13Error) as e:
        L.Lattice(16, 16, p, lid)
    assert e.value.status == 3
