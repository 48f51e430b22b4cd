"""lbm13_create's host-side validation, run without a GPU: every malformed
argument is refused with its status and a message before any device call,
and a parameter set whose linearised step amplifies a mode at rest or at the
walls' speed (the dispersion scan at the end of Sec. 2) is refused with
LBM13_EUNSTABLE.  No handle is returned for a refused call."""
import ctypes as C
import math

import pytest

from paper_1401_0188_gb300 import params as P
from paper_1401_0188_gb300 import workloads as W

EINVAL, EUNSTABLE, ECUDA = 1, 3, 6


@pytest.fixture(scope="module")
def L():
    from paper_1401_0188_gb300 import build, lbm13
    build.build()
    lbm13.lib()
    return lbm13


def _create(L, nx, ny, p, bnd, precision=0, out=True):
    h = C.c_void_p(1234)  # overwritten with NULL on failure
    st = L.lib().lbm13_create(nx, ny, C.byref(L.make_params(p)), C.byref(L.make_boundary(bnd)), precision, None,
                              None, C.byref(h) if out else None)
    msg = L.lib().lbm13_last_error(None).decode()
    return st, h.value, msg


def _box(**kw):
    B = W.WALL_BB
    d = dict(west=W.wall(B), east=W.wall(B), south=W.wall(B), north=W.wall(B))
    d.update(kw)
    return W.boundary(**d)


def _cases():
    p = P.pstar(0.05, 0.71)
    B, M = W.WALL_BB, W.WALL_MIXED
    return {
        "zero width": (0, 8, p, W.boundary(), 0, EINVAL, "size"),
        "one column periodic": (1, 8, p, W.boundary(), 0, EINVAL, "size"),
        "walled axis of 3 rows": (8, 3, p, W.boundary(south=W.wall(B), north=W.wall(B)), 0, EINVAL, "size"),
        "too wide": ((1 << 20) + 1, 4, p, W.boundary(), 0, EINVAL, "size"),
        "too tall": (4, 32769, p, W.boundary(), 0, EINVAL, "size"),
        "unpaired periodic side": (8, 8, p, W.boundary(west=W.wall(B)), 0, EINVAL, "periodic"),
        "halo on an x side": (8, 8, p, W.boundary(west=W.wall(3), east=W.wall(3)), 0, EINVAL, "halo"),
        "unknown wall kind": (8, 8, p, _box(north=W.wall(7)), 0, EINVAL, "wall kind"),
        "non-finite wall speed": (8, 8, p, _box(north=W.wall(B, math.nan)), 0, EINVAL, "non-finite"),
        "non-finite force": (8, 8, p, dict(_box(), gy=math.inf), 0, EINVAL, "non-finite"),
        "unknown wall density rule": (8, 8, p, dict(_box(north=W.wall(M, 0.0, 0.6)), wall_density=2), 0, EINVAL,
                                      "wall_density"),
        "unknown precision": (8, 8, p, W.boundary(), 7, EINVAL, "precision"),
        "rate outside (0, 2)": (8, 8, dict(p, s_r=2.0), W.boundary(), 0, EINVAL, "parameter"),
        "negative viscosity": (8, 8, dict(p, nu=-0.05), W.boundary(), 0, EINVAL, "parameter"),
        "sigma_q <= 0": (8, 8, dict(p, c1=-0.5, E0=-12.0), W.boundary(), 0, EUNSTABLE, "sigma_q"),
        "lid faster than the set's envelope": (16, 16, p, _box(north=W.wall(B, 0.1)), 0, EUNSTABLE, "unstable"),
    }


@pytest.mark.parametrize("case", list(_cases()))
def test_malformed_create_is_refused(L, case):
    nx, ny, p, bnd, precision, status, word = _cases()[case]
    st, h, msg = _create(L, nx, ny, p, bnd, precision)
    assert st == status, (case, st, msg)
    assert h is None
    assert word in msg, msg


def test_null_out_is_refused(L):
    st, _, msg = _create(L, 8, 8, P.pstar(0.05, 0.71), W.boundary(), out=False)
    assert st == EINVAL and "out" in msg


def test_valid_create_without_a_device_reports_cuda(L):
    """On a machine without a GPU a well-formed call gets as far as the device
    query and returns LBM13_ECUDA (the library has no CPU path)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    st, h, msg = _create(L, 16, 16, P.pstar(0.05, 0.71), _box())
    assert st == ECUDA and h is None and "CUDA" in msg
