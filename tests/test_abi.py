"""The C-ABI library builds, loads and exports every entry point that
include/lbm13.h declares; its host-only parameter derivation agrees with the
oracle's (no GPU needed)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1401_0188_gb300 import build, lbm13
    build.build()
    return lbm13.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm13.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm13_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_documented_entry_points():
    from paper_1401_0188_gb300 import lbm13
    assert set(_declared()) == set(lbm13.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_version_and_status_strings(lib):
    from paper_1401_0188_gb300 import lbm13
    assert "D2Q13" in lbm13.lbm13_version()
    assert lib.lbm13_status_string(4).decode().startswith("state diverged")


def test_product_parameter_set_equals_oracle_parameter_set():
    from oracle import oracle as O
    from paper_1401_0188_gb300 import params
    for nu, Pr in ((0.05, 0.71), (0.02, 0.5), (0.1, 0.9)):
        a, b = params.pstar(nu, Pr), O.pstar(nu, Pr)
        assert a.keys() == b.keys()
        for k in a:
            assert a[k] == pytest.approx(b[k], rel=1e-13, abs=1e-13), k


@pytest.mark.parametrize("nu,Pr", [(0.05, 0.71), (0.01, 0.5), (0.3, 0.9)])
def test_derived_constants_match_oracle(lib, nu, Pr):
    from oracle import oracle as O
    from paper_1401_0188_gb300 import lbm13
    p = O.pstar(nu, Pr)
    st, out = lbm13.lbm13_derive(p)
    assert st == 0
    c = O.Lattice(2, 2, p).constants()
    names = ("A", "B", "h1", "k1", "h2", "c2", "c_erho", "sigma_XX", "sigma_q")
    for i, n in enumerate(names):
        assert out[i] == pytest.approx(c[n], rel=1e-13), n
    assert np.allclose(out[9:22], c["s"], rtol=1e-13, atol=0)
    assert np.allclose(out[22:35], c["w"], rtol=1e-12, atol=1e-15)
    assert out[35] == pytest.approx(c["T0"], rel=1e-14)
    assert out[37] == pytest.approx(nu / Pr)


def test_derive_rejects_bad_parameters(lib):
    from oracle import oracle as O
    from paper_1401_0188_gb300 import lbm13
    p = O.pstar()
    assert lbm13.lbm13_derive(dict(p, s_eps=2.0))[0] == 1          # rate outside (0, 2)
    assert lbm13.lbm13_derive(dict(p, nu=-0.1))[0] == 1            # negative viscosity
    assert lbm13.lbm13_derive(dict(p, Pr=float("nan")))[0] == 1
    # B > 0 makes sigma_q negative: no positive relaxation time for q
    assert lbm13.lbm13_derive(dict(p, c1=-0.5, E0=-12.0))[0] == 3
