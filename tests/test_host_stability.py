"""Host-side linear stability module and parameter selection (no GPU): the
analytic moment-space Jacobian agrees with the oracle's finite-difference one,
and the parameter sets that `params.select` hands out scan stable over their
stated (nu, Pr) ranges while pstar is unstable near Pr = 1 (the paper's warning
that the thermal and viscous modes merge near a critical Prandtl number)."""
import numpy as np
import pytest

from paper_1401_0188_gb300 import params, stability

UL = ((0.0, 0.0), (0.03, 0.0), (0.0212, 0.0212))


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1401_0188_gb300 import build
    build.build()


@pytest.mark.parametrize("U", [(0.0, 0.0), (0.02, 0.01)])
def test_analytic_jacobian_matches_oracle(U):
    from oracle import oracle as O, linear
    p = params.pstar(0.05, 0.71)
    J = stability.collision_jacobian(p, U)
    Jo, _ = linear.collision_jacobian(O.Lattice(2, 2, p), 1.0, U[0], U[1])
    assert np.abs(J - Jo).max() < 1e-8


@pytest.mark.parametrize("nu,Pr", [(0.01, 0.5), (0.02, 0.8), (0.05, 0.97), (0.2, 1.0), (0.35, 0.9),
                                   (0.003, 0.6), (0.006, 0.71), (0.08, 0.55), (0.005, 0.8), (0.007, 0.95),
                                   (0.006, 0.9), (0.35, 0.6), (0.15, 0.85), (0.04, 0.93)])
@pytest.mark.parametrize("physical_heating", [True, False])
def test_selected_sets_are_stable(nu, Pr, physical_heating):
    assert stability.max_growth(params.select(nu, Pr, physical_heating), UL, 21) < 1e-9


def test_viscous_heating_factor():
    """phi = sigma_q gamma / nu: -0.53 for pstar, exactly 1 on the heating
    family (c1 from heating_c1 cancels c_epsE out of phi), and 1 for the sets
    select hands out inside that family's range."""
    assert stability.viscous_heating_factor(params.pstar(0.05, 0.71)) == pytest.approx(-0.530182, abs=1e-6)
    for cE in (-3.0, -1.3, 0.5):
        p = dict(params.pstar(0.05, 0.71), c_epsE=cE)
        p["c1"] = stability.heating_c1(p["E0"])
        assert stability.viscous_heating_factor(p) == pytest.approx(1.0, abs=1e-12)
    for nu, Pr in ((0.01, 0.6), (0.3, 0.71), (0.1, 0.9), (0.03, 0.95)):
        assert stability.viscous_heating_factor(params.select(nu, Pr)) == pytest.approx(1.0, abs=1e-12)


def test_pstar_unstable_near_unit_prandtl():
    assert stability.max_growth(params.pstar(0.05, 1.0), UL, 21) > 1e-3


def test_select_refuses_unknown_region():
    with pytest.raises(ValueError):
        params.select(0.004, 0.95, search=False)
    with pytest.raises(ValueError):
        params.select(0.006, 0.99, search=False)
    assert params.stable_viscosity(0.004, 0.95) == 0.005
    assert params.stable_viscosity(0.004, 0.99) == 0.01


@pytest.mark.parametrize("nu,Pr,U", [(0.05, 0.71, (0.0, 0.0)), (0.05, 0.71, (0.03, 0.0)), (0.02, 0.5, (0.02, 0.01)),
                                     (0.005, 0.71, (0.0, 0.0)), (0.05, 1.0, (0.0212, 0.0212))])
def test_library_scan_matches_numpy_scan(nu, Pr, U):
    """The C++ eigenvalue scan (Hessenberg + shifted QR) behind lbm13_create
    agrees with the numpy scan of the same linearised step, stable and unstable
    sets alike."""
    from paper_1401_0188_gb300 import lbm13
    p = params.pstar(nu, Pr)
    g_lib = lbm13.linear_growth(p, U[0], U[1], 13)
    g_np = stability.max_growth(p, (U,), 13)
    assert g_lib == pytest.approx(g_np, abs=1e-10)


def test_create_rejects_a_linearly_unstable_set():
    """lbm13_create refuses pstar at nu = 0.005 (unstable at rest) with
    LBM13_EUNSTABLE before touching a device, and accepts the set select()
    gives for the same viscosity as far as the scan goes."""
    import ctypes
    from paper_1401_0188_gb300 import lbm13
    L = lbm13.lib()
    bnd = lbm13.make_boundary(lbm13.boundary())
    h = ctypes.c_void_p()
    st = L.lbm13_create(16, 16, ctypes.byref(lbm13.make_params(params.pstar(0.005, 0.71))), ctypes.byref(bnd), 0,
                        None, None, ctypes.byref(h))
    assert st == 3 and not h.value
    assert b"linearly unstable" in L.lbm13_last_error(None)
    assert lbm13.linear_growth(params.select(0.005, 0.71)) < 1e-12


def test_batched_search_logic_with_the_host_scan():
    """stability.search_batched with the numpy scan standing in for the GPU:
    from pstar at Pr = 0.95 (unstable) and the tabulated sets it returns a set
    that scans stable on a finer grid."""
    def host_growth(plist, ulist):
        return [stability.max_growth(p, (u,), 9) for p, u in zip(plist, ulist)]
    p, g, raw = stability.search_batched(0.05, 0.95, growth=host_growth, starts=[stability.PSTAR_RAW, params.SET_HIGH_PR],
                                         population=8, generations=3)
    assert g <= 1e-11
    assert stability.max_growth(p, UL, 21) < 1e-9
