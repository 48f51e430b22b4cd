"""Linear stability of the D2Q13 scheme and a search for stable free parameters.

The paper picks its free parameters "by computing the roots of the dispersion
equation for several values of the wave vector ranging from 0 to 2 pi in
magnitude and several directions" (end of Sec. 2) and warns that near Pr = 1
the thermal and viscous modes merge and the scheme tends to go unstable
(Introduction).  This module does that on the host:

- `amplification(params, U, k)`: the linearised time step about the uniform
  state (rho, u, E) = (1, U, E0 + 13 |U|^2) for a Fourier mode exp(i k.x).
  The collision Jacobian is assembled in moment space from the equilibria of
  Eq. (d2q13-moments-equil) and the derived constants of Eqs.
  (d2q13-diffusion), (d2q13-sigma-qx) (taken from the library's
  lbm13_derive), then mapped to populations with M and M^-1 = M^T D^-1;
  streaming a mode over link j multiplies population j by exp(-i k.v_j).
- `max_growth(params, U_list, n)`: max |z| - 1 over an n x n grid of k in
  [-pi, pi]^2 and the given background velocities (<= ~1e-12 means stable).
- `search(nu, Pr, ...)`: Nelder-Mead over the rest weights, c1, k2, c_varpiE
  and the four free rates, starting from a given set, until the scan is
  stable.  c_epsE follows the Prandtl number as in `params.pstar`.
- `search_batched(nu, Pr, ...)`: the same procedure as a population search
  whose candidates are all scanned in one batched call per generation
  (`lbm13.linear_growth_batch` on the GPU by default: every candidate at every
  background velocity and wave vector at once).
"""
import numpy as np

from . import params as _params

_V = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1),
               (2, 0), (0, 2), (-2, 0), (0, -2)], dtype=float)


def moment_matrix():
    """M_kj = p_k(v_j) of Eq. (d2q13-polynomes), q with -3 (orthogonal rows)."""
    x, y = _V[:, 0], _V[:, 1]
    r2 = x * x + y * y
    rows = [np.ones(13), -28 + 13 * r2, 140 + r2 * (-361 / 2 + 77 * r2 / 2),
            -12 + r2 * (581 / 12 + r2 * (-273 / 8 + 137 / 24 * r2)), x, y, x * (-3 + r2), y * (-3 + r2),
            x * (101 / 6 + r2 * (-63 / 4 + 35 / 12 * r2)), y * (101 / 6 + r2 * (-63 / 4 + 35 / 12 * r2)),
            x * x - y * y, x * y, (x * x - y * y) * (-65 / 12 + 17 / 12 * r2)]
    return np.rint(np.array(rows))


_M = moment_matrix()
_D = (_M * _M).sum(axis=1)
_MINV = _M.T / _D


def derived(params):
    """(status, derived constants) from the library's host-only lbm13_derive."""
    from . import lbm13
    return lbm13.lbm13_derive(params)


def collision_jacobian(params, U=(0.0, 0.0)):
    """d f*/d f about rho = 1, j = U, E = E0 + 13 |U|^2 (no force)."""
    st, d = derived(params)
    if st != 0:
        raise ValueError(f"parameter set rejected by lbm13_derive (status {st})")
    h1, k1, h2, c2, cer = d[2], d[3], d[4], d[5], d[6]
    s = d[9:22]
    E0 = params["E0"]
    rho, jx, jy = 1.0, U[0], U[1]
    E = E0 + 13.0 * (jx * jx + jy * jy)
    G = np.zeros((13, 13))  # d m_eq / d m for the conserved (rho 0, E 1, jx 4, jy 5)
    G[2, 0], G[2, 1] = cer, params["c_epsE"]
    G[3, 0], G[3, 1] = params["c_vpi_rho"], params["c_vpi_E"]
    q = params["c1"] + h1 * rho + k1 * E
    r = c2 + h2 * rho + params["k2"] * E
    for kq, kr, jc, jv in ((6, 8, 4, jx), (7, 9, 5, jy)):
        G[kq, jc], G[kq, 0], G[kq, 1] = q, jv * h1, jv * k1
        G[kr, jc], G[kr, 0], G[kr, 1] = r, jv * h2, jv * params["k2"]
    G[10, 4], G[10, 5], G[10, 0] = 2 * jx / rho, -2 * jy / rho, -(jx * jx - jy * jy) / rho ** 2
    G[11, 4], G[11, 5], G[11, 0] = jy / rho, jx / rho, -jx * jy / rho ** 2
    S = np.diag(s)
    return _MINV @ (np.eye(13) - S + S @ G) @ _M


def amplification(J, k):
    return np.exp(-1j * (_V @ np.asarray(k, dtype=float)))[:, None] * J


def max_growth(params, U_list=((0.0, 0.0),), n=25):
    ks = np.linspace(-np.pi, np.pi, n)
    kk = np.array([(a, b) for a in ks for b in ks])
    worst = -1.0
    for U in U_list:
        J = collision_jacobian(params, U)
        ph = np.exp(-1j * (kk @ _V.T))                      # (nk, 13)
        A = ph[:, :, None] * J[None, :, :]                  # (nk, 13, 13)
        z = np.abs(np.linalg.eigvals(A)).max()
        worst = max(worst, z - 1.0)
    return worst


def _heating_moments():
    """(a, b): the first-order viscous heating of a transverse wave u_y = V cos kx
    comes from the q-flux of G = sum_j v_x^2 (|v|^2 - 3) f_eq,j, whose V^2
    coefficient is gamma = a + b c_epsE: projected on the basis, v_x^2 (|v|^2 - 3)
    has weight alpha_E on E (which carries 13 V^2), alpha_eps on eps (whose
    equilibrium carries 13 c_epsE V^2) and alpha_XX on XX (equilibrium -V^2)."""
    x, y = _V[:, 0], _V[:, 1]
    alpha = _M @ (x * x * (x * x + y * y - 3)) / _D
    return 13 * alpha[1] - alpha[10], 13 * alpha[2]


def viscous_heating_factor(params):
    """phi = sigma_q gamma / nu: the viscous heating of the scheme relative to a
    physical gas (phi = 1).  The first-order energy flux of the scheme carries
    13 sigma_q d_x G; for a shear wave that is the viscous work term when
    sigma_q gamma = nu.  With sigma_q = -(1309/2) sigma_XX A / B and
    sigma_XX = 104 nu / A (Eq. d2q13-sigma-qx), phi = -68068 gamma / B."""
    a, b = _heating_moments()
    gamma = a + b * params["c_epsE"]
    B = 114404 + 51051 * params["c1"] - 11492 * params["c_epsE"] + 7854 * params["E0"]
    return -1309 / 2 * 104 * gamma / B


def heating_c1(E0):
    """c1 that makes phi = 1 for any c_epsE: 68068 b = 11492 makes the c_epsE
    terms of gamma and B cancel, leaving 114404 + 51051 c1 + 7854 E0 = -68068 a."""
    a, _ = _heating_moments()
    return (-68068 * a - 114404 - 7854 * E0) / 51051


def make_params(raw, nu, Pr, physical_heating=False):
    """Free parameters from the search vector
    raw = (x0, x1, x2, x3, c1, k2, c_varpiE, s_eps, s_varpi, s_r, s_XXe):
    rest weights proportional to (x0, x1/4 x4, x2/4 x4, x3/4 x4) on the rest,
    unit-axis, diagonal and distance-2 shells."""
    x = np.abs(np.asarray(raw[:4], dtype=float))
    w = np.array([x[0]] + [x[1] / 4] * 4 + [x[2] / 4] * 4 + [x[3] / 4] * 4)
    w = w / w.sum()
    m0 = _M @ w
    E0, eps0, vpi0 = m0[1], m0[2], m0[3]
    c1, k2, cvE = raw[4], raw[5], raw[6]
    if physical_heating:
        c1 = heating_c1(E0)
    A = 13 * c1 + 95 + 2 * E0
    B0 = 114404 + 51051 * c1 + 7854 * E0
    const = 140 + A * B0 / (22984 * Pr) - eps0
    slope = 28 - A * 11492 / (22984 * Pr) + E0
    ceE = -const / slope
    return {"E0": E0, "c1": c1, "k2": k2, "c_epsE": ceE, "c_vpi_rho": vpi0 - cvE * E0, "c_vpi_E": cvE,
            "Pr": Pr, "nu": nu, "s_eps": raw[7], "s_vpi": raw[8], "s_r": raw[9], "s_XXe": raw[10]}


PSTAR_RAW = (0.53, 0.196, 0.07, 0.204, -1.0, 0.4, 0.3, 0.6, 1.25, 1.2, 1.0)


def search(nu, Pr, U_max=0.03, start=PSTAR_RAW, n=17, maxiter=600, seed_scale=0.05, physical_heating=False):
    """Nelder-Mead for a raw vector whose parameter set scans stable (growth
    <= 1e-11) at background speeds 0, U_max along x and along the diagonal.
    With physical_heating, c1 follows E0 through `heating_c1` (phi = 1).
    Returns (params, growth) of the best point found."""
    from scipy.optimize import minimize
    Ul = ((0.0, 0.0), (U_max, 0.0), (U_max / np.sqrt(2), U_max / np.sqrt(2)))

    def objective(raw):
        p = make_params(raw, nu, Pr, physical_heating)
        rates = np.array(raw[7:11])
        if (rates <= 0.02).any() or (rates >= 1.98).any():
            return 1.0
        try:
            g = max_growth(p, Ul, n)
        except ValueError:
            return 1.0
        return max(g, 0.0)

    x0 = np.array(start, dtype=float)
    simplex = [x0] + [x0 * (1 + seed_scale * (np.eye(len(x0))[i] * (1 if i % 2 else -1))) for i in range(len(x0))]
    res = minimize(objective, x0, method="Nelder-Mead",
                   options={"initial_simplex": np.array(simplex), "maxiter": maxiter, "xatol": 1e-6, "fatol": 0.0})
    best = make_params(res.x, nu, Pr, physical_heating)
    return best, max_growth(best, Ul, 25), res.x


def _growth_in_batches(growth, plist, ulist):
    """growth(plist, ulist) with a failing batch split until the failing
    cases are isolated (their growth counts as 1: unusable)."""
    from . import lbm13
    try:
        return np.asarray(growth(plist, ulist), dtype=float)
    except lbm13.Lbm13Error:
        if len(plist) == 1:
            return np.array([1.0])
        h = len(plist) // 2
        return np.concatenate([_growth_in_batches(growth, plist[:h], ulist[:h]),
                               _growth_in_batches(growth, plist[h:], ulist[h:])])


def search_batched(nu, Pr, U_max=0.03, n=17, growth=None, starts=None, population=64, generations=40, seed=1,
                   scale=0.05, physical_heating=False, tol=1e-11, verify_n=25, verify=None):
    """Population search for a raw vector whose parameter set scans stable
    (growth <= tol) at background speeds 0, U_max along x and along the
    diagonal.  Each generation scans every candidate at the three speeds in
    one call of `growth(params_list, velocities)` (default: the library's
    batched GPU scan on an n x n k-grid), keeps the eight best and perturbs
    them (seeded, relative steps of `scale`, shrinking).  A candidate that
    scans stable is scanned again on the finer verify_n grid (`verify`, by
    default the same batched scan), whose growth replaces its score: a coarse
    grid can miss a narrow unstable band.  Returns (params, growth, raw) of
    the first candidate stable on both grids, or of the best one found."""
    from . import lbm13, params as _p
    if growth is None:
        growth = lambda pl, ul: lbm13.linear_growth_batch(pl, ul, n)  # noqa: E731
        if verify is None:
            verify = lambda pl, ul: lbm13.linear_growth_batch(pl, ul, verify_n)  # noqa: E731
    Ul = ((0.0, 0.0), (U_max, 0.0), (U_max / np.sqrt(2), U_max / np.sqrt(2)))
    rng = np.random.Generator(np.random.PCG64(seed))
    if starts is None:
        starts = [_p.SET_HEAT, _p.SET_HIGH_PR, _p.SET_GAP, _p.SET_LOW_NU, PSTAR_RAW]
    pop = [np.array(x, dtype=float) for x in starts]
    while len(pop) < population:
        base = pop[len(pop) % len(starts)]
        pop.append(base * (1.0 + scale * rng.standard_normal(base.shape)))
    best = (None, np.inf, None)
    for gen in range(generations):
        cand, fit = [], np.full(len(pop), 1.0)
        for i, raw in enumerate(pop):
            rates = raw[7:11]
            if (rates <= 0.02).any() or (rates >= 1.98).any() or (raw[:4] <= 0).any():
                continue
            p = make_params(raw, nu, Pr, physical_heating)
            if derived(p)[0] != 0:
                continue
            cand.append((i, p))
        if cand:
            pl = [p for _, p in cand for _ in Ul]
            ul = [u for _ in cand for u in Ul]
            g = _growth_in_batches(growth, pl, ul).reshape(len(cand), len(Ul)).max(axis=1)
            for (i, _), gi in zip(cand, g):
                fit[i] = max(gi, 0.0)
            passed = [(i, p) for (i, p), gi in zip(cand, g) if gi <= tol]
            if passed and verify is not None:
                pl = [p for _, p in passed for _ in Ul]
                ul = [u for _ in passed for u in Ul]
                gv = _growth_in_batches(verify, pl, ul).reshape(len(passed), len(Ul)).max(axis=1)
                for (i, _), gi in zip(passed, gv):
                    fit[i] = max(gi, 0.0)
        order = np.argsort(fit, kind="stable")
        if fit[order[0]] < best[1]:
            best = (make_params(pop[order[0]], nu, Pr, physical_heating), float(fit[order[0]]), pop[order[0]].copy())
        if best[1] <= tol:
            break
        elite = [pop[i] for i in order[:8]]
        step = scale * (0.85 ** gen)
        pop = elite + [elite[k % len(elite)] * (1.0 + step * rng.standard_normal(elite[0].shape))
                       for k in range(population - len(elite))]
    return best
