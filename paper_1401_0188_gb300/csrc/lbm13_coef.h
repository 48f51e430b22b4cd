// lbm13_coef.h -- the per-lattice constants of the step: those of the
// collision (Coef, in lbm13_math.cuh) from the free parameters, the derived
// constants of Sec. 2 (lbm13_derive's output) and the boundary's force and
// energy source, and the wall arguments of the four sides (WallArgs, in
// lbm13_internal.h) with the correction polynomials of Sec. 7's walls.  Host
// code, used by lbm13_create.
#pragma once

#include "lbm13_internal.h"

namespace lbm13 {

// D: the LBM13_DERIVED_COUNT constants of lbm13_derive (A, B, h1, k1, h2, c2,
// c_erho, sigma_XX, sigma_q, the 13 rates s_k, ...).
template <typename C>
void collision_coef(const lbm13_params &p, const double *D, const lbm13_boundary &b, Coef<C> &k)
{
    k.E0 = C(p.E0);
    k.cer = C(D[6]);
    k.ceE = C(p.c_epsE);
    k.cwr = C(p.c_vpi_rho);
    k.cwE = C(p.c_vpi_E);
    k.h1 = C(D[2]);
    k.k1 = C(D[3]);
    k.Q10 = C(p.c1 + D[2] + D[3] * p.E0);
    k.h2 = C(D[4]);
    k.k2 = C(p.k2);
    k.R10 = C(D[5] + D[4] + p.k2 * p.E0);
    const double *s = D + 9;
    k.l_eps = C(s[2] / kD[2]);
    k.l_vpi = C(s[3] / kD[3]);
    k.l_q = C(s[6] / kD[6]);
    k.l_r = C(s[8] / kD[8]);
    k.l_XX = C(s[10] / kD[10]);
    k.l_XY = C(s[11] / kD[11]);
    k.l_XXe = C(s[12] / kD[12]);
    k.gx = C(b.gx);
    k.gy = C(b.gy);
    k.rho_ref = C(b.rho_ref);
    // Energy source q (Sec. 9): equilibria at E + 13 q, so q_eq and r_eq
    // shift by 13 q k1 and 13 q k2 per unit of j.
    const double q = b.heat;
    k.Qh = q == 0.0 ? k.Q10 : C(p.c1 + D[2] + D[3] * (p.E0 + 13.0 * q));
    k.Rh = q == 0.0 ? k.R10 : C(D[5] + D[4] + p.k2 * (p.E0 + 13.0 * q));
    // Scalar block: values of the E, eps, varpi polynomials on the shells
    // (rest, unit axes, diagonals, distance-2 axes); the increment of a
    // population of shell s is eps_s d_eps + varpi_s d_varpi with
    // d_eps = l_eps (c_erho rho + c_epsE E - eps), all linear in the shell sums.
    const double ME[4] = {-28, -15, -2, 24}, Meps[4] = {140, -2, -67, 34}, Mvpi[4] = {-12, 8, -6, 1};
    const double le = s[2] / kD[2], lv = s[3] / kD[3];
    for (int sh = 0; sh < 4; ++sh)
        for (int l = 0; l < 4; ++l)
            k.B[sh][l] = C(Meps[sh] * le * (D[6] + p.c_epsE * ME[l] - Meps[l]) +
                           Mvpi[sh] * lv * (p.c_vpi_rho + p.c_vpi_E * ME[l] - Mvpi[l]));
    // Source: E* gains 26 q, eps and varpi relax toward equilibria raised by
    // 13 q c_epsE and 13 q c_varpiE.
    for (int sh = 0; sh < 4; ++sh)
        k.src[sh] = C(q == 0.0 ? 0.0
                               : ME[sh] * 26.0 * q / kD[1] + Meps[sh] * le * p.c_epsE * 13.0 * q +
                                     Mvpi[sh] * lv * p.c_vpi_E * 13.0 * q);
    // Tensor block: XX = X1 + 4 X9, XXe = -4 X1 + X9 relaxed and mapped back.
    const double lXX = s[10] / kD[10], lXXe = s[12] / kD[12];
    k.t1X1 = C(-lXX - 16.0 * lXXe);
    k.t1X9 = C(-4.0 * lXX + 4.0 * lXXe);
    k.t9X1 = C(-4.0 * lXX + 4.0 * lXXe);
    k.t9X9 = C(-16.0 * lXX - lXXe);
}

// Coefficients (a0 .. a4) of P(drho, dE) = a0 + a1 drho + a2 dE + a3 drho^2 +
// a4 drho dE from values of P, which is exactly of that form: every
// equilibrium moment at rho = 1 + drho, E = E0 + dE, j = rho u is a
// combination of rho, E, rho^2 and rho E (Eq. d2q13-moments-equil).  The
// sample points rho = 1, 1 +- 1/2 and E0, E0 +- 1/2 give the coefficients
// without truncation error.
template <typename F>
void quadratic_coefficients(F P, double a[5])
{
    const double h = 0.5;
    const double p00 = P(0.0, 0.0), pp0 = P(h, 0.0), pm0 = P(-h, 0.0);
    const double p0p = P(0.0, h), p0m = P(0.0, -h), ppp = P(h, h);
    a[0] = p00;
    a[1] = (pp0 - pm0) / (2.0 * h);
    a[2] = (p0p - p0m) / (2.0 * h);
    a[3] = (pp0 + pm0 - 2.0 * p00) / (2.0 * h * h);
    a[4] = (ppp - pp0 - p0p + p00) / (h * h);
}

// Deviation of the equilibrium populations for the wall state (drho, dE) and
// wall velocity (ux, uy), from the double collision constants kd.
inline void wall_equilibrium(const Coef<double> &kd, double drho, double dE, double ux, double uy, double f[Q])
{
    const double rho = 1.0 + drho;
    equilibrium_dev(drho, dE, rho * ux, rho * uy, kd, f);
}

// The four sides' wall arguments (west, east, south, north): kinds, wall
// velocity and temperature terms, zero-flux constants and the correction
// polynomial of each entering link.  D: lbm13_derive's constants; kd: the
// double collision constants of the same lattice.
template <typename C>
void wall_coef(const lbm13_params &p, const double *D, const lbm13_boundary &b, const Coef<double> &kd,
               WallArgs<C> *w)
{
    const lbm13_wall *src[4] = {&b.west, &b.east, &b.south, &b.north};
    for (int s = 0; s < 4; ++s) {
        const lbm13_wall &in = *src[s];
        WallArgs<C> &o = w[s];
        const double ux = s <= EAST ? 0.0 : in.u_t, uy = s <= EAST ? in.u_t : 0.0;
        o.kind = in.kind;
        o.needs_data = in.kind == WALL_MIXED || (in.kind == WALL_BB && in.u_t != 0.0);
        o.ux = C(ux);
        o.uy = C(uy);
        o.base = C(26.0 * in.T - 28.0);
        o.eT = C(26.0 * (in.T - (p.E0 + 28.0) / 26.0));
        o.mass_flux = in.kind == WALL_MIXED && b.wall_density == LBM13_WALL_DENSITY_ZERO_FLUX;
        o.wsum = C(D[22 + 1] + 2.0 * D[22 + 9]);
        // zero-flux density: even parts of the unit-density wall equilibrium on
        // the outgoing unit and distance-2 normal links
        double e[Q];
        wall_equilibrium(kd, 0.0, 26.0 * (in.T - (p.E0 + 28.0) / 26.0) + 13.0 * (ux * ux + uy * uy), ux, uy, e);
        const int ja = s == WEST ? 3 : s == EAST ? 1 : s == SOUTH ? 4 : 2;
        const int jb = s == WEST ? 11 : s == EAST ? 9 : s == SOUTH ? 12 : 10;
        o.zf_ea = C(0.5 * (e[ja] + e[copp(ja)]));
        o.zf_eb = C(0.5 * (e[jb] + e[copp(jb)]));
        for (int i = 0; i < 4; ++i) {
            const int j = wall_link(s, i), jn = copp(j);
            const bool normal = s <= EAST ? cvy(j) == 0 : cvx(j) == 0;
            const bool abb = in.kind == WALL_MIXED && normal;
            double a[5];
            quadratic_coefficients(
                [&](double dr, double de) {
                    double f[Q];
                    wall_equilibrium(kd, dr, de, ux, uy, f);
                    return abb ? f[j] + f[jn] : f[j] - f[jn];
                },
                a);
            for (int m = 0; m < 5; ++m) o.poly[i][m] = C(a[m]);
        }
    }
    // a corner diagonal crosses both walls and takes both walls' corrections
    // for its link (their slots above), each at its own wall's state
}

} // namespace lbm13
