// lbm13_coef.h -- the per-lattice constants of the collision (Coef, in
// lbm13_math.cuh) from the free parameters, the derived constants of Sec. 2
// (lbm13_derive's output) and the boundary's force and energy source.  Host
// code, used by lbm13_create.
#pragma once

#include "../../include/lbm13.h"
#include "lbm13_math.cuh"

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

} // namespace lbm13
