// lbm13_math.cuh -- per-node arithmetic of the D2Q13 scheme, shared by the
// step, initialisation, read-out and reduction kernels of this library.
//
// The state is stored as deviations from the rest populations,
// df_j = f_j - w_j with w_j = f_eq,j(rho = 1, E = E0, j = 0), in both precision
// modes: the moments of w are (1, E0, eps0, varpi0, 0, ..., 0), so every moment
// below is the deviation from that rest state and nothing large is added to
// something small.
//
// Moment transform.  M is the 13 x 13 integer matrix of Sec. 2, Eq.
// (d2q13-polynomes), with q_x = x(-3 + x^2 + y^2) (the sign that makes the rows
// orthogonal; the printed +3 overlaps j_x by 84).  Because the rows are
// orthogonal, M^-1 = M^T D^-1 with D = diag(13, 4004, 42196, 548, 14, 14, 20,
// 20, 70, 70, 68, 4, 68).  Both products are evaluated through the pairs of
// opposite links (1,3) (2,4) (5,7) (6,8) (9,11) (10,12): pair sums feed the
// even moments, pair differences the odd ones, which takes about 50 additions
// or FMAs each way instead of 2 x 169.
#pragma once

#include <cuda_runtime.h>

#define LBM13_HD __host__ __device__ __forceinline__

namespace lbm13 {

constexpr int Q = 13;

// Sec. 2, Eq. (d2q13-vitesses) with Sec. 1, Eqs. (d2q5-vitesses), (d2q9-vitesses).
LBM13_HD constexpr int cvx(int j)
{
    return (j == 1 || j == 5 || j == 8) ? 1 : (j == 3 || j == 6 || j == 7) ? -1 : j == 9 ? 2 : j == 11 ? -2 : 0;
}
LBM13_HD constexpr int cvy(int j)
{
    return (j == 2 || j == 5 || j == 6) ? 1 : (j == 4 || j == 7 || j == 8) ? -1 : j == 10 ? 2 : j == 12 ? -2 : 0;
}
// index of -v_j
LBM13_HD constexpr int copp(int j)
{
    return j == 0 ? 0 : j <= 4 ? ((j + 1) % 4) + 1 : j <= 8 ? ((j - 3) % 4) + 5 : ((j - 7) % 4) + 9;
}
static_assert(copp(1) == 3 && copp(2) == 4 && copp(3) == 1 && copp(4) == 2, "opposites");
static_assert(copp(5) == 7 && copp(6) == 8 && copp(7) == 5 && copp(8) == 6, "opposites");
static_assert(copp(9) == 11 && copp(10) == 12 && copp(11) == 9 && copp(12) == 10, "opposites");

// Squared norms of the basis rows.
constexpr double kD[Q] = {13, 4004, 42196, 548, 14, 14, 20, 20, 70, 70, 68, 4, 68};

// Deviation moments of one node, in the paper's order.
template <typename C>
struct Mom {
    C rho, E, eps, vpi, jx, jy, qx, qy, rx, ry, XX, XY, XXe;
};

// Per-lattice constants of the collision, in the compute type.
template <typename C>
struct Coef {
    C E0;
    C cer, ceE, cwr, cwE;     // eps_eq = cer rho + ceE E, varpi_eq = cwr rho + cwE E
    C Q10, h1, k1;            // q_eq = j (c1 + h1 rho + k1 E) = j (Q10 + h1 drho + k1 dE)
    C R10, h2, k2;            // r_eq = j (c2 + h2 rho + k2 E) = j (R10 + h2 drho + k2 dE)
    C l_eps, l_vpi, l_q, l_r, l_XX, l_XY, l_XXe; // s_k / D_k
    C gx, gy, rho_ref;        // F = (rho - rho_ref) g
};

// m = M df (deviation moments).
template <typename C>
LBM13_HD void forward(const C f[Q], Mom<C> &m)
{
    const C a1 = f[1] + f[3], b1 = f[1] - f[3];
    const C a2 = f[2] + f[4], b2 = f[2] - f[4];
    const C a5 = f[5] + f[7], b5 = f[5] - f[7];
    const C a6 = f[6] + f[8], b6 = f[6] - f[8];
    const C a9 = f[9] + f[11], b9 = f[9] - f[11];
    const C a10 = f[10] + f[12], b10 = f[10] - f[12];
    const C S1 = a1 + a2, X1 = a1 - a2;
    const C S5 = a5 + a6, X5 = a5 - a6;
    const C S9 = a9 + a10, X9 = a9 - a10;
    const C dm = b5 - b6, dp = b5 + b6;
    m.rho = f[0] + S1 + S5 + S9;
    m.E = C(-28) * f[0] + C(-15) * S1 + C(-2) * S5 + C(24) * S9;
    m.eps = C(140) * f[0] + C(-2) * S1 + C(-67) * S5 + C(34) * S9;
    m.vpi = C(-12) * f[0] + C(8) * S1 + C(-6) * S5 + S9;
    m.jx = b1 + dm + C(2) * b9;
    m.jy = b2 + dp + C(2) * b10;
    m.qx = C(-2) * b1 - dm + C(2) * b9;
    m.qy = C(-2) * b2 - dp + C(2) * b10;
    m.rx = C(4) * b1 + C(-3) * dm + b9;
    m.ry = C(4) * b2 + C(-3) * dp + b10;
    m.XX = X1 + C(4) * X9;
    m.XY = X5;
    m.XXe = C(-4) * X1 + X9;
}

// f_j += sum_k M_kj d_k, where d_k is a moment increment already divided by
// D_k.  WithRho adds the rho row (every f_j += d_rho); the collision leaves rho
// unchanged and skips it.
template <bool WithRho, typename C>
LBM13_HD void inverse_add(const Mom<C> &d, C f[Q])
{
    const C b1 = C(-15) * d.E + C(-2) * d.eps + C(8) * d.vpi;
    const C t1 = d.XX + C(-4) * d.XXe;
    const C o1 = d.jx + C(-2) * d.qx + C(4) * d.rx;
    const C o2 = d.jy + C(-2) * d.qy + C(4) * d.ry;
    const C b5 = C(-2) * d.E + C(-67) * d.eps + C(-6) * d.vpi;
    const C sj = d.jx + d.jy, dj = d.jy - d.jx;
    const C sq = d.qx + d.qy, dq = d.qx - d.qy;
    const C sr = d.rx + d.ry, dr = d.rx - d.ry;
    const C o5 = sj - sq + C(-3) * sr;
    const C o6 = dj + dq + C(3) * dr;
    const C b9 = C(24) * d.E + C(34) * d.eps + d.vpi;
    const C t9 = C(4) * d.XX + d.XXe;
    const C o9 = C(2) * (d.jx + d.qx) + d.rx;
    const C o10 = C(2) * (d.jy + d.qy) + d.ry;
    const C e13 = b1 + t1, e24 = b1 - t1;
    const C e57 = b5 + d.XY, e68 = b5 - d.XY;
    const C e911 = b9 + t9, e1012 = b9 - t9;
    C r0 = C(-28) * d.E + C(140) * d.eps + C(-12) * d.vpi;
    if (WithRho) r0 += d.rho;
    C g[Q];
    g[0] = r0;
    g[1] = e13 + o1;
    g[3] = e13 - o1;
    g[2] = e24 + o2;
    g[4] = e24 - o2;
    g[5] = e57 + o5;
    g[7] = e57 - o5;
    g[6] = e68 + o6;
    g[8] = e68 - o6;
    g[9] = e911 + o9;
    g[11] = e911 - o9;
    g[10] = e1012 + o10;
    g[12] = e1012 - o10;
    if (WithRho) {
#pragma unroll
        for (int j = 1; j < Q; ++j) g[j] += d.rho;
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) f[j] += g[j];
}

// One collision in place (deviation form).  Equilibria of Sec. 2, Eq.
// (d2q13-moments-equil) at j + F/2; the nine non-conserved moments relax as
// m* = m + s (m_eq - m); j* = j + F and E* = E + 13 (|j + F|^2 - |j|^2)/rho
// (the force's work on the mean flow); rho is unchanged.
template <bool Force, typename C>
LBM13_HD void collide(C f[Q], const Coef<C> &k)
{
    Mom<C> m;
    forward(f, m);
    const C rho = C(1) + m.rho;
    const C inv_rho = C(1) / rho;
    C Fx = C(0), Fy = C(0), jxh = m.jx, jyh = m.jy;
    if (Force) {
        const C w = rho - k.rho_ref;
        Fx = w * k.gx;
        Fy = w * k.gy;
        jxh = m.jx + C(0.5) * Fx;
        jyh = m.jy + C(0.5) * Fy;
    }
    const C Q1 = k.Q10 + k.h1 * m.rho + k.k1 * m.E;
    const C R1 = k.R10 + k.h2 * m.rho + k.k2 * m.E;
    Mom<C> d;
    d.rho = C(0);
    if (Force) {
        d.E = C(13.0 / 4004.0) * ((C(2) * m.jx + Fx) * Fx + (C(2) * m.jy + Fy) * Fy) * inv_rho;
        d.jx = Fx * C(1.0 / 14.0);
        d.jy = Fy * C(1.0 / 14.0);
    } else {
        d.E = C(0);
        d.jx = C(0);
        d.jy = C(0);
    }
    d.eps = k.l_eps * (k.cer * m.rho + k.ceE * m.E - m.eps);
    d.vpi = k.l_vpi * (k.cwr * m.rho + k.cwE * m.E - m.vpi);
    d.qx = k.l_q * (jxh * Q1 - m.qx);
    d.qy = k.l_q * (jyh * Q1 - m.qy);
    d.rx = k.l_r * (jxh * R1 - m.rx);
    d.ry = k.l_r * (jyh * R1 - m.ry);
    d.XX = k.l_XX * ((jxh * jxh - jyh * jyh) * inv_rho - m.XX);
    d.XY = k.l_XY * (jxh * jyh * inv_rho - m.XY);
    d.XXe = -k.l_XXe * m.XXe;
    inverse_add<false>(d, f);
}

// Deviation of the equilibrium populations from w for the conserved values
// rho = 1 + drho, E = E0 + dE, (jx, jy): f_eq - w = M^-1 (m_eq - m_rest).
template <typename C>
LBM13_HD void equilibrium_dev(C drho, C dE, C jx, C jy, const Coef<C> &k, C f[Q])
{
    const C inv_rho = C(1) / (C(1) + drho);
    const C Q1 = k.Q10 + k.h1 * drho + k.k1 * dE;
    const C R1 = k.R10 + k.h2 * drho + k.k2 * dE;
    Mom<C> d;
    d.rho = drho * C(1.0 / 13.0);
    d.E = dE * C(1.0 / 4004.0);
    d.eps = (k.cer * drho + k.ceE * dE) * C(1.0 / 42196.0);
    d.vpi = (k.cwr * drho + k.cwE * dE) * C(1.0 / 548.0);
    d.jx = jx * C(1.0 / 14.0);
    d.jy = jy * C(1.0 / 14.0);
    d.qx = jx * Q1 * C(1.0 / 20.0);
    d.qy = jy * Q1 * C(1.0 / 20.0);
    d.rx = jx * R1 * C(1.0 / 70.0);
    d.ry = jy * R1 * C(1.0 / 70.0);
    d.XX = (jx * jx - jy * jy) * inv_rho * C(1.0 / 68.0);
    d.XY = jx * jy * inv_rho * C(1.0 / 4.0);
    d.XXe = C(0);
#pragma unroll
    for (int j = 0; j < Q; ++j) f[j] = C(0);
    inverse_add<true>(d, f);
}

// Energy-moment deviation of one node: sum_j (-28 + 13 |v_j|^2) df_j.
template <typename C>
LBM13_HD C energy_dev(const C f[Q])
{
    return C(-28) * f[0] + C(-15) * (f[1] + f[2] + f[3] + f[4]) + C(-2) * (f[5] + f[6] + f[7] + f[8]) +
           C(24) * (f[9] + f[10] + f[11] + f[12]);
}

template <typename C>
LBM13_HD C mass_dev(const C f[Q])
{
    return f[0] + ((f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8])) + ((f[9] + f[10]) + (f[11] + f[12]));
}

} // namespace lbm13
