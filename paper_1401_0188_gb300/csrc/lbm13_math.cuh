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

#include <cmath>

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
    // Collision only: Q10 and R10 at E0 + 13 q (equilibria half-way through
    // the energy source q), and the increments of the four shells from the
    // source (26 q on E, the shifted eps and varpi equilibria); Qh = Q10,
    // Rh = R10 and src = 0 without a source.
    C Qh, Rh;
    C src[4];
    // The relaxation of eps and varpi is linear in the four shell sums
    // (f0, unit axes, diagonals, distance-2 axes): B[s][l] gives the increment
    // of every population of shell s per unit of shell sum l.
    C B[4][4];
    // XX and XXe relax linearly in X1 = (f1+f3)-(f2+f4) and X9 = (f9+f11)-(f10+f12):
    // t1 = l_XX XX_eq + t1X1 X1 + t1X9 X9, t9 = 4 l_XX XX_eq + t9X1 X1 + t9X9 X9.
    C t1X1, t1X9, t9X1, t9X9;
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

// 1/x: an FP32 reciprocal as the seed, then Newton's iteration for 1/x,
// r <- r + r (1 - x r), which squares the relative error each time (two steps
// take 2^-23 below double rounding).  FP32 uses its own division.
LBM13_HD double recip(double x)
{
#ifdef __CUDA_ARCH__
    double r = double(1.0f / float(x));
    r = fma(r, fma(-x, r, 1.0), r);
    r = fma(r, fma(-x, r, 1.0), r);
    return r;
#else
    return 1.0 / x;
#endif
}
LBM13_HD float recip(float x) { return 1.0f / x; }

// 1/rho for the collision, where it only scales second-order terms (the
// momentum-flux equilibria j_x^2 - j_y^2 and j_x j_y, the force's work): one
// Newton step after the FP32 seed leaves a relative error near 2^-47, i.e.
// below 1e-18 in those terms at |u| ~ 0.01.  FP32 takes CUDA's fast division
// (__fdividef, within 2 ulp for divisors in [2^-126, 2^126]): a relative
// error of about 2.4e-7 in terms no larger than the deviations they are added
// to, i.e. at the level of those deviations' own FP32 rounding; every kernel
// rounds it the same way.
LBM13_HD double recip_uu(double x)
{
#ifdef __CUDA_ARCH__
    const double r = double(1.0f / float(x));
    return fma(r, fma(-x, r, 1.0), r);
#else
    return 1.0 / x;
#endif
}
LBM13_HD float recip_uu(float x)
{
#ifdef __CUDA_ARCH__
    return __fdividef(1.0f, x);
#else
    return 1.0f / x;
#endif
}

// Explicitly rounded products for the collision.  Every product in collide
// is written as rn_mul (never merged with an addition) or rn_fma (one
// rounding), so the compiler neither contracts nor splits any of them: the
// collision rounds identically in every kernel that inlines it, wherever that
// kernel holds the coefficients (kernel parameters, shared memory or
// registers).  Sums need no wrapper: a lone addition cannot be contracted and
// nothing is reassociated.
LBM13_HD float rn_mul(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
LBM13_HD double rn_mul(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
LBM13_HD float rn_fma(float a, float b, float c)
{
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}
LBM13_HD double rn_fma(double a, double b, double c)
{
#ifdef __CUDA_ARCH__
    return __fma_rn(a, b, c);
#else
    return fma(a, b, c);
#endif
}

// One collision in place (deviation form).  Equilibria of Sec. 2, Eq.
// (d2q13-moments-equil) at j + F/2 and E + 13 q; the nine non-conserved
// moments relax as m* = m + s (m_eq - m); j* = j + F and
// E* = E + 13 (|j + F|^2 - |j|^2)/rho + 26 q (the force's work on the mean
// flow and the energy source q of Sec. 9); rho is unchanged.  Force selects
// the instantiation that carries the body force and the energy source.
template <bool Force, typename C>
LBM13_HD void collide(C f[Q], const Coef<C> &k)
{
    // pair sums and differences of opposite links, then shell sums
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
    // conserved and odd moments (deviations)
    const C drho = f[0] + S1 + S5 + S9;
    const C dE = rn_fma(C(24), S9, rn_fma(C(-2), S5, rn_fma(C(-15), S1, rn_mul(C(-28), f[0]))));
    const C jx = rn_fma(C(2), b9, b1 + dm);
    const C jy = rn_fma(C(2), b10, b2 + dp);
    const C qx = rn_fma(C(2), b9, rn_fma(C(-2), b1, -dm));
    const C qy = rn_fma(C(2), b10, rn_fma(C(-2), b2, -dp));
    const C rx = rn_fma(C(-3), dm, rn_mul(C(4), b1)) + b9;
    const C ry = rn_fma(C(-3), dp, rn_mul(C(4), b2)) + b10;
    const C rho = C(1) + drho;
    const C inv_rho = recip_uu(rho);
    C Fx = C(0), Fy = C(0), jxh = jx, jyh = jy;
    if (Force) {
        const C w = rho - k.rho_ref;
        Fx = rn_mul(w, k.gx);
        Fy = rn_mul(w, k.gy);
        jxh = rn_fma(C(0.5), Fx, jx);
        jyh = rn_fma(C(0.5), Fy, jy);
    }
    const C Q1 = rn_fma(k.k1, dE, rn_fma(k.h1, drho, k.Qh));
    const C R1 = rn_fma(k.k2, dE, rn_fma(k.h2, drho, k.Rh));
    // scalar block: eps and varpi relax toward c rho + c' E (linear in the shells)
    C i0 = rn_fma(k.B[0][3], S9, rn_fma(k.B[0][2], S5, rn_fma(k.B[0][1], S1, rn_mul(k.B[0][0], f[0]))));
    C i1 = rn_fma(k.B[1][3], S9, rn_fma(k.B[1][2], S5, rn_fma(k.B[1][1], S1, rn_mul(k.B[1][0], f[0]))));
    C i5 = rn_fma(k.B[2][3], S9, rn_fma(k.B[2][2], S5, rn_fma(k.B[2][1], S1, rn_mul(k.B[2][0], f[0]))));
    C i9 = rn_fma(k.B[3][3], S9, rn_fma(k.B[3][2], S5, rn_fma(k.B[3][1], S1, rn_mul(k.B[3][0], f[0]))));
    C djx = C(0), djy = C(0);
    if (Force) {
        // j* = j + F and E* = E + 13 (|j + F|^2 - |j|^2) / rho
        const C tx = rn_fma(C(2), jx, Fx), ty = rn_fma(C(2), jy, Fy);
        const C dEF = rn_mul(rn_mul(C(13.0 / 4004.0), rn_fma(tx, Fx, rn_mul(ty, Fy))), inv_rho);
        i0 = i0 + rn_fma(C(-28), dEF, k.src[0]);
        i1 = i1 + rn_fma(C(-15), dEF, k.src[1]);
        i5 = i5 + rn_fma(C(-2), dEF, k.src[2]);
        i9 = i9 + rn_fma(C(24), dEF, k.src[3]);
        djx = rn_mul(Fx, C(1.0 / 14.0));
        djy = rn_mul(Fy, C(1.0 / 14.0));
    }
    // odd block: q and r relax toward j (c + h rho + k E), at j + F/2
    const C dqx = rn_mul(k.l_q, rn_fma(jxh, Q1, -qx)), dqy = rn_mul(k.l_q, rn_fma(jyh, Q1, -qy));
    const C drx = rn_mul(k.l_r, rn_fma(jxh, R1, -rx)), dry = rn_mul(k.l_r, rn_fma(jyh, R1, -ry));
    // tensor block: XX, XY toward the momentum flux, XXe toward 0
    const C XXeq = rn_mul(rn_fma(jxh, jxh, -rn_mul(jyh, jyh)), inv_rho);
    const C XXl = rn_mul(k.l_XX, XXeq);
    const C t1 = rn_fma(k.t1X9, X9, rn_fma(k.t1X1, X1, XXl));
    const C t9 = rn_fma(k.t9X9, X9, rn_fma(k.t9X1, X1, rn_mul(C(4), XXl)));
    const C dXY = rn_mul(k.l_XY, rn_fma(rn_mul(jxh, jyh), inv_rho, -X5));
    // back to populations through the pairs
    const C o1 = rn_fma(C(4), drx, rn_fma(C(-2), dqx, djx));
    const C o2 = rn_fma(C(4), dry, rn_fma(C(-2), dqy, djy));
    const C sj = djx + djy, dj = djy - djx;
    const C sq = dqx + dqy, dq = dqx - dqy;
    const C sr = drx + dry, dr = drx - dry;
    const C o5 = rn_fma(C(-3), sr, sj - sq);
    const C o6 = rn_fma(C(3), dr, dj + dq);
    const C o9 = rn_fma(C(2), djx + dqx, drx);
    const C o10 = rn_fma(C(2), djy + dqy, dry);
    const C e13 = i1 + t1, e24 = i1 - t1;
    const C e57 = i5 + dXY, e68 = i5 - dXY;
    const C e911 = i9 + t9, e1012 = i9 - t9;
    f[0] += i0;
    f[1] += e13 + o1;
    f[3] += e13 - o1;
    f[2] += e24 + o2;
    f[4] += e24 - o2;
    f[5] += e57 + o5;
    f[7] += e57 - o5;
    f[6] += e68 + o6;
    f[8] += e68 - o6;
    f[9] += e911 + o9;
    f[11] += e911 - o9;
    f[10] += e1012 + o10;
    f[12] += e1012 - o10;
}

// Deviation of the equilibrium populations from w for the conserved values
// rho = 1 + drho, E = E0 + dE, (jx, jy): f_eq - w = M^-1 (m_eq - m_rest).
template <typename C>
LBM13_HD void equilibrium_dev(C drho, C dE, C jx, C jy, const Coef<C> &k, C f[Q])
{
    const C inv_rho = recip(C(1) + drho);
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
