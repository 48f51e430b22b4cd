// lbm13_linear.cu -- linear stability of the time step about a uniform state:
// one scan on the host (linear_growth) and many scans at once on the GPU
// (linear_growth_batch), with the same eigenvalue code.
//
// End of Sec. 2: the free parameters are chosen by computing the roots of the
// dispersion equation for wave vectors of magnitude 0 .. 2 pi in several
// directions.  Linearised about (rho, j, E) = (1, U, E0 + 13 |U|^2), the
// collision is f* = J f with J = M^-1 (I - S + S G) M, G the derivative of the
// equilibria of Eq. (d2q13-moments-equil) with respect to the moments; pulling
// a Fourier mode exp(i k.x) along link j multiplies population j by
// exp(-i k.v_j).  The scan takes the largest eigenvalue modulus of
// diag(exp(-i k.v)) J over an n x n grid of k in [-pi, pi]^2; the step is
// linearly stable when it does not exceed 1.
//
// Eigenvalues: Householder reduction to upper Hessenberg form, then the
// shifted QR iteration with Givens rotations, Wilkinson shifts and deflation
// (the textbook complex QR algorithm), on 13 x 13 matrices.  The routines are
// host and device code (cuda::std::complex), so the GPU scan runs exactly the
// algorithm of the host scan.
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda/std/complex>

#include "lbm13_internal.h"

namespace lbm13 {

namespace {

using cplx = cuda::std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

// Upper Hessenberg form by Householder reflections (similarity transform).
__host__ __device__ void hessenberg(cplx A[Q][Q])
{
    using cuda::std::abs;
    using cuda::std::conj;
    using cuda::std::norm;
    for (int k = 0; k < Q - 2; ++k) {
        double norm2 = 0.0;
        for (int i = k + 1; i < Q; ++i) norm2 += norm(A[i][k]);
        const double nrm = sqrt(norm2);
        if (nrm == 0.0) continue;
        const cplx x0 = A[k + 1][k];
        const cplx phase = abs(x0) > 0.0 ? x0 / abs(x0) : cplx(1.0, 0.0);
        cplx v[Q] = {};
        for (int i = k + 1; i < Q; ++i) v[i] = A[i][k];
        v[k + 1] += phase * nrm;
        double vn2 = 0.0;
        for (int i = k + 1; i < Q; ++i) vn2 += norm(v[i]);
        if (vn2 == 0.0) continue;
        // A <- (I - 2 v v^H / |v|^2) A (I - 2 v v^H / |v|^2)
        for (int j = 0; j < Q; ++j) {
            cplx s = 0.0;
            for (int i = k + 1; i < Q; ++i) s += conj(v[i]) * A[i][j];
            s *= 2.0 / vn2;
            for (int i = k + 1; i < Q; ++i) A[i][j] -= v[i] * s;
        }
        for (int i = 0; i < Q; ++i) {
            cplx s = 0.0;
            for (int j = k + 1; j < Q; ++j) s += A[i][j] * v[j];
            s *= 2.0 / vn2;
            for (int j = k + 1; j < Q; ++j) A[i][j] -= s * conj(v[j]);
        }
        for (int i = k + 2; i < Q; ++i) A[i][k] = 0.0;
    }
}

// Eigenvalues of an upper Hessenberg matrix (destroyed).  Returns false if
// an eigenvalue did not converge within the iteration limit.
__host__ __device__ bool hessenberg_eigenvalues(cplx H[Q][Q], cplx w[Q])
{
    using cuda::std::abs;
    using cuda::std::conj;
    using cuda::std::norm;
    const double eps = 1e-15;
    int hi = Q - 1, iter = 0;
    while (hi >= 0) {
        if (hi == 0) {
            w[0] = H[0][0];
            break;
        }
        int l = hi;
        while (l > 0) {
            const double scale = abs(H[l - 1][l - 1]) + abs(H[l][l]);
            if (abs(H[l][l - 1]) <= eps * (scale > 0.0 ? scale : 1.0)) {
                H[l][l - 1] = 0.0;
                break;
            }
            --l;
        }
        if (l == hi) {
            w[hi] = H[hi][hi];
            --hi;
            iter = 0;
            continue;
        }
        if (++iter > 400) return false;
        // Wilkinson shift from the trailing 2 x 2 block (an exceptional shift
        // every 12 iterations breaks cycles)
        const cplx a = H[hi - 1][hi - 1], b = H[hi - 1][hi], c = H[hi][hi - 1], d = H[hi][hi];
        cplx mu;
        if (iter % 12 == 0) {
            mu = d + abs(H[hi][hi - 1]);
        } else {
            const cplx half = 0.5 * (a - d);
            const cplx disc = cuda::std::sqrt(half * half + b * c);
            const cplx m1 = d - b * c / (half + disc), m2 = d - b * c / (half - disc);
            const bool ok1 = isfinite(m1.real()) && isfinite(m1.imag());
            const bool ok2 = isfinite(m2.real()) && isfinite(m2.imag());
            if (ok1 && (!ok2 || abs(m1 - d) <= abs(m2 - d))) mu = m1;
            else if (ok2) mu = m2;
            else mu = d;
        }
        // one QR step on the active block l..hi: H - mu I = Q R, H <- R Q + mu I
        for (int k = l; k <= hi; ++k) H[k][k] -= mu;
        cplx gc[Q], gs[Q];
        for (int k = l; k < hi; ++k) {
            const cplx x = H[k][k], y = H[k + 1][k];
            const double r = cuda::std::sqrt(norm(x) + norm(y));
            const cplx cc = r > 0.0 ? x / r : cplx(1.0, 0.0), ss = r > 0.0 ? y / r : cplx(0.0, 0.0);
            gc[k] = cc;
            gs[k] = ss;
            for (int j = k; j <= hi; ++j) {
                const cplx u = H[k][j], v = H[k + 1][j];
                H[k][j] = conj(cc) * u + conj(ss) * v;
                H[k + 1][j] = -ss * u + cc * v;
            }
        }
        for (int k = l; k < hi; ++k) {
            const cplx cc = gc[k], ss = gs[k];
            const int top = k + 2 < hi ? k + 2 : hi;
            for (int i = l; i <= top; ++i) {
                const cplx u = H[i][k], v = H[i][k + 1];
                H[i][k] = u * cc + v * ss;
                H[i][k + 1] = -u * conj(ss) + v * conj(cc);
            }
        }
        for (int k = l; k <= hi; ++k) H[k][k] += mu;
    }
    return true;
}

// Collision Jacobian in population space about rho = 1, j = (ux, uy),
// E = E0 + 13 |u|^2 (no force), from the derived constants of lbm13_derive.
void collision_jacobian(const lbm13_params &p, const double *D, double ux, double uy, double J[Q][Q])
{
    // M from the structured transform: column j = forward(e_j)
    double M[Q][Q];
    for (int j = 0; j < Q; ++j) {
        double e[Q] = {};
        e[j] = 1.0;
        Mom<double> m;
        forward(e, m);
        const double col[Q] = {m.rho, m.E, m.eps, m.vpi, m.jx, m.jy, m.qx, m.qy, m.rx, m.ry, m.XX, m.XY, m.XXe};
        for (int k = 0; k < Q; ++k) M[k][j] = col[k];
    }
    const double h1 = D[2], k1 = D[3], h2 = D[4], c2 = D[5], cer = D[6];
    const double *s = D + 9;
    const double rho = 1.0, jx = ux, jy = uy;
    const double E = p.E0 + 13.0 * (jx * jx + jy * jy);
    // G = d m_eq / d m (columns: the conserved rho 0, E 1, jx 4, jy 5)
    double G[Q][Q] = {};
    G[2][0] = cer;
    G[2][1] = p.c_epsE;
    G[3][0] = p.c_vpi_rho;
    G[3][1] = p.c_vpi_E;
    const double qf = p.c1 + h1 * rho + k1 * E, rf = c2 + h2 * rho + p.k2 * E;
    const int kq[2] = {6, 7}, kr[2] = {8, 9}, kj[2] = {4, 5};
    const double jv[2] = {jx, jy};
    for (int a = 0; a < 2; ++a) {
        G[kq[a]][kj[a]] = qf;
        G[kq[a]][0] = jv[a] * h1;
        G[kq[a]][1] = jv[a] * k1;
        G[kr[a]][kj[a]] = rf;
        G[kr[a]][0] = jv[a] * h2;
        G[kr[a]][1] = jv[a] * p.k2;
    }
    G[10][4] = 2.0 * jx / rho;
    G[10][5] = -2.0 * jy / rho;
    G[10][0] = -(jx * jx - jy * jy) / (rho * rho);
    G[11][4] = jy / rho;
    G[11][5] = jx / rho;
    G[11][0] = -jx * jy / (rho * rho);
    // K = I - S + S G (moment space), then J = M^T D^-1 K M
    double K[Q][Q];
    for (int r = 0; r < Q; ++r)
        for (int c = 0; c < Q; ++c) K[r][c] = (r == c ? 1.0 - s[r] : 0.0) + s[r] * G[r][c];
    double KM[Q][Q];
    for (int r = 0; r < Q; ++r)
        for (int c = 0; c < Q; ++c) {
            double t = 0.0;
            for (int m = 0; m < Q; ++m) t += K[r][m] * M[m][c];
            KM[r][c] = t;
        }
    for (int r = 0; r < Q; ++r)
        for (int c = 0; c < Q; ++c) {
            double t = 0.0;
            for (int m = 0; m < Q; ++m) t += M[m][r] / kD[m] * KM[m][c];
            J[r][c] = t;
        }
}

// Largest |z| of the amplification matrix diag(exp(-i k.v)) J at grid point
// (a, b) of the n x n k-grid of [-pi, pi]^2 (k = 0 for n = 1); negative when
// the eigenvalue iteration failed.
__host__ __device__ double grid_point_zmax(const double J[Q][Q], int n, int a, int b)
{
    const double kx = n > 1 ? -kPi + 2.0 * kPi * a / (n - 1) : 0.0;
    const double ky = n > 1 ? -kPi + 2.0 * kPi * b / (n - 1) : 0.0;
    cplx A[Q][Q];
    for (int r = 0; r < Q; ++r) {
        const cplx ph = cuda::std::exp(cplx(0.0, -(kx * cvx(r) + ky * cvy(r))));
        for (int c = 0; c < Q; ++c) A[r][c] = ph * J[r][c];
    }
    hessenberg(A);
    cplx w[Q];
    if (!hessenberg_eigenvalues(A, w)) return -1.0;
    double z = 0.0;
    for (int i = 0; i < Q; ++i) z = fmax(z, cuda::std::abs(w[i]));
    return z;
}

// One thread per (case, grid point): the case's largest |z| by an atomic max
// on the bit pattern (order-preserving for doubles >= 0); a failed
// eigenvalue iteration sets *fail.
__global__ void __launch_bounds__(128) growth_kernel(const double *__restrict__ J, int count, int n,
                                                     unsigned long long *zmax, int *fail)
{
    const long long per = (long long)n * n;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= per * count) return;
    const int c = int(t / per);
    const int kk = int(t - (long long)c * per);
    double Jc[Q][Q];
    for (int r = 0; r < Q; ++r)
        for (int q = 0; q < Q; ++q) Jc[r][q] = J[((long long)c * Q + r) * Q + q];
    const double z = grid_point_zmax(Jc, n, kk / n, kk % n);
    if (z < 0.0) {
        atomicOr(fail, 1);
        return;
    }
    atomicMax(zmax + c, static_cast<unsigned long long>(__double_as_longlong(z)));
}

} // namespace

int linear_growth(const lbm13_params &p, const double *D, double ux, double uy, int n, double *growth)
{
    double J[Q][Q];
    collision_jacobian(p, D, ux, uy, J);
    double worst = -1.0;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            const double z = grid_point_zmax(J, n, a, b);
            if (z < 0.0) return LBM13_EINVAL;
            worst = std::fmax(worst, z - 1.0);
        }
    *growth = worst;
    return LBM13_OK;
}

int linear_growth_batch(const lbm13_params *p, const double *D, const double *ux, const double *uy, int count, int n,
                        double *growth, cudaStream_t s)
{
    std::vector<double> J(size_t(count) * Q * Q);
    for (int c = 0; c < count; ++c)
        collision_jacobian(p[c], D + size_t(c) * LBM13_DERIVED_COUNT, ux[c], uy[c],
                           reinterpret_cast<double(*)[Q]>(J.data() + size_t(c) * Q * Q));
    double *dJ = nullptr;
    unsigned long long *dz = nullptr;
    int *dfail = nullptr;
    cudaError_t e = cudaMallocAsync(&dJ, J.size() * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&dz, size_t(count) * sizeof(unsigned long long) + sizeof(int), s);
    if (e == cudaSuccess) {
        dfail = reinterpret_cast<int *>(dz + count);
        e = cudaMemcpyAsync(dJ, J.data(), J.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(dz, 0, size_t(count) * sizeof(unsigned long long) + sizeof(int), s);
    if (e == cudaSuccess) {
        const long long threads = (long long)count * n * n;
        growth_kernel<<<unsigned((threads + 127) / 128), 128, 0, s>>>(dJ, count, n, dz, dfail);
        e = cudaGetLastError();
    }
    std::vector<unsigned long long> zb(size_t(count) + 1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(zb.data(), dz, size_t(count) * sizeof(unsigned long long) + sizeof(int),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (dJ) cudaFreeAsync(dJ, s);
    if (dz) cudaFreeAsync(dz, s);
    if (e != cudaSuccess) return LBM13_ECUDA;
    int failed = 0;
    std::memcpy(&failed, zb.data() + count, sizeof(int));
    if (failed) return LBM13_EINVAL;
    for (int c = 0; c < count; ++c) {
        double z;
        std::memcpy(&z, &zb[size_t(c)], sizeof z);
        growth[c] = z - 1.0;
    }
    return LBM13_OK;
}

} // namespace lbm13
