// The interpolation variant of the Legendre stage (Sec. 3.4, "Notes on
// interpolation", Eq. interpolation), built on the host to measure what it
// would cost against the butterfly on HEALPix nodes.  Nothing here runs on
// the device path.
//
// For one chain (order m, parity t: rows l = m + t + 2j, j < n) the variant
// evaluates q at the n positive roots z_i of P_{m+t+2n}^m instead of at the
// Z = 2 Nside half-rings, and then interpolates to the rings:
//   q(y) = sum_i W(y, z_i) q(z_i),  W(y, z) = P_{l*}(y) 2 z / (P'_{l*}(z) (y^2 - z^2)),
// l* = m + t + 2n.  This is Eq. interpolation with omega(y) = P_{l*}(y) and
// gamma(z_i) = 2 z_i / P'_{l*}(z_i): q = y^t (1 - y^2)^{m/2} p(y^2) with p of
// degree < n, and P_{l*} = c y^t (1 - y^2)^{m/2} pi(y^2) with pi vanishing at
// the z_i^2, so Lagrange interpolation of p in x = y^2 gives W (c cancels).
// At a root, (1 - z^2) P'_l(z) = sqrt((2l+1)(l^2 - m^2)/(2l-1)) P_{l-1}(z).
//
// The roots are the positive eigenvalues of the Jacobi matrix of the
// Gegenbauer polynomials C^(m+1/2) of degree t + 2n (zero diagonal,
// off-diagonals b_l = sqrt((l^2 - m^2)/(4 l^2 - 1)), l = m+1 .. l*-1, the
// one-step recurrence coefficients), found one by one by bisection on the
// Sturm count of its LDL^T factorisation.
//
// Costs are counted as stored matrix elements (each one FMA per real
// component of every map, as in the butterfly kernels):
//   * Lambda at the roots (n x n), compressed by the same butterfly builder;
//   * W (Z x n), compressed by the same butterfly builder;
//   * W compressed hierarchically (the algebraic counterpart of the FMM):
//     recursive bisection of the rings and roots by position, each
//     off-diagonal block replaced by its interpolative decomposition;
//   * Lambda at the rings (n x Z), compressed by the butterfly builder (the
//     plan's operator).
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "shtb_butterfly.h"
#include "shtb_plan_detail.h"

namespace shtb {
namespace {

// b_l = sqrt((l^2 - m^2)/(4 l^2 - 1)), l = m+1 .. lmax (index l - m)
std::vector<double> step_coefs(int lmax, int m)
{
    std::vector<double> b(lmax - m + 1, 0.0);
    for (int l = m + 1; l <= lmax; ++l)
        b[l - m] = std::sqrt(((double)l * l - (double)m * m) / (4.0 * (double)l * l - 1.0));
    return b;
}

// number of eigenvalues below x of the symmetric tridiagonal matrix with zero
// diagonal and off-diagonals off[1..D-1]
int sturm_count(const std::vector<double> &off, int D, double x)
{
    int neg = 0;
    double d = -x;
    if (d < 0) ++neg;
    for (int i = 1; i < D; ++i) {
        const double prev = d == 0.0 ? 1e-300 : d;
        d = -x - off[i] * off[i] / prev;
        if (d < 0) ++neg;
    }
    return neg;
}

// the n positive roots of P_{m+t+2n}^m, descending (pole first)
std::vector<double> chain_roots(int m, int t, int n)
{
    const int D = t + 2 * n;                  // degree of the Gegenbauer factor
    const std::vector<double> b = step_coefs(m + D, m);
    std::vector<double> off(D, 0.0);
    for (int i = 1; i < D; ++i) off[i] = b[i];
    std::vector<double> z(n);
    const int nthreads = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int w = 0; w < nthreads; ++w)
        pool.emplace_back([&, w] {
            for (int i = w; i < n; i += nthreads) {
                // the (D - n + i + 1)-th smallest eigenvalue, i ascending
                const int want = D - n + i + 1;
                double lo = 0.0, hi = 1.0;
                for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
                    const double mid = 0.5 * (lo + hi);
                    if (mid <= lo || mid >= hi) break;
                    if (sturm_count(off, D, mid) >= want) hi = mid;
                    else lo = mid;
                }
                z[n - 1 - i] = 0.5 * (lo + hi);
            }
        });
    for (auto &th : pool) th.join();
    return z;
}

// a point of (0, 1) as a ring description for the Legendre column routine
HalfRing point(double z)
{
    HalfRing h;
    h.z = z;
    h.z2 = z * z;
    const DD s2 = ddmul(1.0 - z, 1.0 + z);
    h.s2 = to_double(s2);
    h.eps1 = 1.0 - z;
    h.sdd = sqrt(s2);
    return h;
}

// stored elements of one interpolative decomposition of the rows x cols
// block starting at A (column-major, leading dimension lda): the skeleton
// columns (rows x k) and the interpolation matrix (k x (cols - k))
long long id_cost(const double *A, int rows, int cols, int lda, double eps)
{
    if (rows == 0 || cols == 0) return 0;
    const IdResult id = interp_decomp(A, rows, cols, lda, eps, 1e-30);
    const long long dense = (long long)rows * cols;
    const long long c = (long long)rows * id.k + (long long)id.k * (cols - id.k);
    return std::min(dense, c);
}

// hierarchical compression of W (rows = rings, columns = roots, both in
// descending position; column-major, leading dimension Z)
long long hodlr_cost(const std::vector<double> &W, int Z, const std::vector<double> &y,
                     const std::vector<double> &z, int r0, int r1, int c0, int c1, double eps, int leaf)
{
    const int rows = r1 - r0, cols = c1 - c0;
    if (rows <= leaf || cols <= leaf) return (long long)rows * cols;
    const int rm = (r0 + r1) / 2;
    const double cut = 0.5 * (y[rm - 1] + y[rm]);
    int cm = c0;
    while (cm < c1 && z[cm] > cut) ++cm;
    const double *base = W.data();
    long long cost = id_cost(base + (size_t)cm * Z + r0, rm - r0, c1 - cm, Z, eps) +
                     id_cost(base + (size_t)c0 * Z + rm, r1 - rm, cm - c0, Z, eps);
    cost += hodlr_cost(W, Z, y, z, r0, rm, c0, cm, eps, leaf);
    cost += hodlr_cost(W, Z, y, z, rm, r1, cm, c1, eps, leaf);
    return cost;
}

long long chain_elements(const BfChain &ch)
{
    long long e = 0;
    for (const auto &it : ch.items)
        for (int s = 0; s < 2; ++s) e += (long long)it.T[s].size() + it.k[s];
    for (const auto &rb : ch.rblocks) e += (long long)rb.data.size();
    return e;
}

}  // namespace
}  // namespace shtb

// Host-only measurement of the interpolation variant for one chain: see the
// file comment.  a: the chain's n coefficients; q_interp (Z values) = W
// (Lambda_roots^T a) evaluated densely, q_exact = Lambda_rings^T a; info[0..7]
// = {n, butterfly elements of Lambda at the roots, butterfly elements of W,
// hierarchical elements of W, butterfly elements of Lambda at the rings,
// n Z (the dense operator), n^2 + Z n (the dense two-step variant), depth of
// the rings' butterfly}.
extern "C" int shtb_test_host_interp(int nside, int lmax, double eps, int m, int t, int leaf_cols,
                                     const double *a, double *q_interp, double *q_exact, long long *info)
{
    using namespace shtb;
    if (nside < 1 || lmax < 0 || m < 0 || m > lmax || t < 0 || t > 1 || !(eps > 0) || leaf_cols < 1 ||
        leaf_cols > kMaxCand || !a || !q_interp || !q_exact || !info)
        return shtb_fail(SHTB_EINVAL, "bad arguments");
    const int n = chain_len(lmax, m, t);
    if (n < 1) return shtb_fail(SHTB_EINVAL, "empty chain");
    const int Z = 2 * nside;
    const int lstar = m + t + 2 * n;          // > lmax: its roots are the nodes
    const std::vector<DD> cm = diag_norms(lstar);
    const std::vector<double> b = one_step_coefs(lstar, m);

    // rings and roots, each in descending position
    std::vector<HalfRing> hr(Z);
    std::vector<double> y(Z);
    for (int r = 0; r < Z; ++r) {
        hr[r] = half_ring(nside, r + 1);
        y[r] = hr[r].z;
    }
    const std::vector<double> z = chain_roots(m, t, n);

    // Lambda at the rings and at the roots (column-major, n rows), and the
    // interpolation weights from P_{l*} and P_{l*-1}
    std::vector<double> lam_rings((size_t)n * Z), lam_roots((size_t)n * n), col(lstar - m + 1);
    std::vector<double> omega(Z), gamma(n);
    for (int r = 0; r < Z; ++r) {
        legendre_column(lstar, m, hr[r], cm[m], b, col.data());
        for (int j = 0; j < n; ++j) lam_rings[(size_t)r * n + j] = col[t + 2 * j];
        omega[r] = col[lstar - m];
    }
    const double dl = lstar;
    const double dcoef = std::sqrt((2.0 * dl + 1.0) * (dl * dl - (double)m * m) / (2.0 * dl - 1.0));
    for (int i = 0; i < n; ++i) {
        legendre_column(lstar, m, point(z[i]), cm[m], b, col.data());
        for (int j = 0; j < n; ++j) lam_roots[(size_t)i * n + j] = col[t + 2 * j];
        const double dP = dcoef * col[lstar - 1 - m] / ((1.0 - z[i]) * (1.0 + z[i]));
        gamma[i] = 2.0 * z[i] / dP;
    }
    std::vector<double> W((size_t)Z * n);     // column-major: W[i * Z + r]
    for (int i = 0; i < n; ++i)
        for (int r = 0; r < Z; ++r) W[(size_t)i * Z + r] = omega[r] * gamma[i] / (y[r] * y[r] - z[i] * z[i]);

    // both routes, densely
    std::vector<double> qz(n);
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += lam_roots[(size_t)i * n + j] * a[j];
        qz[i] = s;
    }
    for (int r = 0; r < Z; ++r) {
        double s = 0.0, e = 0.0;
        for (int i = 0; i < n; ++i) s += W[(size_t)i * Z + r] * qz[i];
        for (int j = 0; j < n; ++j) e += lam_rings[(size_t)r * n + j] * a[j];
        q_interp[r] = s;
        q_exact[r] = e;
    }

    // compressed sizes
    BfParams prm;
    prm.eps = eps;
    prm.leaf_cols = leaf_cols;
    BfChain c_rings, c_roots, c_w;
    compress_chain(lam_rings.data(), n, Z, prm, &c_rings);
    compress_chain(lam_roots.data(), n, n, prm, &c_roots);
    std::vector<double> wt((size_t)n * Z);    // W^T as the n x Z operator of q_roots
    for (int i = 0; i < n; ++i)
        for (int r = 0; r < Z; ++r) wt[(size_t)r * n + i] = W[(size_t)i * Z + r];
    compress_chain(wt.data(), n, Z, prm, &c_w);
    info[0] = n;
    info[1] = chain_elements(c_roots);
    info[2] = chain_elements(c_w);
    info[3] = hodlr_cost(W, Z, y, z, 0, Z, 0, n, eps, leaf_cols);
    info[4] = chain_elements(c_rings);
    info[5] = (long long)n * Z;
    info[6] = (long long)n * n + (long long)Z * n;
    info[7] = c_rings.depth;
    return SHTB_OK;
}
