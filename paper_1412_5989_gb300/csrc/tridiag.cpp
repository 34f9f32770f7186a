// Symmetric tridiagonal eigensolver used by the Lanczos driver (host side).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "cih_internal.h"

namespace cih {

// Symmetric tridiagonal eigenproblem (diagonal d, off-diagonal e) by
// implicit QR steps with Wilkinson shifts, chasing the bulge with Givens
// rotations.  Each rotation of columns (k, k + 1) is applied to rows
// row0..n-1 of Z (row0 = 0: the eigenvectors; row0 = n - 1: only their last
// components, which is all the Lanczos residual bounds need).  Eigenvalues
// are returned ascending, Z's columns permuted to match.
static void qr_sweeps(int n, std::vector<double> &d, std::vector<double> e, std::vector<double> &Z, int row0)
{
    const int nrows = n - row0;
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, guard = 0;
    while (hi > 0 && guard < 64 * n + 100) {
        if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
            e[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
        ++guard;
        double t = 0.5 * (d[hi - 1] - d[hi]), b2 = e[hi - 1] * e[hi - 1];
        double root = std::sqrt(t * t + b2);
        double mu = d[hi] - b2 / (t + (t >= 0 ? root : -root));
        double x = d[lo] - mu, z = e[lo];
        for (int k = lo; k < hi; ++k) {
            double r = std::hypot(x, z);
            double c = r == 0.0 ? 1.0 : x / r, s = r == 0.0 ? 0.0 : z / r;
            if (k > lo) e[k - 1] = r;
            double dk = d[k], dk1 = d[k + 1], ek = e[k];
            d[k] = c * c * dk + 2.0 * c * s * ek + s * s * dk1;
            d[k + 1] = s * s * dk - 2.0 * c * s * ek + c * c * dk1;
            e[k] = c * s * (dk1 - dk) + (c * c - s * s) * ek;
            if (k + 1 < hi) {
                x = e[k];
                z = s * e[k + 1];
                e[k + 1] *= c;
            }
            for (int i = 0; i < nrows; ++i) {
                double zk = Z[(size_t)i * n + k], zk1 = Z[(size_t)i * n + k + 1];
                Z[(size_t)i * n + k] = c * zk + s * zk1;
                Z[(size_t)i * n + k + 1] = -s * zk + c * zk1;
            }
        }
    }
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return d[a] < d[b]; });
    std::vector<double> d2(n), Z2((size_t)nrows * n);
    for (int j = 0; j < n; ++j) {
        d2[j] = d[ord[j]];
        for (int i = 0; i < nrows; ++i) Z2[(size_t)i * n + j] = Z[(size_t)i * n + ord[j]];
    }
    d.swap(d2);
    Z.swap(Z2);
}

void tridiag_qr(int n, std::vector<double> &d, std::vector<double> e, std::vector<double> &Z)
{
    Z.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
    qr_sweeps(n, d, std::move(e), Z, 0);
}

// Eigenvalues ascending (into d) and the last component of each eigenvector
// (into zlast): the QR sweeps above with only the last row of Z rotated.
void tridiag_qr_last(int n, std::vector<double> &d, std::vector<double> e, std::vector<double> &zlast)
{
    zlast.assign((size_t)n, 0.0);
    zlast[(size_t)n - 1] = 1.0;
    qr_sweeps(n, d, std::move(e), zlast, n - 1);
}

// normalised eigenvector for the eigenvalue estimate theta: three steps of
// inverse iteration, (T - theta I) z_new = z, solved by Gaussian elimination
// with partial pivoting on the tridiagonal
void tridiag_eigenvector(int n, const double *d, const double *e, double theta, double *z)
{
    std::vector<double> a(n), b(n), c(n);     // sub, main, super
    const double scale = 1e-14 * (std::fabs(theta) + 1.0);
    for (int k = 0; k < n; ++k) z[k] = 1.0 / std::sqrt((double)n) * (1.0 + 0.1 * ((k * 7919) % 13));
    for (int step = 0; step < 3; ++step) {
        for (int k = 0; k < n; ++k) {
            a[k] = k ? e[k - 1] : 0.0;
            b[k] = d[k] - theta;
            c[k] = k + 1 < n ? e[k] : 0.0;
            if (b[k] == 0.0) b[k] = scale;
        }
        // elimination with pivoting: rows k and k+1, keeping two superdiagonals
        std::vector<double> r2(n, 0.0), rhs(z, z + n);
        for (int k = 0; k + 1 < n; ++k) {
            if (std::fabs(a[k + 1]) > std::fabs(b[k])) {       // swap rows k and k+1
                std::swap(b[k], a[k + 1]);
                std::swap(c[k], b[k + 1]);
                std::swap(r2[k], c[k + 1]);
                std::swap(rhs[k], rhs[k + 1]);
            }
            if (b[k] == 0.0) b[k] = scale;
            const double f = a[k + 1] / b[k];
            b[k + 1] -= f * c[k];
            c[k + 1] -= f * r2[k];
            rhs[k + 1] -= f * rhs[k];
            a[k + 1] = 0.0;
        }
        if (b[n - 1] == 0.0) b[n - 1] = scale;
        for (int k = n - 1; k >= 0; --k) {
            double x = rhs[k];
            if (k + 1 < n) x -= c[k] * z[k + 1];
            if (k + 2 < n) x -= r2[k] * z[k + 2];
            z[k] = x / b[k];
        }
        double nrm = 0.0;
        for (int k = 0; k < n; ++k) nrm += z[k] * z[k];
        nrm = std::sqrt(nrm);
        for (int k = 0; k < n; ++k) z[k] /= nrm;
    }
}

}  // namespace cih

extern "C" int cih_tridiag_eigen(int32_t n, const double *diag, const double *offdiag, double *evals,
                                 double *evecs)
{
    if (n < 1 || !diag || !evals || (n > 1 && !offdiag)) return cih::fail(CIH_ERR_ARG, "bad tridiagonal");
    try {
        std::vector<double> d(diag, diag + n), e(offdiag ? offdiag : diag, offdiag ? offdiag + (n - 1) : diag);
        if (e.empty()) e.push_back(0.0);
        std::vector<double> Z;
        cih::tridiag_qr(n, d, e, Z);
        std::copy(d.begin(), d.end(), evals);
        if (evecs) std::copy(Z.begin(), Z.end(), evecs);
    } catch (...) {
        return cih::fail(CIH_ERR_NOMEM, "host allocation failed");
    }
    return CIH_OK;
}
