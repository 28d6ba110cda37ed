// The k smallest eigenpairs of a symmetric tridiagonal matrix (host code): the
// Lanczos matrix T of a PCG run, from which cr_deflation_lanczos and cr_solve_ritz
// take Ritz vectors.  Eigenvalues by bisection on Sturm counts of the LDL^t pivots,
// eigenvectors by inverse iteration with partial pivoting, each orthogonalised
// against those found before it.  Plain C++, no CUDA: the CPU tests compile it.
#pragma once

#include <cmath>
#include <utility>
#include <vector>

namespace crhyb {
namespace tridiag_detail {

// Number of eigenvalues of the symmetric tridiagonal (a, b) below x (Sturm count of
// the LDL^t pivots of T - x I).
inline int sturm_below(const std::vector<double>& a, const std::vector<double>& b, double x) {
    int cnt = 0;
    double d = 1.0;
    const size_t n = a.size();
    for (size_t i = 0; i < n; ++i) {
        const double off = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
        d = a[i] - x - (i > 0 ? off / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// Solve (T - s I) y = v for symmetric tridiagonal T by Gaussian elimination with
// partial pivoting (the factor gains a second superdiagonal).
inline void tridiag_solve(const std::vector<double>& a, const std::vector<double>& b, double s, std::vector<double>& y) {
    const size_t n = a.size();
    std::vector<double> dl(n, 0.0), d(n), du(n, 0.0), du2(n, 0.0);
    for (size_t i = 0; i < n; ++i) {
        d[i] = a[i] - s;
        if (i + 1 < n) du[i] = b[i], dl[i] = b[i];
    }
    for (size_t i = 0; i + 1 < n; ++i) {
        if (std::fabs(d[i]) >= std::fabs(dl[i])) {
            if (d[i] == 0.0) d[i] = 1e-300;
            const double f = dl[i] / d[i];
            d[i + 1] -= f * du[i];
            y[i + 1] -= f * y[i];
            dl[i] = 0.0;
        } else {   // swap rows i and i+1
            const double f = d[i] / dl[i];
            d[i] = dl[i];
            const double t = d[i + 1];
            d[i + 1] = du[i] - f * t;
            du[i] = t;
            if (i + 2 < n) {
                du2[i] = du[i + 1];
                du[i + 1] = -f * du2[i];
            }
            std::swap(y[i], y[i + 1]);
            y[i + 1] -= f * y[i];
        }
    }
    if (d[n - 1] == 0.0) d[n - 1] = 1e-300;
    y[n - 1] /= d[n - 1];
    if (n > 1) y[n - 2] = (y[n - 2] - du[n - 2] * y[n - 1]) / d[n - 2];
    for (size_t i = n >= 3 ? n - 3 : 0; n >= 3; --i) {
        y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) / d[i];
        if (i == 0) break;
    }
}

}  // namespace tridiag_detail

// The k smallest eigenpairs of the symmetric tridiagonal matrix with diagonal a and
// off-diagonal b: eigenvalues by bisection on Sturm counts, eigenvectors by inverse
// iteration, orthogonalised against those already found (S column-major [n][k]:
// S[t * k + l] is component t of vector l).
inline void tridiag_smallest_eigen(const std::vector<double>& a, const std::vector<double>& b, int k,
                            std::vector<double>& theta, std::vector<double>& S) {
    const int n = int(a.size());
    k = k < n ? k : n;
    double lo = a[0], hi = a[0];
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(b[i]) : 0.0);
        lo = std::fmin(lo, a[i] - r);
        hi = std::fmax(hi, a[i] + r);
    }
    const double span = std::fmax(hi - lo, 1e-300);
    theta.assign(k, 0.0);
    S.assign(size_t(n) * k, 0.0);
    std::vector<std::vector<double>> vecs;
    for (int l = 0; l < k; ++l) {
        double x0 = lo, x1 = hi;   // the (l+1)-th smallest eigenvalue lies in [x0, x1]
        for (int it = 0; it < 200 && x1 - x0 > 1e-15 * std::fmax(std::fabs(x0) + std::fabs(x1), span * 1e-300); ++it) {
            const double mid = 0.5 * (x0 + x1);
            if (tridiag_detail::sturm_below(a, b, mid) > l) x1 = mid;
            else x0 = mid;
        }
        const double th = 0.5 * (x0 + x1);
        theta[l] = th;
        std::vector<double> y(n);
        for (int t = 0; t < n; ++t) y[t] = 1.0 + 0.001 * ((t * 7919) % 13);   // a start with every component
        const double shift = th - 1e-13 * span;
        for (int it = 0; it < 4; ++it) {
            tridiag_detail::tridiag_solve(a, b, shift, y);
            for (const auto& v : vecs) {   // the eigenvectors of nearby eigenvalues, projected out
                double dot = 0.0;
                for (int t = 0; t < n; ++t) dot += v[t] * y[t];
                for (int t = 0; t < n; ++t) y[t] -= dot * v[t];
            }
            double nrm = 0.0;
            for (int t = 0; t < n; ++t) nrm += y[t] * y[t];
            nrm = std::sqrt(nrm);
            if (!(nrm > 0.0)) break;
            for (int t = 0; t < n; ++t) y[t] /= nrm;
        }
        for (int t = 0; t < n; ++t) S[size_t(t) * k + l] = y[t];
        vecs.push_back(y);
    }
}

}  // namespace crhyb
