// Guided modes of an x-invariant cross-section, for eigenmode sources and
// mode-overlap monitors (the multi-mode devices of Sec. III).  Host code, double
// precision; set-up work, not part of a design iteration.
//
// A guide eps[i][j] = eps_line[j] carries source-free fields
// E[i][j] = phi[j] exp(-i theta i) of the FDFD operator of Eq. 1-2 when phi is an
// eigenvector of H = k0dx^2 diag(eps_line) + tridiag(1, -2, 1) (the y-part of the
// stencil, PEC one cell beyond both ends, no PML on the cross-section), with
// eigenvalue mu = 2 - 2 cos(theta) = 4 sin^2(theta / 2).
//
// Eigenvalues: bisection on the Sturm count of the symmetric tridiagonal H
// (Barth, Martin and Wilkinson, 1967), to full double precision.  Eigenvectors:
// inverse iteration with the converged shift, each step a tridiagonal solve by
// Gaussian elimination with partial pivoting (Golub and Van Loan, Sec. 4.3.5),
// re-orthogonalised against the modes already found.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <vector>

#include "fdfd.h"

namespace {

constexpr double kPivMin = 1e-290;

// Number of eigenvalues of H below x: negative pivots of the LDL^T factorisation
// of H - x I (off-diagonal entries are all 1).
int sturm_count(const std::vector<double>& a, double x) {
  int count = 0;
  double q = 1.0;
  for (size_t i = 0; i < a.size(); ++i) {
    q = (a[i] - x) - (i ? 1.0 / q : 0.0);
    if (std::fabs(q) < kPivMin) q = -kPivMin;
    if (q < 0) ++count;
  }
  return count;
}

// k-th smallest eigenvalue (0-based) by bisection inside the Gershgorin interval.
double bisect(const std::vector<double>& a, int k, double lo, double hi) {
  for (int it = 0; it < 400; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (hi - lo <= 2.0 * DBL_EPSILON * std::max(std::fabs(lo), std::fabs(hi)) + kPivMin) break;
    if (sturm_count(a, mid) > k) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Solves (H - shift I) y = x in place of x, Gaussian elimination with row
// interchanges on the band (one extra superdiagonal of fill).  A zero pivot is
// replaced by a tiny one (the shift is an eigenvalue to working precision).
void shifted_solve(const std::vector<double>& a, double shift, double scale, std::vector<double>& x) {
  const size_t n = a.size();
  std::vector<double> d(n), du(n, 0.0), du2(n, 0.0), dl(n, 0.0);
  std::vector<char> swapped(n, 0);
  for (size_t i = 0; i < n; ++i) {
    d[i] = a[i] - shift;
    if (i + 1 < n) { du[i] = 1.0; dl[i] = 1.0; }
  }
  const double tiny = DBL_EPSILON * scale;
  for (size_t i = 0; i + 1 < n; ++i) {
    if (std::fabs(d[i]) >= std::fabs(dl[i])) {
      if (d[i] == 0.0) d[i] = tiny;
      const double l = dl[i] / d[i];
      dl[i] = l;
      d[i + 1] -= l * du[i];
    } else {
      // rows i and i+1 trade places: the subdiagonal entry becomes the pivot
      const double l = d[i] / dl[i];
      const double row1_diag = d[i + 1];
      const double row1_sup = (i + 2 < n) ? du[i + 1] : 0.0;
      d[i] = dl[i];
      dl[i] = l;
      d[i + 1] = du[i] - l * row1_diag;
      du[i] = row1_diag;
      du2[i] = row1_sup;
      if (i + 2 < n) du[i + 1] = -l * row1_sup;
      swapped[i] = 1;
    }
  }
  if (d[n - 1] == 0.0) d[n - 1] = tiny;
  for (size_t i = 0; i + 1 < n; ++i) {       // forward: apply the interchanges and L^-1
    if (swapped[i]) std::swap(x[i], x[i + 1]);
    x[i + 1] -= dl[i] * x[i];
  }
  for (size_t ii = n; ii-- > 0;) {           // back substitution with U (three bands)
    double s = x[ii];
    if (ii + 1 < n) s -= du[ii] * x[ii + 1];
    if (ii + 2 < n) s -= du2[ii] * x[ii + 2];
    x[ii] = s / d[ii];
  }
}

double norm2(const std::vector<double>& v) {
  double s = 0;
  for (double t : v) s += t * t;
  return std::sqrt(s);
}

}  // namespace

extern "C" fdfd_status fdfd_slab_modes(int ny, double k0dx, const double* eps_line, int n_modes, double* mu,
                                       double* theta, double* phi) {
  if (ny < 1 || n_modes < 1 || n_modes > ny || !eps_line || !mu || !phi || !std::isfinite(k0dx))
    return FDFD_ERR_ARG;
  std::vector<double> a(ny);
  double amin = INFINITY, amax = -INFINITY;
  for (int j = 0; j < ny; ++j) {
    if (!std::isfinite(eps_line[j])) return FDFD_ERR_ARG;
    a[j] = k0dx * k0dx * eps_line[j] - 2.0;
    amin = std::min(amin, a[j]);
    amax = std::max(amax, a[j]);
  }
  const double scale = std::max(std::fabs(amin), std::fabs(amax)) + 2.0;
  const double glo = amin - 2.0 - 1e-12 * scale, ghi = amax + 2.0 + 1e-12 * scale;
  uint32_t seed = 0x9e3779b9u;
  std::vector<std::vector<double>> found;
  for (int m = 0; m < n_modes; ++m) {
    const int k = ny - 1 - m;                  // the m-th largest eigenvalue
    const double lam = bisect(a, k, glo, ghi);
    std::vector<double> x(ny);
    for (int j = 0; j < ny; ++j) {             // deterministic start with every component present
      seed = seed * 1664525u + 1013904223u;
      x[j] = 0.5 + (seed >> 8) * (1.0 / 16777216.0);
    }
    for (int it = 0; it < 4; ++it) {
      shifted_solve(a, lam, scale, x);
      for (int pass = 0; pass < 2; ++pass)
        for (const auto& p : found) {
          double dot = 0;
          for (int j = 0; j < ny; ++j) dot += p[j] * x[j];
          for (int j = 0; j < ny; ++j) x[j] -= dot * p[j];
        }
      const double nx = norm2(x);
      if (!(nx > 0) || !std::isfinite(nx)) return FDFD_ERR_PIVOT;
      for (double& t : x) t /= nx;
    }
    // sign: the first entry reaching half the largest magnitude is positive
    double big = 0;
    for (double t : x) big = std::max(big, std::fabs(t));
    for (int j = 0; j < ny; ++j)
      if (std::fabs(x[j]) >= 0.5 * big) {
        if (x[j] < 0)
          for (double& t : x) t = -t;
        break;
      }
    mu[m] = lam;
    if (theta) theta[m] = (lam > 0 && lam < 4) ? 2.0 * std::asin(std::sqrt(lam) / 2.0) : NAN;
    std::copy(x.begin(), x.end(), phi + (size_t)m * ny);
    found.push_back(std::move(x));
  }
  return FDFD_OK;
}
