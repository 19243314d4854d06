// Extrapolation of energies in the number of kept block states M (host code).
//
// The method description estimates the truncation-free energy by fitting runs at several
// M with E(M) = E_inf + X1 M^X2 (three free parameters); the 64Ge results bound it from
// above with a second-order polynomial fit, read here as a polynomial in 1/M.  Both are
// ordinary least squares over the given points.
//
// Power law: at a fixed exponent b the model is linear in (E_inf, X1), so the residual
// sum of squares S(b) of that linear fit is a function of b alone; b is bracketed on a
// grid over [-8, -1e-4] and refined by golden-section search inside the best grid cell.
// M is scaled by its largest value first, u = (M / M_top)^b, which keeps the columns of
// the linear fit of order one whatever M and b are.
// Polynomial: x = M_low / M in (0, 1], columns 1, x, x^2 orthogonalised by modified
// Gram-Schmidt (twice), coefficients scaled back to 1/M afterwards.
#include <cmath>
#include <vector>

#include "common.h"

namespace {

constexpr double kX2Lo = -8.0, kX2Hi = -1e-4;
constexpr int kGrid = 4001;

// least squares E = a + c u at u_i = (M_i / top)^b; returns the residual sum of squares
double linear_at(const std::vector<double>& M, const std::vector<double>& E, double top,
                 double b, std::vector<double>& u, double* a, double* c) {
  const int n = int(M.size());
  double ub = 0.0, eb = 0.0;
  for (int i = 0; i < n; ++i) {
    u[i] = std::pow(M[i] / top, b);
    ub += u[i];
    eb += E[i];
  }
  ub /= n;
  eb /= n;
  double suu = 0.0, sue = 0.0;
  for (int i = 0; i < n; ++i) {
    suu += (u[i] - ub) * (u[i] - ub);
    sue += (u[i] - ub) * (E[i] - eb);
  }
  const double cc = suu > 0.0 ? sue / suu : 0.0;
  const double aa = eb - cc * ub;
  double ss = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = E[i] - aa - cc * u[i];
    ss += r * r;
  }
  *a = aa;
  *c = cc;
  return ss;
}

int check_points(int32_t n, const double* M, const double* E, std::vector<double>& m,
                 std::vector<double>& e) {
  if (n < 3 || !M || !E) return DMRG_EINVAL;
  m.assign(M, M + n);
  e.assign(E, E + n);
  std::vector<double> distinct;
  for (int i = 0; i < n; ++i) {
    if (!std::isfinite(m[i]) || !std::isfinite(e[i]) || !(m[i] > 0.0)) return DMRG_EINVAL;
    bool seen = false;
    for (double d : distinct) seen = seen || d == m[i];
    if (!seen) distinct.push_back(m[i]);
  }
  return distinct.size() >= 3 ? DMRG_OK : DMRG_EINVAL;
}

int fit_power(const std::vector<double>& M, const std::vector<double>& E, double* coef,
              double* rms) {
  const int n = int(M.size());
  double top = 0.0;
  for (double x : M) top = std::max(top, x);
  std::vector<double> u(n);
  double a, c;
  int best = 0;
  double best_ss = INFINITY;
  const double h = (kX2Hi - kX2Lo) / (kGrid - 1);
  for (int g = 0; g < kGrid; ++g) {
    const double ss = linear_at(M, E, top, kX2Lo + g * h, u, &a, &c);
    if (ss < best_ss) {
      best_ss = ss;
      best = g;
    }
  }
  if (best == 0 || best == kGrid - 1 || !std::isfinite(best_ss)) return DMRG_ENOCONV;
  // golden-section search on [b_lo, b_hi] around the best grid point
  const double phi = 0.5 * (std::sqrt(5.0) - 1.0);
  double lo = kX2Lo + (best - 1) * h, hi = kX2Lo + (best + 1) * h;
  double x1 = hi - phi * (hi - lo), x2 = lo + phi * (hi - lo);
  double f1 = linear_at(M, E, top, x1, u, &a, &c), f2 = linear_at(M, E, top, x2, u, &a, &c);
  for (int it = 0; it < 200 && hi - lo > 1e-14 * (1.0 + std::fabs(lo)); ++it) {
    if (f1 <= f2) {
      hi = x2;
      x2 = x1;
      f2 = f1;
      x1 = hi - phi * (hi - lo);
      f1 = linear_at(M, E, top, x1, u, &a, &c);
    } else {
      lo = x1;
      x1 = x2;
      f1 = f2;
      x2 = lo + phi * (hi - lo);
      f2 = linear_at(M, E, top, x2, u, &a, &c);
    }
  }
  double b = 0.5 * (lo + hi);
  double ss = linear_at(M, E, top, b, u, &a, &c);
  if (best_ss < ss) {   // the grid point itself was better (flat minimum)
    b = kX2Lo + best * h;
    ss = linear_at(M, E, top, b, u, &a, &c);
  }
  coef[0] = a;
  coef[1] = c * std::pow(top, -b);   // c (M / top)^b = c top^-b M^b
  coef[2] = b;
  *rms = std::sqrt(ss / n);
  return DMRG_OK;
}

int fit_quadratic(const std::vector<double>& M, const std::vector<double>& E, double* coef,
                  double* rms) {
  const int n = int(M.size());
  double low = INFINITY;
  for (double x : M) low = std::min(low, x);
  // Q R = [1, x, x^2], x = low / M; then R d = Q^T E
  std::vector<double> Q(3 * size_t(n));
  double R[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int i = 0; i < n; ++i) {
    const double x = low / M[i];
    Q[i] = 1.0;
    Q[n + i] = x;
    Q[2 * n + i] = x * x;
  }
  for (int j = 0; j < 3; ++j) {
    double* q = &Q[size_t(j) * n];
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 0; k < j; ++k) {
        const double* qk = &Q[size_t(k) * n];
        double d = 0.0;
        for (int i = 0; i < n; ++i) d += qk[i] * q[i];
        for (int i = 0; i < n; ++i) q[i] -= d * qk[i];
        R[k][j] += d;
      }
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) nrm += q[i] * q[i];
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0)) return DMRG_EINVAL;
    R[j][j] = nrm;
    for (int i = 0; i < n; ++i) q[i] /= nrm;
  }
  double z[3];
  for (int j = 0; j < 3; ++j) {
    z[j] = 0.0;
    for (int i = 0; i < n; ++i) z[j] += Q[size_t(j) * n + i] * E[i];
  }
  double d[3];
  for (int j = 2; j >= 0; --j) {
    double s = z[j];
    for (int k = j + 1; k < 3; ++k) s -= R[j][k] * d[k];
    d[j] = s / R[j][j];
  }
  double ss = 0.0;
  for (int i = 0; i < n; ++i) {
    const double x = low / M[i];
    const double r = E[i] - (d[0] + d[1] * x + d[2] * x * x);
    ss += r * r;
  }
  coef[0] = d[0];
  coef[1] = d[1] * low;
  coef[2] = d[2] * low * low;
  *rms = std::sqrt(ss / n);
  return DMRG_OK;
}

}  // namespace

extern "C" int dmrg_extrapolate(int32_t kind, int32_t n, const double* M, const double* E,
                                double* coef, double* rms) {
  try {
    if (!coef || !rms || (kind != DMRG_FIT_POWER && kind != DMRG_FIT_QUADRATIC))
      return DMRG_EINVAL;
    std::vector<double> m, e;
    const int rc = check_points(n, M, E, m, e);
    if (rc != DMRG_OK) return rc;
    return kind == DMRG_FIT_POWER ? fit_power(m, e, coef, rms) : fit_quadratic(m, e, coef, rms);
  } catch (const std::bad_alloc&) {
    return DMRG_ENOMEM;
  } catch (...) {
    return DMRG_EINVAL;
  }
}
