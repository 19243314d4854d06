// Orbital ordering from the two-orbital mutual information (host code).
//
// The paper places the orbitals along the chain so that the entanglement distance
// sum_ij I_ij |i - j|^eta, eta = 2, is small, with spectral graph theory: relaxing the
// positions to real numbers x (sum x = 0, |x| = 1) turns the distance into
// 2 x^T L x with the graph Laplacian L = D - I, whose minimiser is the eigenvector of
// the second smallest eigenvalue (the Fiedler vector).  The orbitals are sorted by its
// components.
//
// The Laplacian (n <= 1024) is diagonalised by the cyclic Jacobi method in FP64: every
// off-diagonal pair is annihilated in turn by a plane rotation, sweeps repeat until the
// off-diagonal part is below 1e-15 of the matrix norm.  Sign of the Fiedler vector: among
// the components within 1e-9 (relative) of the largest magnitude, the one of the lowest
// index is positive; equal components sort by index.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.h"

namespace {

// eigenvalues w (unsorted, diagonal of the rotated A) and eigenvectors (columns of V)
void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& w) {
  V.assign(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) V[size_t(i) * n + i] = 1.0;
  double norm = 0.0;
  for (double x : A) norm += x * x;
  norm = std::sqrt(norm);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[size_t(i) * n + j] * A[size_t(i) * n + j];
    if (std::sqrt(2.0 * off) <= 1e-15 * norm) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[size_t(p) * n + q];
        if (apq == 0.0) continue;
        const double app = A[size_t(p) * n + p], aqq = A[size_t(q) * n + q];
        // rotation angle zeroing A[p][q]: tan of the angle is the smaller root of
        // t^2 + 2 theta t - 1 = 0 with theta = (aqq - app) / (2 apq)
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {   // columns p, q
          const double akp = A[size_t(k) * n + p], akq = A[size_t(k) * n + q];
          A[size_t(k) * n + p] = c * akp - s * akq;
          A[size_t(k) * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q
          const double apk = A[size_t(p) * n + k], aqk = A[size_t(q) * n + k];
          A[size_t(p) * n + k] = c * apk - s * aqk;
          A[size_t(q) * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[size_t(k) * n + p], vkq = V[size_t(k) * n + q];
          V[size_t(k) * n + p] = c * vkp - s * vkq;
          V[size_t(k) * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[size_t(i) * n + i];
}

}  // namespace

extern "C" int dmrg_fiedler_order(int32_t n, const double* I, int32_t* order, double* fiedler) {
  try {
    if (n < 2 || n > 1024 || !I || !order) return DMRG_EINVAL;
    double scale = 0.0;
    for (int64_t k = 0; k < int64_t(n) * n; ++k) {
      if (!std::isfinite(I[k])) return DMRG_EINVAL;
      scale = std::max(scale, std::fabs(I[k]));
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        if (i == j) continue;
        const double a = I[size_t(i) * n + j], b = I[size_t(j) * n + i];
        if (std::fabs(a - b) > 1e-12 * scale || a < -1e-12 * scale) return DMRG_EINVAL;
      }
    // Laplacian of the off-diagonal weights
    std::vector<double> L(size_t(n) * n, 0.0);
    for (int i = 0; i < n; ++i) {
      double deg = 0.0;
      for (int j = 0; j < n; ++j)
        if (j != i) {
          const double wij = 0.5 * (I[size_t(i) * n + j] + I[size_t(j) * n + i]);
          L[size_t(i) * n + j] = -wij;
          deg += wij;
        }
      L[size_t(i) * n + i] = deg;
    }
    std::vector<double> V, w;
    jacobi_eigen(n, L, V, w);
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return w[a] < w[b] || (w[a] == w[b] && a < b); });
    const double trace = std::accumulate(w.begin(), w.end(), 0.0);
    // a disconnected graph (second eigenvalue zero) gives no order between its parts
    if (!(w[idx[1]] > 1e-12 * std::max(trace, 1e-300))) return DMRG_EINVAL;
    std::vector<double> v(n);
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) {
      v[i] = V[size_t(i) * n + idx[1]];
      nrm += v[i] * v[i];
    }
    nrm = std::sqrt(nrm);
    double amax = 0.0;
    for (int i = 0; i < n; ++i) {
      v[i] /= nrm;
      amax = std::max(amax, std::fabs(v[i]));
    }
    int k = 0;
    while (std::fabs(v[k]) < amax * (1.0 - 1e-9)) ++k;
    if (v[k] < 0)
      for (double& x : v) x = -x;
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return v[a] < v[b] || (v[a] == v[b] && a < b); });
    for (int i = 0; i < n; ++i) order[i] = ord[i];
    if (fiedler) std::copy(v.begin(), v.end(), fiedler);
    return DMRG_OK;
  } catch (const std::bad_alloc&) {
    return DMRG_ENOMEM;
  } catch (...) {
    return DMRG_EINVAL;
  }
}
