// Small dense host linear algebra (see linalg.hpp): the k x k projected
// eigenproblem of the non-symmetric Davidson (roots of Eq. 1-4; the paper
// names no eigensolver) by the textbook Hessenberg reduction and shifted QR,
// and the DIIS linear systems of the CCSDT iterations. O(k^3), k <= a few
// hundred; all vector-length work stays on the device.
#include "linalg.hpp"

#include <algorithm>
#include <cmath>
#include <limits>

namespace fnocc {

using cd = std::complex<double>;

namespace {

// Complex LU solve with partial pivoting; returns false when singular.
bool lu_solve(int n, std::vector<cd> a, std::vector<cd> &b) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = std::abs(a[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::abs(a[i * n + k]) > best) { best = std::abs(a[i * n + k]); piv = i; }
    if (best == 0.0) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(a[k * n + j], a[piv * n + j]);
      std::swap(b[k], b[piv]);
    }
    for (int i = k + 1; i < n; ++i) {
      cd f = a[i * n + k] / a[k * n + k];
      if (f == cd(0)) continue;
      for (int j = k; j < n; ++j) a[i * n + j] -= f * a[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    cd s = b[i];
    for (int j = i + 1; j < n; ++j) s -= a[i * n + j] * b[j];
    b[i] = s / a[i * n + i];
  }
  return true;
}

}  // namespace

void eig_nonsym(int n, const std::vector<double> &A, std::vector<cd> &w, std::vector<cd> &V) {
  w.assign(n, cd(0));
  V.assign((size_t)n * n, cd(0));
  if (n == 0) return;
  std::vector<cd> H(A.begin(), A.end());
  auto h = [&](int i, int j) -> cd & { return H[(size_t)i * n + j]; };
  // Householder reduction to upper Hessenberg form
  for (int k = 0; k + 2 < n; ++k) {
    double alpha = 0;
    for (int i = k + 1; i < n; ++i) alpha += std::norm(h(i, k));
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    cd x0 = h(k + 1, k);
    cd phase = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1);
    std::vector<cd> v(n, cd(0));
    v[k + 1] = x0 + phase * alpha;
    for (int i = k + 2; i < n; ++i) v[i] = h(i, k);
    double vn = 0;
    for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
    if (vn == 0.0) continue;
    // H = (I - 2 v v^* / vn) H
    for (int j = 0; j < n; ++j) {
      cd s = 0;
      for (int i = k + 1; i < n; ++i) s += std::conj(v[i]) * h(i, j);
      s *= 2.0 / vn;
      for (int i = k + 1; i < n; ++i) h(i, j) -= v[i] * s;
    }
    // H = H (I - 2 v v^* / vn)
    for (int i = 0; i < n; ++i) {
      cd s = 0;
      for (int j = k + 1; j < n; ++j) s += h(i, j) * v[j];
      s *= 2.0 / vn;
      for (int j = k + 1; j < n; ++j) h(i, j) -= s * std::conj(v[j]);
    }
    for (int i = k + 2; i < n; ++i) h(i, k) = 0;
  }
  // shifted QR on the Hessenberg matrix
  const double eps = std::numeric_limits<double>::epsilon();
  int hi = n - 1;
  int iter = 0;
  while (hi >= 0) {
    if (hi == 0) {
      w[0] = h(0, 0);
      break;
    }
    int l = hi;
    while (l > 0) {
      double s = std::abs(h(l - 1, l - 1)) + std::abs(h(l, l));
      if (s == 0) s = 1.0;
      if (std::abs(h(l, l - 1)) <= eps * s) {
        h(l, l - 1) = 0;
        break;
      }
      --l;
    }
    if (l == hi) {
      w[hi] = h(hi, hi);
      --hi;
      iter = 0;
      continue;
    }
    ++iter;
    if (iter > 1000) {  // give up on this window: report diagonal
      for (int i = l; i <= hi; ++i) w[i] = h(i, i);
      hi = l - 1;
      iter = 0;
      continue;
    }
    // Wilkinson shift from the trailing 2x2 block
    cd a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
    cd tr = a + d, det = a * d - b * c;
    cd disc = std::sqrt(tr * tr - 4.0 * det);
    cd mu1 = 0.5 * (tr + disc), mu2 = 0.5 * (tr - disc);
    cd mu = (std::abs(mu1 - d) < std::abs(mu2 - d)) ? mu1 : mu2;
    if (iter % 11 == 10) mu = d + cd(std::abs(h(hi, hi - 1)), 0.0);  // exceptional shift
    for (int i = l; i <= hi; ++i) h(i, i) -= mu;
    std::vector<cd> al(hi - l), be(hi - l);
    for (int k = l; k < hi; ++k) {
      cd x = h(k, k), y = h(k + 1, k);
      double r = std::sqrt(std::norm(x) + std::norm(y));
      cd aa = r > 0 ? x / r : cd(1), bb = r > 0 ? y / r : cd(0);
      al[k - l] = aa;
      be[k - l] = bb;
      for (int j = k; j <= hi; ++j) {
        cd u = h(k, j), t = h(k + 1, j);
        h(k, j) = std::conj(aa) * u + std::conj(bb) * t;
        h(k + 1, j) = -bb * u + aa * t;
      }
    }
    for (int k = l; k < hi; ++k) {
      cd aa = al[k - l], bb = be[k - l];
      int rmax = std::min(k + 2, hi);
      for (int i = l; i <= rmax; ++i) {
        cd u = h(i, k), t = h(i, k + 1);
        h(i, k) = u * aa + t * bb;
        h(i, k + 1) = -u * std::conj(bb) + t * std::conj(aa);
      }
    }
    for (int i = l; i <= hi; ++i) h(i, i) += mu;
  }
  // eigenvectors by inverse iteration on A
  double anorm = 0;
  for (double x : A) anorm = std::max(anorm, std::abs(x));
  if (anorm == 0) anorm = 1;
  for (int j = 0; j < n; ++j) {
    cd lam = w[j] + cd(1e-10 * anorm, 0.0);
    std::vector<cd> M((size_t)n * n);
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) M[(size_t)r * n + c] = cd(A[(size_t)r * n + c]) - (r == c ? lam : cd(0));
    std::vector<cd> x(n, cd(1.0 / std::sqrt((double)n)));
    for (int it = 0; it < 4; ++it) {
      std::vector<cd> y = x;
      if (!lu_solve(n, M, y)) {
        lam += cd(1e-8 * anorm, 0);
        for (int r = 0; r < n; ++r) M[(size_t)r * n + r] -= cd(1e-8 * anorm, 0);
        continue;
      }
      double nr = 0;
      for (auto &z : y) nr += std::norm(z);
      nr = std::sqrt(nr);
      if (nr == 0) break;
      for (int r = 0; r < n; ++r) x[r] = y[r] / nr;
    }
    for (int r = 0; r < n; ++r) V[(size_t)r * n + j] = x[r];
  }
}

bool solve_linear(int n, std::vector<double> A, std::vector<double> b, std::vector<double> &x) {
  double scale = 0;
  for (double a : A) scale = std::max(scale, std::abs(a));
  if (scale == 0) return false;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::abs(A[i * n + k]) > std::abs(A[piv * n + k])) piv = i;
    if (std::abs(A[piv * n + k]) <= 1e-300 + 1e-15 * scale * 1e-10) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[piv * n + j]);
      std::swap(b[k], b[piv]);
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  x.assign(n, 0.0);
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
    x[i] = s / A[i * n + i];
  }
  return true;
}

}  // namespace fnocc
