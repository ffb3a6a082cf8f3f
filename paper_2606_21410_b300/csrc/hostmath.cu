// Host-side FP64 dense linear algebra for plan set-up (small matrices only):
// the transform-route differentiation matrix, matrix products, inversion by
// Gauss-Jordan elimination, and a real eigen-decomposition for matrices with
// real eigenvalues (Householder reduction to Hessenberg form, shifted QR
// iterations with Givens rotations, eigenvectors of the triangular Schur
// factor by back substitution; Golub & Van Loan, Matrix Computations, 7.4).
#include <algorithm>
#include <cmath>
#include <vector>

#include "hostmath.h"

namespace cheb {

// Clenshaw-Curtis quadrature: integrate the degree-N interpolant.  With the
// interpolant's Chebyshev coefficients a_k = (c_k / N) sum_n m_n f_n
// cos(pi k n / N) (m = 1 at the ends, 2 inside; c = 1/2 at k = 0, N, else 1)
// and int_{-1}^{1} T_k = 2 / (1 - k^2) for even k (0 for odd k), the weight
// of node n is w_n = (m_n / N) sum_{even k} c_k cos(pi k n / N) 2 / (1 - k^2).
std::vector<double> cc_weights(int N, double half_len) {
  std::vector<double> w(N + 1, 0.0);
  for (int n = 0; n <= N; ++n) {
    double s = 0.0;
    for (int k = 0; k <= N; k += 2) {
      const double ck = (k == 0 || k == N) ? 0.5 : 1.0;
      s += ck * std::cos(M_PI * (double)((long long)k * n % (2 * N)) / N) * 2.0 / (1.0 - (double)k * k);
    }
    const double mn = (n == 0 || n == N) ? 1.0 : 2.0;
    w[n] = mn / N * s * half_len;
  }
  return w;
}

std::vector<double> dense_deriv_matrix(int N, double scale) {
  // D e_col for every unit vector, by the transform-route definition:
  // F = DCT-I(e_col), G_k = k c_k scale F_k / N, beta_k = sum_{j>k, j-k odd} G_j,
  // derivative = DCT-I(beta) (direct cosine sums, FP64).
  const int n = N + 1;
  std::vector<double> cosv(2 * N);
  for (int t = 0; t < 2 * N; ++t) cosv[t] = std::cos(M_PI * t / N);
  auto m = [&](int k) { return (k == 0 || k == N) ? 1.0 : 2.0; };
  std::vector<double> D((size_t)n * n), G(n), beta(n);
  for (int col = 0; col < n; ++col) {
    for (int k = 0; k < n; ++k) {
      const double F = m(col) * cosv[((long)k * col) % (2 * N)];
      const double ck = (k == N) ? 0.5 : 1.0;
      G[k] = k * ck * scale / N * F;
    }
    for (int k = 0; k < n; ++k) {
      double s = 0.0;
      for (int j = k + 1; j <= N; j += 2) s += G[j];
      beta[k] = (k == N) ? 0.0 : s;
    }
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += m(k) * cosv[((long)k * i) % (2 * N)] * beta[k];
      D[(size_t)i * n + col] = s;
    }
  }
  return D;
}

std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B, int m, int k,
                           int n) {
  std::vector<double> C((size_t)m * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int l = 0; l < k; ++l) {
      const double a = A[(size_t)i * k + l];
      if (a == 0.0) continue;
      for (int j = 0; j < n; ++j) C[(size_t)i * n + j] += a * B[(size_t)l * n + j];
    }
  return C;
}

bool invert(std::vector<double>& A, int n) {
  // Gauss-Jordan with partial pivoting, in place.
  std::vector<int> piv(n);
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)p * n + c])) p = r;
    if (A[(size_t)p * n + c] == 0.0) return false;
    if (p != c)
      for (int j = 0; j < n; ++j) {
        std::swap(A[(size_t)p * n + j], A[(size_t)c * n + j]);
        std::swap(inv[(size_t)p * n + j], inv[(size_t)c * n + j]);
      }
    const double d = 1.0 / A[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) { A[(size_t)c * n + j] *= d; inv[(size_t)c * n + j] *= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[(size_t)r * n + j] -= f * A[(size_t)c * n + j];
        inv[(size_t)r * n + j] -= f * inv[(size_t)c * n + j];
      }
    }
  }
  A.swap(inv);
  return true;
}

namespace {

// apply the Givens rotation [c s; -s c] to rows (or columns) p, q
inline void rot_rows(std::vector<double>& H, int n, int p, int q, double c, double s, int j0, int j1) {
  for (int j = j0; j < j1; ++j) {
    const double a = H[(size_t)p * n + j], b = H[(size_t)q * n + j];
    H[(size_t)p * n + j] = c * a + s * b;
    H[(size_t)q * n + j] = -s * a + c * b;
  }
}
inline void rot_cols(std::vector<double>& H, int n, int p, int q, double c, double s, int i0, int i1) {
  for (int i = i0; i < i1; ++i) {
    const double a = H[(size_t)i * n + p], b = H[(size_t)i * n + q];
    H[(size_t)i * n + p] = c * a + s * b;
    H[(size_t)i * n + q] = -s * a + c * b;
  }
}

}  // namespace

bool eig_real(const std::vector<double>& A0, int n, std::vector<double>& lam,
              std::vector<double>& V) {
  std::vector<double> H = A0;
  std::vector<double> Z((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
  // 1. Householder reduction to upper Hessenberg form: H = Z^T A Z
  std::vector<double> v(n);
  for (int k = 0; k + 2 < n; ++k) {
    double alpha = 0.0;
    for (int i = k + 1; i < n; ++i) alpha += H[(size_t)i * n + k] * H[(size_t)i * n + k];
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    const double x0 = H[(size_t)(k + 1) * n + k];
    if (x0 > 0) alpha = -alpha;
    for (int i = 0; i < n; ++i) v[i] = 0.0;
    v[k + 1] = x0 - alpha;
    for (int i = k + 2; i < n; ++i) v[i] = H[(size_t)i * n + k];
    double vv = 0.0;
    for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    // H = (I - beta v v^T) H
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = k + 1; i < n; ++i) s += v[i] * H[(size_t)i * n + j];
      s *= beta;
      for (int i = k + 1; i < n; ++i) H[(size_t)i * n + j] -= s * v[i];
    }
    // H = H (I - beta v v^T), Z = Z (I - beta v v^T)
    for (int i = 0; i < n; ++i) {
      double s = 0.0, t = 0.0;
      for (int j = k + 1; j < n; ++j) {
        s += H[(size_t)i * n + j] * v[j];
        t += Z[(size_t)i * n + j] * v[j];
      }
      s *= beta;
      t *= beta;
      for (int j = k + 1; j < n; ++j) {
        H[(size_t)i * n + j] -= s * v[j];
        Z[(size_t)i * n + j] -= t * v[j];
      }
    }
    for (int i = k + 2; i < n; ++i) H[(size_t)i * n + k] = 0.0;
  }
  // 2. shifted QR iterations (real shifts; the eigenvalues are real)
  double anorm = 0.0;
  for (double x : H) anorm = std::max(anorm, std::fabs(x));
  const double eps = 2.2e-16;
  int hi = n - 1, iter = 0, total = 0;
  std::vector<double> cs(n), sn(n);
  while (hi > 0) {
    int l = hi;
    while (l > 0) {
      const double sub = std::fabs(H[(size_t)l * n + l - 1]);
      const double diag = std::fabs(H[(size_t)(l - 1) * n + l - 1]) + std::fabs(H[(size_t)l * n + l]);
      if (sub <= eps * (diag > 0 ? diag : anorm)) { H[(size_t)l * n + l - 1] = 0.0; break; }
      --l;
    }
    if (l == hi) { --hi; iter = 0; continue; }
    if (++iter > 60 || ++total > 60 * n) return false;
    // shift: eigenvalue of the trailing 2 x 2 block nearest H[hi][hi]
    const double a = H[(size_t)(hi - 1) * n + hi - 1], b = H[(size_t)(hi - 1) * n + hi];
    const double c = H[(size_t)hi * n + hi - 1], d = H[(size_t)hi * n + hi];
    double mu = d;
    const double tr = 0.5 * (a + d), det = a * d - b * c, disc = tr * tr - det;
    if (disc >= 0) {
      const double r = std::sqrt(disc);
      const double e1 = tr + r, e2 = tr - r;
      mu = std::fabs(e1 - d) < std::fabs(e2 - d) ? e1 : e2;
    }
    if (iter % 11 == 10) mu = d + 0.75 * std::fabs(c);  // exceptional shift
    // QR step on the active block [l, hi]: H - mu I = Q R, H <- R Q + mu I
    for (int k = l; k <= hi; ++k) H[(size_t)k * n + k] -= mu;
    for (int k = l; k < hi; ++k) {
      const double x = H[(size_t)k * n + k], y = H[(size_t)(k + 1) * n + k];
      const double r = std::hypot(x, y);
      const double cc = r == 0 ? 1.0 : x / r, ss = r == 0 ? 0.0 : y / r;
      cs[k] = cc;
      sn[k] = ss;
      rot_rows(H, n, k, k + 1, cc, ss, k, n);  // full rows: keeps the Schur form of H
    }
    for (int k = l; k < hi; ++k) {
      rot_cols(H, n, k, k + 1, cs[k], sn[k], 0, std::min(k + 2, hi) + 1);
      rot_cols(Z, n, k, k + 1, cs[k], sn[k], 0, n);
    }
    for (int k = l; k <= hi; ++k) H[(size_t)k * n + k] += mu;
  }
  // 3. eigenvectors of the upper-triangular T = H, then V = Z Y
  lam.assign(n, 0.0);
  for (int k = 0; k < n; ++k) lam[k] = H[(size_t)k * n + k];
  std::vector<double> Y((size_t)n * n, 0.0);
  for (int k = 0; k < n; ++k) {
    Y[(size_t)k * n + k] = 1.0;
    for (int i = k - 1; i >= 0; --i) {
      double s = 0.0;
      for (int j = i + 1; j <= k; ++j) s += H[(size_t)i * n + j] * Y[(size_t)j * n + k];
      double den = H[(size_t)i * n + i] - lam[k];
      if (std::fabs(den) < eps * anorm) den = (den >= 0 ? 1 : -1) * eps * anorm;
      Y[(size_t)i * n + k] = -s / den;
    }
  }
  V = matmul(Z, Y, n, n, n);
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += V[(size_t)i * n + k] * V[(size_t)i * n + k];
    s = 1.0 / std::sqrt(s);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + k] *= s;
  }
  // 4. check A V = V Lambda
  double res = 0.0, sc = 0.0;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += A0[(size_t)i * n + j] * V[(size_t)j * n + k];
      res = std::max(res, std::fabs(s - lam[k] * V[(size_t)i * n + k]));
      sc = std::max(sc, std::fabs(lam[k]));
    }
  return res <= 1e-9 * std::max(sc, anorm);
}

}  // namespace cheb
