// Host-side FP64 dense linear algebra used at plan set-up (hostmath.cu).
#pragma once

#include <vector>

namespace cheb {

// Row-major (N+1) x (N+1) derivative matrix on an interval with 2/(hi-lo) = scale.
std::vector<double> dense_deriv_matrix(int N, double scale);
// Clenshaw-Curtis weights at the N + 1 CGL nodes of [-1, 1] times half_len.
std::vector<double> cc_weights(int N, double half_len);
// C (m x n) = A (m x k) B (k x n), row-major.
std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B, int m, int k,
                           int n);
// In-place inverse of an n x n matrix; false when singular.
bool invert(std::vector<double>& A, int n);
// A = V diag(lam) V^{-1} for a matrix with real eigenvalues; V columns
// have unit 2-norm.  False when the iteration fails or the check A V = V L
// does not hold.
bool eig_real(const std::vector<double>& A, int n, std::vector<double>& lam, std::vector<double>& V);

}  // namespace cheb
