// Device-side Hessenberg / Givens state of one LGMRES cycle (Alg. 2's least
// squares problem), shared by the single-instance and the batched drivers.
// Layout of the FP64 block (nb = basis size): H[(nb+1) x nb] unrotated,
// R[(nb+1) x nb] rotated, cs[nb], sn[nb], g[nb+1], res[nb] (|g_{j+1}| after
// step j).
#pragma once

namespace cheb {

struct HessLayout {
  int nb;
  __host__ __device__ size_t H() const { return 0; }
  __host__ __device__ size_t R() const { return (size_t)(nb + 1) * nb; }
  __host__ __device__ size_t cs() const { return 2 * (size_t)(nb + 1) * nb; }
  __host__ __device__ size_t sn() const { return cs() + nb; }
  __host__ __device__ size_t g() const { return sn() + nb; }
  __host__ __device__ size_t res() const { return g() + nb + 1; }
  __host__ __device__ size_t total() const { return res() + nb; }
};

// column j of H from the Gram-Schmidt coefficients of one pass (block-strided)
__device__ __forceinline__ void hess_column(double* hess, const HessLayout& L, int j, int pass,
                                            const double* __restrict__ dv) {
  double* H = hess + L.H();
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double v = dv[i];
    H[(size_t)i * L.nb + j] = pass == 0 ? v : H[(size_t)i * L.nb + j] + v;
  }
}

// H[j+1][j] = |w|, rotate column j with the earlier rotations, make rotation
// j, update g and record |g_{j+1}|, which is returned (one thread).
__device__ __forceinline__ double hess_givens(double* hess, const HessLayout& L, int j, double norm2) {
  double* H = hess + L.H();
  double* R = hess + L.R();
  double* cs = hess + L.cs();
  double* sn = hess + L.sn();
  double* g = hess + L.g();
  const int nb = L.nb;
  const double hn = sqrt(fmax(0.0, norm2));
  H[(size_t)(j + 1) * nb + j] = hn;
  for (int i = 0; i <= j + 1; ++i) R[(size_t)i * nb + j] = H[(size_t)i * nb + j];
  for (int i = 0; i < j; ++i) {
    const double a = R[(size_t)i * nb + j], b = R[(size_t)(i + 1) * nb + j];
    R[(size_t)i * nb + j] = cs[i] * a + sn[i] * b;
    R[(size_t)(i + 1) * nb + j] = -sn[i] * a + cs[i] * b;
  }
  const double a = R[(size_t)j * nb + j], b = R[(size_t)(j + 1) * nb + j];
  const double den = hypot(a, b);
  cs[j] = den > 0 ? a / den : 1.0;
  sn[j] = den > 0 ? b / den : 0.0;
  R[(size_t)j * nb + j] = den;
  R[(size_t)(j + 1) * nb + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  const double r = fabs(g[j + 1]);
  hess[L.res() + j] = r;
  return r;
}

}  // namespace cheb
