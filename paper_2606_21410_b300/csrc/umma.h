// Blackwell tensor-core contraction (tcgen05 + TMA) used by the FP32
// fast-diagonalization preconditioner (umma.cu).
#pragma once

#include "internal.h"

namespace cheb {

// Y[n * M + m] = sum_k X[m * K + k] * W[n * K + k]  for m < M, n < N.
//
// One contraction of the tensor-product factorisation along the contiguous
// axis of X, written with the output transposed: X viewed as [M][K] (K the
// contracted axis, contiguous), W an N x K row-major matrix given as its
// split-TF32 pair (Wh = tf32(W), Wl = tf32(W - Wh), both n_rows x K with
// n_rows = umma_n_tile(N) and zero rows past N), Y written as [N][M].
// Arithmetic: three TF32 tensor-core products Xh Wh + Xh Wl + Xl Wh with
// FP32 accumulation, X split on the fly; FP32-level accuracy.  Wl = null:
// W is taken as exactly TF32 (Wh) and two products Xh Wh + Xl Wh are formed,
// so Wh is applied to X with FP32-level accuracy.
// Requirements (checked by umma_ok): K >= 32, K % 4 == 0, 32 <= N <= 256,
// M >= 128, 16-byte aligned X and W.  X and Y must not overlap.
//
// Epilogue modes (row m = rs * mpf + rf: rf the fast row axis, rs the slow
// one; column n = the contracted axis after the contraction):
//   0: Y[n * M + m] = acc
//   1: Y[n * M + m] = acc / (kref (lf[rf] + ls[rs] + lc[n])) on the valid
//      entries (rf < mf, rs < ms, n < mc), 0 on the padding  (the eigenvalue
//      division of the fast-diagonalization inverse)
//   2: no Y; acc goes to the interior of the full grid x at
//      xoff + rf xs_f + rs xs_s + n xs_c for valid entries, and the two end
//      values of every column-axis line are set from the elimination
//      x_end = G (line) + Binv r_end  (G: 2 x mc, Binv 2 x 2 row-major)
struct UmmaEpi {
  int mode = 0;
  int mpf = 1, mf = 1, ms = 1, mc = 1;
  const float* lf = nullptr;
  const float* ls = nullptr;
  const float* lc = nullptr;
  float kref = 1.f;
  float* x = nullptr;
  const float* r = nullptr;
  long long xoff = 0, xs_f = 0, xs_s = 0, xs_c = 0;
  int ncol = 0;  // points of the column axis, ends included
  const float* G = nullptr;
  const float* Binv = nullptr;
  const int* active = nullptr;  // batched solves: the CTA returns at entry while *active == 0
};
int umma_tf32x3_rot(const float* X, const float* Wh, const float* Wl, float* Y, int M, int N, int K,
                    const UmmaEpi& ep, cudaStream_t s);
bool umma_ok(int M, int N, int K);
int umma_n_tile(int N);
// Split-TF32 pair of a row-major matrix (host): hi = tf32(x), lo = tf32(x - hi).
void tf32_split_host(const double* x, size_t n, float* hi, float* lo);
// Tensor-core route of the FP32 operator apply (dense D on every line):
// one axis pass of A u, writing (first) or accumulating into out with the
// boundary rows of this axis; resources are built on first use and freed
// with the plan.
struct TensorApply;
bool tensor_route_ok(const cheb_plan_s* p, int axis);
int tensor_apply_pass(const cheb_plan_s* p, int axis, bool first, const float* K, const float* u, float* out,
                      cudaStream_t s);
void tensor_apply_free(TensorApply* t);

// Reads and clears the device-side error word the kernel sets when one of
// its bounded waits gives up (returns 0 when no wait gave up).
int umma_take_error();
// Runs the bounded-wait self-test kernel (a wait that nothing completes,
// limit wait_cycles) on stream s and synchronises it.
int umma_wait_selftest(long long wait_cycles, cudaStream_t s);

}  // namespace cheb
