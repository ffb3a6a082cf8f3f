// Vector-kernel launchers shared by the solver drivers.
#pragma once

#include <type_traits>
#include <utility>

#include "internal.h"

namespace cheb {

constexpr int kMaxVecs = 40;      // basis vectors one fused kernel reads
constexpr int kRedBlocks = 592;   // reduction CTAs (4 per SM)

template <typename T>
struct VecList { const T* p[kMaxVecs]; };
struct CoefList { double c[kMaxVecs]; };

// f(std::integral_constant<int, N>()) for N == cnt, 0 <= cnt <= kMaxVecs
// (else CHEB_ERR_ARG).  The fused multi-vector kernels are compiled for each
// exact vector count: a kernel written for a bound with a run-time count
// issues the loads and FMAs of the absent vectors as predicated-off
// instructions (for a one-vector norm, 40 times the issue slots it needs).
template <typename F, int... I>
inline int count_dispatch_impl(int cnt, F& f, std::integer_sequence<int, I...>) {
  int r = CHEB_ERR_ARG;
  (void)((cnt == I ? (r = f(std::integral_constant<int, I>()), true) : false) || ...);
  return r;
}
template <typename F>
inline int count_dispatch(int cnt, F&& f) {
  return count_dispatch_impl(cnt, f, std::make_integer_sequence<int, kMaxVecs + 1>());
}

// Scratch of the deterministic reductions: kMaxVecs+1 partial rows of
// kRedBlocks doubles and a completion counter (zero between launches).
struct ReduceScratch {
  double* part = nullptr;
  unsigned* counter = nullptr;
};

template <typename T>
int k_mdot(const ReduceScratch& rs, const T* const* src, int cnt, const T* w, size_t n,
           bool with_self, double* out_dev, cudaStream_t s);
template <typename T>
int k_maxpy(const ReduceScratch& rs, const T* const* src, const double* coef, int cnt, double beta,
            T* y, size_t n, double* norm2_dev, cudaStream_t s);
// same with coefficients read on the device: c_i = sign * coef_dev[i]
template <typename T>
int k_maxpy_dev(const ReduceScratch& rs, const T* const* src, const double* coef_dev, double sign,
                int cnt, double beta, T* y, size_t n, double* norm2_dev, cudaStream_t s);
template <typename T>
int k_scale_inv_norm(T* y, const double* norm2_dev, size_t n, cudaStream_t s);
int k_sum_log(const ReduceScratch& rs, const double* K, size_t n, double* out_dev, cudaStream_t s);
// out = sum of wx[i] wy[j] wz[k] a b over the field (wy / wz may be null: weight 1)
int k_wsum3(const ReduceScratch& rs, const double* a, const double* b, const double* wx, const double* wy,
            const double* wz, int nx, int ny, size_t n, double* out_dev, cudaStream_t s);
template <typename T>
int k_scale(T* y, const T* x, double sc, size_t n, cudaStream_t s);
template <typename To, typename Ti>
int k_cast_scale(To* y, const Ti* x, double sc, size_t n, cudaStream_t s);
template <typename Ti>
int k_axpy64(double* y, const Ti* x, double sc, size_t n, cudaStream_t s);
template <typename T>
int k_residual(T* r, const T* b, size_t n, cudaStream_t s);

}  // namespace cheb
