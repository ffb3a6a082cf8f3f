// Vector-kernel launchers shared by the solver drivers.
#pragma once

#include "internal.h"

namespace cheb {

constexpr int kMaxVecs = 40;      // basis vectors one fused kernel reads
constexpr int kRedBlocks = 592;   // reduction CTAs (4 per SM)

template <typename T>
struct VecList { const T* p[kMaxVecs]; };
struct CoefList { double c[kMaxVecs]; };

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
