// Vector kernels of the LGMRES Arnoldi process and the refinement loop:
// fused multi-dot products (one read of w for all basis vectors), fused
// multi-axpy with the norm of the result, scaling, casts and the FP64
// residual update.  Reductions are deterministic: per-CTA partials in a
// fixed order, the last CTA to finish sums the partials in index order.
#include <algorithm>
#include <cstdint>

#include "krylov.h"

namespace cheb {

constexpr int kRedThreads = 256;

static int red_blocks(size_t n) {
  // enough CTAs to fill the GPU (148 SMs), never more than the work needs
  size_t b = (n + kRedThreads * 16 - 1) / (kRedThreads * 16);
  return (int)std::max<size_t>(1, std::min<size_t>(b, kRedBlocks));
}

template <typename T>
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  return v;
}

// Block-reduce per-thread values and store the block's sums to
// part[o * gridDim.x + blockIdx.x]: slot i < cnt goes to output o = i and,
// when `extra`, the last slot MAXV-1 goes to output o = cnt.  Then the last
// CTA sums the partials (fixed order, FP64) into out[o].  The slot loop is
// unrolled so acc stays in registers.
template <typename T, int MAXV>
__device__ void block_reduce_store(T (&acc)[MAXV], int cnt, bool extra, double* part,
                                   unsigned* counter, double* out) {
  __shared__ double sred[kRedThreads / 32][MAXV];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nout = cnt + (extra ? 1 : 0);
#pragma unroll
  for (int i = 0; i < MAXV; ++i) {
    const bool active = (i < cnt) || (extra && i == MAXV - 1);
    if (active) {
      const int o = (i < cnt) ? i : cnt;
      T v = warp_sum_t<T>(acc[i]);
      if (lane == 0) sred[wid][o] = (double)v;
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) s += sred[w][o];
    part[(size_t)o * gridDim.x + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // one warp per output value, lanes stride the partials, fixed tree order
  for (int o = wid; o < nout; o += kRedThreads / 32) {
    double s = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(part + (size_t)o * gridDim.x + b);
    s = warp_sum<double>(s);
    if (lane == 0) out[o] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;  // ready for the next launch
}

// 16-byte vectors of the streaming loops.  Krylov vectors are carved from
// one allocation at offsets of i * n elements, so they are 16-byte aligned
// only for some n: the host passes vec = 1 only when every pointer of the
// launch is, and otherwise the whole range runs element-wise.
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  typedef float4 t;
  static constexpr int W = 4;
  __device__ static float at(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
  __device__ static void set(float4& v, int k, float x) {
    if (k == 0) v.x = x; else if (k == 1) v.y = x; else if (k == 2) v.z = x; else v.w = x;
  }
};
template <> struct Vec16<double> {
  typedef double2 t;
  static constexpr int W = 2;
  __device__ static double at(const double2& v, int k) { return k == 0 ? v.x : v.y; }
  __device__ static void set(double2& v, int k, double x) {
    if (k == 0) v.x = x; else v.y = x;
  }
};

// Elements per thread and loop iteration of the fused kernels: enough that a
// thread has at least four independent 16-byte loads in flight.
template <int NLOADS>
constexpr int unroll_for() { return NLOADS >= 4 ? 1 : NLOADS >= 2 ? 2 : 4; }
// Resident CTAs asked of the register allocator: two below 16 vectors, one
// above, where a thread's 16 or more loads in flight already cover the
// memory latency and the larger register budget avoids spills.
template <int NV>
constexpr int min_ctas() { return NV >= 16 ? 1 : 2; }

// out[i] = <src_i, w>, i < NV; with_self: also <w, w>, stored at out[NV].
// 16-byte vector loads (when vec), element-wise tail.
template <typename T, int NV>
__global__ void __launch_bounds__(kRedThreads, min_ctas<NV>())
mdot_kernel(VecList<T> src, const T* __restrict__ w, size_t n, int with_self, int vec, double* part,
            unsigned* counter, double* out) {
  typedef typename Vec16<T>::t V;
  constexpr int W = Vec16<T>::W;
  constexpr int U = unroll_for<NV + 1>();
  T acc[NV + 1];
#pragma unroll
  for (int i = 0; i <= NV; ++i) acc[i] = (T)0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t nv = vec ? n / W : 0;
  const V* wv4 = reinterpret_cast<const V*>(w);
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; e + (U - 1) * stride < nv; e += U * stride) {
    V wv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) wv[u] = wv4[e + u * stride];
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const V sv = reinterpret_cast<const V*>(src.p[i])[e + u * stride];
#pragma unroll
        for (int k = 0; k < W; ++k) acc[i] += Vec16<T>::at(sv, k) * Vec16<T>::at(wv[u], k);
      }
      if (with_self) {
#pragma unroll
        for (int k = 0; k < W; ++k) acc[NV] += Vec16<T>::at(wv[u], k) * Vec16<T>::at(wv[u], k);
      }
    }
  }
  for (; e < nv; e += stride) {
    const V wv = wv4[e];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const V sv = reinterpret_cast<const V*>(src.p[i])[e];
#pragma unroll
      for (int k = 0; k < W; ++k) acc[i] += Vec16<T>::at(sv, k) * Vec16<T>::at(wv, k);
    }
    if (with_self) {
#pragma unroll
      for (int k = 0; k < W; ++k) acc[NV] += Vec16<T>::at(wv, k) * Vec16<T>::at(wv, k);
    }
  }
  for (size_t t = nv * W + blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += stride) {
    const T x = w[t];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] += src.p[i][t] * x;
    if (with_self) acc[NV] += x * x;
  }
  block_reduce_store<T, NV + 1>(acc, NV, with_self != 0, part, counter, out);
}

// y = beta * y + sum_i c_i src_i, i < NV; c_i = csign * cdev[i] when cdev,
// else coef.c[i].  want_norm: ||y||^2 -> out[0].
template <typename T, int NV>
__global__ void __launch_bounds__(kRedThreads, min_ctas<NV>())
maxpy_kernel(VecList<T> src, CoefList coef, const double* __restrict__ cdev, double csign, double beta,
             T* __restrict__ y, size_t n, int want_norm, int vec, double* part, unsigned* counter,
             double* out) {
  typedef typename Vec16<T>::t V;
  constexpr int W = Vec16<T>::W;
  constexpr int U = unroll_for<NV + 1>();
  T c[NV > 0 ? NV : 1];
#pragma unroll
  for (int i = 0; i < NV; ++i) c[i] = (T)(cdev ? csign * cdev[i] : coef.c[i]);
  T acc[1] = {(T)0};
  const T b = (T)beta;
  const bool keep = beta != 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t nv = vec ? n / W : 0;
  V* y4 = reinterpret_cast<V*>(y);
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; e + (U - 1) * stride < nv; e += U * stride) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (keep) {
        const V yo = y4[e + u * stride];
#pragma unroll
        for (int k = 0; k < W; ++k) Vec16<T>::set(v[u], k, b * Vec16<T>::at(yo, k));
      } else {
#pragma unroll
        for (int k = 0; k < W; ++k) Vec16<T>::set(v[u], k, (T)0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const V sv = reinterpret_cast<const V*>(src.p[i])[e + u * stride];
#pragma unroll
        for (int k = 0; k < W; ++k)
          Vec16<T>::set(v[u], k, Vec16<T>::at(v[u], k) + c[i] * Vec16<T>::at(sv, k));
      }
      y4[e + u * stride] = v[u];
#pragma unroll
      for (int k = 0; k < W; ++k) acc[0] += Vec16<T>::at(v[u], k) * Vec16<T>::at(v[u], k);
    }
  }
  for (; e < nv; e += stride) {
    V v;
    if (keep) {
      const V yo = y4[e];
#pragma unroll
      for (int k = 0; k < W; ++k) Vec16<T>::set(v, k, b * Vec16<T>::at(yo, k));
    } else {
#pragma unroll
      for (int k = 0; k < W; ++k) Vec16<T>::set(v, k, (T)0);
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const V sv = reinterpret_cast<const V*>(src.p[i])[e];
#pragma unroll
      for (int k = 0; k < W; ++k) Vec16<T>::set(v, k, Vec16<T>::at(v, k) + c[i] * Vec16<T>::at(sv, k));
    }
    y4[e] = v;
#pragma unroll
    for (int k = 0; k < W; ++k) acc[0] += Vec16<T>::at(v, k) * Vec16<T>::at(v, k);
  }
  for (size_t t = nv * W + blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += stride) {
    T v = keep ? b * y[t] : (T)0;
#pragma unroll
    for (int i = 0; i < NV; ++i) v += c[i] * src.p[i][t];
    y[t] = v;
    acc[0] += v * v;
  }
  if (want_norm) block_reduce_store<T, 1>(acc, 1, false, part, counter, out);
}

// The element-wise kernels below walk their grid-stride loop four elements
// at a time (the four loads issued before the first store: four loads in
// flight per thread instead of one), then the remainder one by one.
template <typename T>
__global__ void scale_kernel(T* __restrict__ y, const T* __restrict__ x, double s, size_t n) {
  const T sv = (T)s;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; e + 3 * stride < n; e += 4 * stride) {
    T v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = x[e + u * stride];
#pragma unroll
    for (int u = 0; u < 4; ++u) y[e + u * stride] = sv * v[u];
  }
  for (; e < n; e += stride) y[e] = sv * x[e];
}

// y (To) = s * x (Ti)
template <typename To, typename Ti>
__global__ void cast_scale_kernel(To* __restrict__ y, const Ti* __restrict__ x, double s, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; e + 3 * stride < n; e += 4 * stride) {
    Ti v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = x[e + u * stride];
#pragma unroll
    for (int u = 0; u < 4; ++u) y[e + u * stride] = (To)(s * (double)v[u]);
  }
  for (; e < n; e += stride) y[e] = (To)(s * (double)x[e]);
}

// y (FP64) += s * x (Ti)
template <typename Ti>
__global__ void axpy64_kernel(double* __restrict__ y, const Ti* __restrict__ x, double s, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; e + 3 * stride < n; e += 4 * stride) {
    Ti v[4];
    double w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      v[u] = x[e + u * stride];
      w[u] = y[e + u * stride];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) y[e + u * stride] = w[u] + s * (double)v[u];
  }
  for (; e < n; e += stride) y[e] += s * (double)x[e];
}

// r = b - r  (r holds A x on entry)
template <typename T>
__global__ void residual_kernel(T* __restrict__ r, const T* __restrict__ b, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; e + 3 * stride < n; e += 4 * stride) {
    T v[4], w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      v[u] = b[e + u * stride];
      w[u] = r[e + u * stride];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) r[e + u * stride] = v[u] - w[u];
  }
  for (; e < n; e += stride) r[e] = b[e] - r[e];
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int elem_blocks(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)std::max<size_t>(1, std::min<size_t>(b, 148 * 8));
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

template <typename T>
int k_mdot(const ReduceScratch& rs, const T* const* src, int cnt, const T* w, size_t n,
           bool with_self, double* out_dev, cudaStream_t s) {
  if (cnt < 0 || cnt > kMaxVecs) { set_error("bad vector count in multi-dot"); return CHEB_ERR_ARG; }
  VecList<T> L;
  bool vec = aligned16(w);
  for (int i = 0; i < kMaxVecs; ++i) {
    L.p[i] = i < cnt ? src[i] : nullptr;
    if (i < cnt) vec = vec && aligned16(src[i]);
  }
  const int nb = red_blocks(n);
  return count_dispatch(cnt, [&](auto c) -> int {
    mdot_kernel<T, decltype(c)::value><<<nb, kRedThreads, 0, s>>>(L, w, n, with_self ? 1 : 0, vec ? 1 : 0,
                                                                  rs.part, rs.counter, out_dev);
    CHEB_LAUNCH_CHECK("mdot_kernel");
    return CHEB_OK;
  });
}

template <typename T>
static int maxpy_launch(const ReduceScratch& rs, const T* const* src, const double* coef, const double* coef_dev,
                        double sign, int cnt, double beta, T* y, size_t n, double* norm2_dev, cudaStream_t s) {
  if (cnt < 0 || cnt > kMaxVecs) { set_error("bad vector count in multi-axpy"); return CHEB_ERR_ARG; }
  VecList<T> L;
  CoefList C;
  bool vec = aligned16(y);
  for (int i = 0; i < kMaxVecs; ++i) {
    L.p[i] = i < cnt ? src[i] : nullptr;
    C.c[i] = (i < cnt && coef) ? coef[i] : 0.0;
    if (i < cnt) vec = vec && aligned16(src[i]);
  }
  const int nb = red_blocks(n);
  return count_dispatch(cnt, [&](auto c) -> int {
    maxpy_kernel<T, decltype(c)::value><<<nb, kRedThreads, 0, s>>>(L, C, coef_dev, sign, beta, y, n,
                                                                   norm2_dev ? 1 : 0, vec ? 1 : 0, rs.part,
                                                                   rs.counter, norm2_dev);
    CHEB_LAUNCH_CHECK("maxpy_kernel");
    return CHEB_OK;
  });
}

template <typename T>
int k_maxpy(const ReduceScratch& rs, const T* const* src, const double* coef, int cnt, double beta,
            T* y, size_t n, double* norm2_dev, cudaStream_t s) {
  return maxpy_launch<T>(rs, src, coef, nullptr, 0.0, cnt, beta, y, n, norm2_dev, s);
}

template <typename T>
int k_maxpy_dev(const ReduceScratch& rs, const T* const* src, const double* coef_dev, double sign,
                int cnt, double beta, T* y, size_t n, double* norm2_dev, cudaStream_t s) {
  return maxpy_launch<T>(rs, src, nullptr, coef_dev, sign, cnt, beta, y, n, norm2_dev, s);
}

// y *= 1 / sqrt(*norm2) (when positive).  vec: y is 16-byte aligned, and
// each thread keeps four 16-byte loads in flight.
template <typename T>
__global__ void scale_inv_norm_kernel(T* __restrict__ y, const double* __restrict__ norm2, size_t n, int vec) {
  typedef typename Vec16<T>::t V;
  constexpr int W = Vec16<T>::W;
  const double nrm2 = *norm2;
  if (!(nrm2 > 0.0)) return;
  const T sv = (T)(1.0 / sqrt(nrm2));
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t nv = vec ? n / W : 0;
  V* y4 = reinterpret_cast<V*>(y);
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; e + 3 * stride < nv; e += 4 * stride) {
    V v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = y4[e + u * stride];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < W; ++k) Vec16<T>::set(v[u], k, sv * Vec16<T>::at(v[u], k));
      y4[e + u * stride] = v[u];
    }
  }
  for (; e < nv; e += stride) {
    V v = y4[e];
#pragma unroll
    for (int k = 0; k < W; ++k) Vec16<T>::set(v, k, sv * Vec16<T>::at(v, k));
    y4[e] = v;
  }
  for (size_t t = nv * W + blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += stride) y[t] *= sv;
}

template <typename T>
int k_scale_inv_norm(T* y, const double* norm2_dev, size_t n, cudaStream_t s) {
  scale_inv_norm_kernel<T><<<elem_blocks(n), 256, 0, s>>>(y, norm2_dev, n, aligned16(y) ? 1 : 0);
  CHEB_LAUNCH_CHECK("scale_inv_norm_kernel");
  return CHEB_OK;
}

__global__ void __launch_bounds__(kRedThreads)
sum_log_kernel(const double* __restrict__ K, size_t n, double* part, unsigned* counter, double* out) {
  double acc[1] = {0.0};
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += stride) acc[0] += log(K[e]);
  block_reduce_store<double, 1>(acc, 1, false, part, counter, out);
}

int k_sum_log(const ReduceScratch& rs, const double* K, size_t n, double* out_dev, cudaStream_t s) {
  sum_log_kernel<<<red_blocks(n), kRedThreads, 0, s>>>(K, n, rs.part, rs.counter, out_dev);
  CHEB_LAUNCH_CHECK("sum_log_kernel");
  return CHEB_OK;
}

// out = sum_{i,j,k} wx[i] wy[j] wz[k] a[c] b[c] over the field (c = (k ny + j)
// nx + i); a unit weight stands in for the weights of unused axes.
__global__ void __launch_bounds__(kRedThreads)
wsum3_kernel(const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ wx,
             const double* __restrict__ wy, const double* __restrict__ wz, int nx, int ny, size_t n,
             double* part, unsigned* counter, double* out) {
  double acc[1] = {0.0};
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t nxy = (size_t)nx * ny;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += stride) {
    const size_t k = e / nxy;
    const size_t r = e - k * nxy;
    const size_t j = r / nx;
    const size_t i = r - j * nx;
    double w = wx[i];
    if (wy) w *= wy[j];
    if (wz) w *= wz[k];
    acc[0] += w * a[e] * b[e];
  }
  block_reduce_store<double, 1>(acc, 1, false, part, counter, out);
}

int k_wsum3(const ReduceScratch& rs, const double* a, const double* b, const double* wx, const double* wy,
            const double* wz, int nx, int ny, size_t n, double* out_dev, cudaStream_t s) {
  wsum3_kernel<<<red_blocks(n), kRedThreads, 0, s>>>(a, b, wx, wy, wz, nx, ny, n, rs.part, rs.counter,
                                                     out_dev);
  CHEB_LAUNCH_CHECK("wsum3_kernel");
  return CHEB_OK;
}

template <typename T>
int k_scale(T* y, const T* x, double sc, size_t n, cudaStream_t s) {
  scale_kernel<T><<<elem_blocks(n), 256, 0, s>>>(y, x, sc, n);
  CHEB_LAUNCH_CHECK("scale_kernel");
  return CHEB_OK;
}

template <typename To, typename Ti>
int k_cast_scale(To* y, const Ti* x, double sc, size_t n, cudaStream_t s) {
  cast_scale_kernel<To, Ti><<<elem_blocks(n), 256, 0, s>>>(y, x, sc, n);
  CHEB_LAUNCH_CHECK("cast_scale_kernel");
  return CHEB_OK;
}

template <typename Ti>
int k_axpy64(double* y, const Ti* x, double sc, size_t n, cudaStream_t s) {
  axpy64_kernel<Ti><<<elem_blocks(n), 256, 0, s>>>(y, x, sc, n);
  CHEB_LAUNCH_CHECK("axpy64_kernel");
  return CHEB_OK;
}

template <typename T>
int k_residual(T* r, const T* b, size_t n, cudaStream_t s) {
  residual_kernel<T><<<elem_blocks(n), 256, 0, s>>>(r, b, n);
  CHEB_LAUNCH_CHECK("residual_kernel");
  return CHEB_OK;
}

template int k_mdot<double>(const ReduceScratch&, const double* const*, int, const double*, size_t, bool, double*, cudaStream_t);
template int k_mdot<float>(const ReduceScratch&, const float* const*, int, const float*, size_t, bool, double*, cudaStream_t);
template int k_maxpy<double>(const ReduceScratch&, const double* const*, const double*, int, double, double*, size_t, double*, cudaStream_t);
template int k_maxpy<float>(const ReduceScratch&, const float* const*, const double*, int, double, float*, size_t, double*, cudaStream_t);
template int k_maxpy_dev<double>(const ReduceScratch&, const double* const*, const double*, double, int, double, double*, size_t, double*, cudaStream_t);
template int k_maxpy_dev<float>(const ReduceScratch&, const float* const*, const double*, double, int, double, float*, size_t, double*, cudaStream_t);
template int k_scale_inv_norm<double>(double*, const double*, size_t, cudaStream_t);
template int k_scale_inv_norm<float>(float*, const double*, size_t, cudaStream_t);
template int k_scale<double>(double*, const double*, double, size_t, cudaStream_t);
template int k_scale<float>(float*, const float*, double, size_t, cudaStream_t);
template int k_cast_scale<float, double>(float*, const double*, double, size_t, cudaStream_t);
template int k_cast_scale<double, float>(double*, const float*, double, size_t, cudaStream_t);
template int k_cast_scale<double, double>(double*, const double*, double, size_t, cudaStream_t);
template int k_axpy64<float>(double*, const float*, double, size_t, cudaStream_t);
template int k_axpy64<double>(double*, const double*, double, size_t, cudaStream_t);
template int k_residual<double>(double*, const double*, size_t, cudaStream_t);
template int k_residual<float>(float*, const float*, size_t, cudaStream_t);

}  // namespace cheb
