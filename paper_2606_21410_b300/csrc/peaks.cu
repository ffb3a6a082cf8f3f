// Throughput probe of the CUDA-core FMA pipes (FP64 and FP32), the peaks the
// ALU-bound kernels of the library are measured against.  Every thread runs
// kChains independent fused multiply-add recurrences x <- x * a + b for
// `iters` steps (a, b kernel arguments, so nothing folds at compile time;
// |a| < 1 keeps the values bounded), enough threads per SM to hide the pipe
// latency; one FMA counts as two flops.  Timed with CUDA events around
// back-to-back launches on a private stream.
#include <algorithm>

#include "internal.h"

namespace cheb {

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + 1 + c) * (T)1e-3;
#pragma unroll 16
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-1) out[blockIdx.x] = s;  // never true; keeps the chains live
}

template <typename T>
int run_peak(double* tflops, double* ms_out) {
  int dev = 0, sms = 0;
  CHEB_CUDA(cudaGetDevice(&dev));
  CHEB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8;  // 2048 threads per SM
  T* out = nullptr;
  CHEB_CUDA(cudaMalloc(&out, sizeof(T) * blocks));
  cudaStream_t s = nullptr;
  CHEB_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CHEB_CUDA(cudaEventCreate(&e0));
  CHEB_CUDA(cudaEventCreate(&e1));
  const T a = (T)0.999999, b = (T)1e-7;
  // calibrate the length to about 20 ms per launch
  int iters = sizeof(T) == 8 ? 1024 : 16384;
  float t = 0.f;
  int st = CHEB_OK;
  for (int cal = 0; cal < 8 && st == CHEB_OK; ++cal) {
    cudaEventRecord(e0, s);
    fma_peak_kernel<T><<<blocks, kPeakThreads, 0, s>>>(out, iters, a, b);
    count_launch();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) { st = cuda_fail(cudaGetLastError(), "fma_peak_kernel"); break; }
    cudaEventElapsedTime(&t, e0, e1);
    if (t >= 15.f) break;
    iters = (int)std::min<double>(1 << 24, iters * std::max(2.0, 20.0 / std::max(t, 0.05f)));
  }
  const int reps = 5;
  if (st == CHEB_OK) {
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) {
      fma_peak_kernel<T><<<blocks, kPeakThreads, 0, s>>>(out, iters, a, b);
      count_launch();
    }
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "fma_peak_kernel");
    else cudaEventElapsedTime(&t, e0, e1);
  }
  if (st == CHEB_OK) {
    const double flops = 2.0 * kChains * (double)iters * blocks * kPeakThreads * reps;
    *tflops = flops / (t * 1e-3) / 1e12;
    if (ms_out) *ms_out = t / reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  cudaFree(out);
  return st;
}

}  // namespace

}  // namespace cheb

using namespace cheb;

extern "C" int cheb_fma_peak(int prec, double* tflops, double* ms_per_launch) {
  if (!tflops) { set_error("null argument"); return CHEB_ERR_ARG; }
  if (prec == CHEB_FP64) return run_peak<double>(tflops, ms_per_launch);
  if (prec == CHEB_FP32) return run_peak<float>(tflops, ms_per_launch);
  set_error("prec must be CHEB_FP64 or CHEB_FP32");
  return CHEB_ERR_ARG;
}
