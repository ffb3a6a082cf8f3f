// Tiled SIMT GEMM for the per-axis dense contractions of the fast-
// diagonalization preconditioner: C[b] = A[b] B[b], row-major, batched by
// strides.  64 x 64 block tile, 16-deep K slices in shared memory, 4 x 4
// outputs per thread.
#include "gemm.h"

namespace cheb {

template <typename T>
__global__ void __launch_bounds__(256)
gemm_kernel(int M, int N, int K, const T* __restrict__ A, int lda, long long sA,
            const T* __restrict__ B, int ldb, long long sB, T* __restrict__ C, int ldc,
            long long sC) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const long long bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      const int r = e / BK, c = e % BK;
      const int gm = m0 + r, gk = k0 + c;
      As[c][r] = (gm < M && gk < K) ? A[(long long)gm * lda + gk] : (T)0;
    }
#pragma unroll
    for (int e = threadIdx.x; e < BK * BN; e += 256) {
      const int r = e / BN, c = e % BN;
      const int gk = k0 + r, gn = n0 + c;
      Bs[r][c] = (gk < K && gn < N) ? B[(long long)gk * ldb + gn] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn < N) C[(long long)gm * ldc + gn] = acc[i][j];
    }
  }
}

template <typename T>
int k_gemm(int M, int N, int K, const T* A, int lda, long long sA, const T* B, int ldb,
           long long sB, T* C, int ldc, long long sC, int batch, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return CHEB_OK;
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
  gemm_kernel<T><<<grid, 256, 0, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC);
  CHEB_LAUNCH_CHECK("gemm_kernel");
  return CHEB_OK;
}

template int k_gemm<double>(int, int, int, const double*, int, long long, const double*, int, long long, double*, int, long long, int, cudaStream_t);
template int k_gemm<float>(int, int, int, const float*, int, long long, const float*, int, long long, float*, int, long long, int, cudaStream_t);

}  // namespace cheb
