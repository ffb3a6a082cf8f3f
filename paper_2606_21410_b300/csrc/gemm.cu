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

// ---------------------------------------------------------------------------
// FP32 GEMM on the tensor cores with split-TF32 arithmetic ("3xTF32"): each
// operand x = x_hi + x_lo with x_hi = tf32(x), x_lo = tf32(x - x_hi), and
// a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, accumulated in FP32 (relative
// error close to FP32 arithmetic).  mma.sync m16n8k8 TF32 tiles; 128 x 128
// block tile, 8 warps of 64 x 32, BK = 16 with cp.async double buffering.
// Needs K, lda, ldb, ldc, strides multiples of 4 and 16-byte aligned
// pointers (rows are read as 16-byte chunks); M and N are arbitrary.
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ unsigned to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void cp16(void* sdst, const void* gsrc, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  const int bytes = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc), "r"(bytes) : "memory");
}
}  // namespace

__global__ void __launch_bounds__(256)
gemm_tf32x3_kernel(int M, int N, int K, const float* __restrict__ A, int lda, long long sA,
                   const float* __restrict__ B, int ldb, long long sB, float* __restrict__ C, int ldc,
                   long long sC) {
  constexpr int BM = 128, BN = 128, BK = 16, APAD = 4, BPAD = 8;
  __shared__ __align__(16) float As[2][BM][BK + APAD];
  __shared__ __align__(16) float Bs[2][BK][BN + BPAD];
  const long long bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;      // 2 x 4 warps
  const int g = lane >> 2, tig = lane & 3;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

  auto load_tile = [&](int buf, int k0) {
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int c = tid + it * 256;         // 512 chunks of 4 floats
      const int r = c >> 2, kc = (c & 3) * 4;
      const bool v = (m0 + r < M) && (k0 + kc < K);
      cp16(&As[buf][r][kc], v ? (const void*)(A + (long long)(m0 + r) * lda + k0 + kc) : (const void*)A, v);
    }
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int c = tid + it * 256;
      const int k = c >> 5, nc = (c & 31) * 4;
      const bool v = (k0 + k < K) && (n0 + nc < N);
      cp16(&Bs[buf][k][nc], v ? (const void*)(B + (long long)(k0 + k) * ldb + n0 + nc) : (const void*)B, v);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  const int ktiles = (K + BK - 1) / BK;
  load_tile(0, 0);
  for (int kt = 0; kt < ktiles; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < ktiles) {
      load_tile(cur ^ 1, (kt + 1) * BK);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 8) {
      unsigned ahi[4][4], alo[4][4], bhi[4][2], blo[4][2];
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const int r = wm * 64 + mt * 16 + g;
        const float x[4] = {As[cur][r][ks + tig], As[cur][r + 8][ks + tig], As[cur][r][ks + tig + 4],
                            As[cur][r + 8][ks + tig + 4]};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ahi[mt][q] = to_tf32(x[q]);
          alo[mt][q] = to_tf32(x[q] - __uint_as_float(ahi[mt][q]));
        }
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int cidx = wn * 32 + nt * 8 + g;
        const float y0 = Bs[cur][ks + tig][cidx], y1 = Bs[cur][ks + tig + 4][cidx];
        bhi[nt][0] = to_tf32(y0);
        bhi[nt][1] = to_tf32(y1);
        blo[nt][0] = to_tf32(y0 - __uint_as_float(bhi[nt][0]));
        blo[nt][1] = to_tf32(y1 - __uint_as_float(bhi[nt][1]));
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          mma_tf32(acc[mt][nt], alo[mt], bhi[nt]);
          mma_tf32(acc[mt][nt], ahi[mt], blo[nt]);
          mma_tf32(acc[mt][nt], ahi[mt], bhi[nt]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int r = m0 + wm * 64 + mt * 16 + g;
      const int cidx = n0 + wn * 32 + nt * 8 + 2 * tig;
      if (r < M) {
        if (cidx < N) C[(long long)r * ldc + cidx] = acc[mt][nt][0];
        if (cidx + 1 < N) C[(long long)r * ldc + cidx + 1] = acc[mt][nt][1];
      }
      if (r + 8 < M) {
        if (cidx < N) C[(long long)(r + 8) * ldc + cidx] = acc[mt][nt][2];
        if (cidx + 1 < N) C[(long long)(r + 8) * ldc + cidx + 1] = acc[mt][nt][3];
      }
    }
}

namespace cheb {

bool tf32x3_ok(int K, const void* A, int lda, long long sA, const void* B, int ldb, long long sB) {
  return K % 4 == 0 && lda % 4 == 0 && ldb % 4 == 0 && sA % 4 == 0 && sB % 4 == 0 &&
         ((size_t)A & 15) == 0 && ((size_t)B & 15) == 0;
}

int k_gemm_tf32x3(int M, int N, int K, const float* A, int lda, long long sA, const float* B, int ldb,
                  long long sB, float* C, int ldc, long long sC, int batch, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return CHEB_OK;
  if (!tf32x3_ok(K, A, lda, sA, B, ldb, sB)) {
    set_error("tensor-core GEMM needs 16-byte aligned operands and K, ld multiples of 4");
    return CHEB_ERR_ARG;
  }
  dim3 grid((N + 127) / 128, (M + 127) / 128, batch);
  gemm_tf32x3_kernel<<<grid, 256, 0, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC);
  CHEB_LAUNCH_CHECK("gemm_tf32x3_kernel");
  return CHEB_OK;
}

}  // namespace cheb
