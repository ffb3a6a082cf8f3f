// Row-major batched GEMM launcher (gemm.cu).
#pragma once

#include "internal.h"

namespace cheb {

// C[b] = A[b] B[b] for b < batch; A: M x K (lda), B: K x N (ldb), C: M x N (ldc);
// sA, sB, sC: element strides between batch entries.
template <typename T>
int k_gemm(int M, int N, int K, const T* A, int lda, long long sA, const T* B, int ldb,
           long long sB, T* C, int ldc, long long sC, int batch, cudaStream_t s);

}  // namespace cheb
