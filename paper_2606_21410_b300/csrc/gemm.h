// Row-major batched GEMM launcher (gemm.cu).
#pragma once

#include "internal.h"

namespace cheb {

// C[b] = A[b] B[b] for b < batch; A: M x K (lda), B: K x N (ldb), C: M x N (ldc);
// sA, sB, sC: element strides between batch entries.
template <typename T>
int k_gemm(int M, int N, int K, const T* A, int lda, long long sA, const T* B, int ldb,
           long long sB, T* C, int ldc, long long sC, int batch, cudaStream_t s);

// FP32 GEMM on the tensor cores with split-TF32 (3xTF32) arithmetic; same
// argument meaning as k_gemm; K, ld and strides multiples of 4, 16-byte
// aligned operands.
int k_gemm_tf32x3(int M, int N, int K, const float* A, int lda, long long sA, const float* B, int ldb,
                  long long sB, float* C, int ldc, long long sC, int batch, cudaStream_t s);
bool tf32x3_ok(int K, const void* A, int lda, long long sA, const void* B, int ldb, long long sB);

}  // namespace cheb
