// FP64-accurate GEMM on the BF16 tensor cores by exact slicing (oz_gemm.cu).
#pragma once

#include <cuda_bf16.h>

#include "internal.h"

namespace lls {

// Device bytes of the workspace oz_gemm needs for an m x n x k product.
size_t oz_gemm_workspace_bytes(int64_t m, int64_t n, int64_t k);

// C = alpha op(A) op(B) + beta C, same operand conventions as gemm();
// transC stores the m x n result transposed (C[j + i ldc]).  err: device
// int raised when a device-side wait timed out.
Status oz_gemm(bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t m, int64_t n, int64_t k,
               double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
               double beta, double* C, int64_t ldc, bool transC, Scratch ws, int* err,
               cudaStream_t st);

}  // namespace lls
