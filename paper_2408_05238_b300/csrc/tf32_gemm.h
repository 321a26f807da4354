// FP64-operand GEMM on the TF32 tensor cores with split operands
// (tf32_gemm.cu): 3xTF32 (terms = 3) or plain TF32 (terms = 1).
#pragma once

#include "internal.h"

namespace lls {

// Device bytes of the workspace tf32_gemm needs for an m x n x k product.
size_t tf32_gemm_workspace_bytes(int64_t m, int64_t n, int64_t k, int terms);

// C = alpha op(A) op(B) + beta C, operand conventions of gemm().  err: device
// int raised when a device-side wait timed out.
Status tf32_gemm(bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t m, int64_t n, int64_t k,
                 double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                 double beta, double* C, int64_t ldc, int terms, Scratch ws, int* err,
                 cudaStream_t st);

}  // namespace lls
