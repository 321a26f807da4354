// tcgen05 BF16 GEMM (tc_gemm_bf16.cu): D (M x N, FP32, column-major) =
// X^T Z with X K x M and Z K x N column-major BF16 (ld % 8 == 0, 16-byte
// aligned), N <= 128.  err: device int raised on a timed-out wait.
#pragma once

#include "internal.h"

namespace lls {

size_t tc_gemm_scratch_bytes(int M, int N, int K);
Status tc_gemm_bf16(int M, int N, int K, const void* X, int64_t ldx, const void* Z, int64_t ldz,
                    float* D, int64_t ldd, Scratch scratch, int* err, cudaStream_t st);

}  // namespace lls
