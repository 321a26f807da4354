// Mixed-precision sampling (step a2 of Fig. 2): Y = (A^T A)^q A^T G with the
// products in BF16 on the tcgen05 tensor cores and FP32 accumulation.
//
// Only the sample Y is computed in low precision.  Y merely chooses the
// orthogonal V of the step (its span is what matters); T = U^T A V is still
// formed by the FP64 Householder QR of Y and the FP64 updates, so the
// factorization stays exact to FP64 rounding whatever Y is.  Per step:
//   1. s = 2^-e with 2^e >= sqrt(m n) max |A| of the whole matrix (exact
//      power-of-two scaling, from one pass over A at the first step: the
//      steps' orthogonal updates keep every entry of T below ||A||_F <=
//      sqrt(m n) max |A|, so the later steps need no pass of their own);
//   2. A16 = bf16(s A_BR) (m' x n') and A16t = its transpose, one pass;
//   3. G16 = bf16 of the same Philox sketch as the FP64 path;
//   4. Y = A16^T G16; then q times W = A16t^T Y16, Y = A16^T W16, each
//      intermediate rescaled by a power of two and rounded to BF16;
//   5. Y is written as FP64 into the W_V buffer for the FP64 QR.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "solver.h"
#include "tc_gemm.h"

namespace lls {
namespace {

// FP64 arithmetic issues at a small fraction of the integer rate on this
// part, so the conversions below work on the bits: |x| compares as its
// 63-bit pattern, the power-of-two scaling is a shift of the exponent field
// and the rounding to BF16 is done on the mantissa bits.

__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

// max |A(i, j)| as its bit pattern (a NaN-free input, checked on entry):
// block (row group of 1024, column group), four rows per thread, two
// columns per pass, so eight loads are in flight per thread.
__global__ void __launch_bounds__(256) maxabs_f64_kernel(int64_t m, int64_t n,
                                                         const double* __restrict__ A,
                                                         int64_t lda, unsigned long long* out) {
  unsigned long long mx = 0;
  const int64_t i0 = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  for (int64_t j = blockIdx.y; j < n; j += 2 * (int64_t)gridDim.y) {
    const int64_t j2 = j + gridDim.y;
    double v[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + 256 * u;
      v[u] = i < m ? __ldg(A + i + j * lda) : 0.0;
      v[4 + u] = (i < m && j2 < n) ? __ldg(A + i + j2 * lda) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const unsigned long long b = abs_bits(v[u]);
      mx = b > mx ? b : mx;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = t > mx ? t : mx;
  }
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

__global__ void maxabs_f32_kernel(int64_t m, int64_t n, const float* __restrict__ A, int64_t lda,
                                  unsigned int* out) {
  float mx = 0.f;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    float v = fabsf(A[(idx % m) + (idx / m) * lda]);
    mx = v > mx ? v : mx;
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));
}

// Power of two 2^-e with 2^e >= maxabs (1 when maxabs is 0).
__device__ __forceinline__ double pow2_scale(double maxabs) {
  if (!(maxabs > 0.0)) return 1.0;
  int e;
  frexp(maxabs, &e);  // maxabs = f 2^e, f in [0.5, 1)
  return ldexp(1.0, -e);
}

// The e of pow2_scale from the maximum's bits: 2^e > max (frexp convention).
__device__ __forceinline__ int scale_exp(unsigned long long maxbits) {
  const int E = (int)(maxbits >> 52);
  return maxbits == 0 ? 0 : (E == 0 ? -1021 : E - 1022);
}

// bf16(v 2^-e) from the bits of v, rounded to nearest with ties to even on
// the 45 dropped mantissa bits; values that fall below BF16's normal range
// (below 2^-126, i.e. 2^-126 relative to the scaled maximum 1) become +-0.
__device__ __forceinline__ unsigned short bf16_scaled_bits(double v, int e) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned short sgn = (unsigned short)((u >> 63) << 15);
  const int E = (int)((u >> 52) & 0x7FF);
  int eb = E - e - 1023 + 127;
  if (E == 0 || eb <= 0) return sgn;
  const unsigned long long mant = u & ((1ull << 52) - 1);
  unsigned int m7 = (unsigned int)(mant >> 45);
  const unsigned long long rem = mant & ((1ull << 45) - 1), half = 1ull << 44;
  if (rem > half || (rem == half && (m7 & 1u))) {
    if (++m7 == 128u) {
      m7 = 0;
      ++eb;
    }
  }
  return (unsigned short)(sgn | (unsigned short)(eb << 7) | (unsigned short)m7);
}

// A16 (m x n, ld16) and A16t (n x m, ld16t) = bf16(2^-e A), through a 32 x 32
// shared-memory tile so both writes are coalesced; the four loads of a
// thread are issued before any conversion.
__global__ void __launch_bounds__(256) convert_transpose_kernel(
    int64_t m, int64_t n, const double* __restrict__ A, int64_t lda,
    const unsigned long long* maxbits, int extra, __nv_bfloat16* __restrict__ A16, int64_t ld16,
    __nv_bfloat16* __restrict__ A16t, int64_t ld16t) {
  __shared__ unsigned short tile[32][33];
  const int e = scale_exp(*maxbits) + extra;
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int64_t i = i0 + tx;
  double v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t j = j0 + ty + 8 * q;
    v[q] = (i < m && j < n) ? __ldg(A + i + j * lda) : 0.0;
  }
  unsigned short* a16 = reinterpret_cast<unsigned short*>(A16);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = ty + 8 * q;
    const int64_t j = j0 + r;
    const unsigned short bits = bf16_scaled_bits(v[q], e);
    if (i < m && j < n) a16[i + j * ld16] = bits;
    tile[r][tx] = bits;
  }
  __syncthreads();
  unsigned short* a16t = reinterpret_cast<unsigned short*>(A16t);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = ty + 8 * q;
    const int64_t j = j0 + tx, ii = i0 + r;
    if (ii < m && j < n) a16t[j + ii * ld16t] = tile[tx][r];
  }
}

__global__ void f32_to_bf16_kernel(int64_t m, int64_t n, const float* __restrict__ X, int64_t ldx,
                                   const unsigned int* maxbits, __nv_bfloat16* __restrict__ Y,
                                   int64_t ldy) {
  const double s = pow2_scale((double)__uint_as_float(*maxbits));
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % m, j = idx / m;
    Y[i + j * ldy] = __float2bfloat16((float)((double)X[i + j * ldx] * s));
  }
}

__global__ void f32_to_f64_kernel(int64_t m, int64_t n, const float* __restrict__ X, int64_t ldx,
                                  double* __restrict__ Y, int64_t ldy) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % m, j = idx / m;
    Y[i + j * ldy] = (double)X[i + j * ldx];
  }
}

unsigned grid_of(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 148 * 16));
}

int64_t pad8(int64_t x) { return std::max<int64_t>(8, (x + 7) / 8 * 8); }

}  // namespace

Status sample_bf16(Handle& h, const double* A, int64_t lda, int64_t mp, int64_t np, int64_t b,
                   int q, uint64_t seed, int64_t step, double* Y, int64_t ldy) {
  cudaStream_t st = h.stream;
  if (b > 128) return make_error(LLS_ERR_ARG, "mixed precision sampling needs nb <= 128", 2);
  if (mp > INT32_MAX || np > INT32_MAX) return make_error(LLS_ERR_ARG, "matrix too large");
  const int64_t ld16 = pad8(mp), ld16t = pad8(np);
  const int64_t mx = std::max(mp, np);
  LLS_TRY(h.A16.reserve(2 * (size_t)ld16 * std::max<int64_t>(np, 1)));
  LLS_TRY(h.A16t.reserve(2 * (size_t)ld16t * std::max<int64_t>(mp, 1)));
  LLS_TRY(h.G16.reserve(2 * (size_t)ld16 * 128));
  LLS_TRY(h.Z16.reserve(2 * (size_t)pad8(mx) * 128));
  LLS_TRY(h.F32.reserve(4 * (size_t)mx * 128));
  LLS_TRY(h.tc_ws.reserve(std::max(tc_gemm_scratch_bytes((int)np, (int)b, (int)mp),
                                   tc_gemm_scratch_bytes((int)mp, (int)b, (int)np))));
  LLS_TRY(h.mixed_misc.reserve(64));
  unsigned long long* amax = h.mixed_misc.as<unsigned long long>();
  unsigned int* fmax = reinterpret_cast<unsigned int*>(amax + 1);
  DevStatus* ds = h.dstat.as<DevStatus>();
  Scratch tws{h.tc_ws.p, h.tc_ws.bytes};
  auto* A16 = h.A16.as<__nv_bfloat16>();
  auto* A16t = h.A16t.as<__nv_bfloat16>();
  auto* G16 = h.G16.as<__nv_bfloat16>();
  auto* Z16 = h.Z16.as<__nv_bfloat16>();
  float* F = h.F32.as<float>();

  {
    TraceScope ts(kTrConvertBf16, st, 0.0, (step == 0 ? 8.0 : 0.0) * mp * np + (8.0 + 4.0) * mp * np);
    if (step == 0) {  // max |A| of the whole matrix, and the bound sqrt(m n) on its growth
      LLS_CUDA(cudaMemsetAsync(amax, 0, 16, st));
      const unsigned gx = (unsigned)ceil_div(mp, 1024);
      const unsigned gy = (unsigned)std::max<int64_t>(
          1, std::min<int64_t>({np, 65535, ceil_div(148 * 8, gx)}));
      maxabs_f64_kernel<<<dim3(gx, gy), 256, 0, st>>>(mp, np, A, lda, amax);
      LLS_LAUNCHED("maxabs_f64_kernel");
      h.bf16_scale_extra = (int)std::ceil(0.5 * std::log2(std::max(1.0, (double)mp * (double)np)));
    }
    dim3 grid((unsigned)ceil_div(mp, 32), (unsigned)ceil_div(np, 32));
    convert_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(mp, np, A, lda, amax, h.bf16_scale_extra,
                                                           A16, ld16, A16t, ld16t);
    LLS_LAUNCHED("convert_transpose_kernel");
  }
  LLS_TRY(launch_sketch_bf16(seed, step, mp, b, G16, ld16, st));
  // Y = A^T G  (X = A16: K = m', M = n')
  LLS_TRY(tc_gemm_bf16((int)np, (int)b, (int)mp, A16, ld16, G16, ld16, F, np, tws,
                       &ds->barrier_err, st));
  for (int it = 0; it < q; ++it) {
    // Y16 <- Y, W = A Y  (X = A16t: K = n', M = m')
    LLS_CUDA(cudaMemsetAsync(fmax, 0, 4, st));
    maxabs_f32_kernel<<<grid_of(np * b), 256, 0, st>>>(np, b, F, np, fmax);
    LLS_LAUNCHED("maxabs_f32_kernel");
    f32_to_bf16_kernel<<<grid_of(np * b), 256, 0, st>>>(np, b, F, np, fmax, Z16, ld16t);
    LLS_LAUNCHED("f32_to_bf16_kernel");
    LLS_TRY(tc_gemm_bf16((int)mp, (int)b, (int)np, A16t, ld16t, Z16, ld16t, F, mp, tws,
                         &ds->barrier_err, st));
    // W16 <- W, Y = A^T W
    LLS_CUDA(cudaMemsetAsync(fmax, 0, 4, st));
    maxabs_f32_kernel<<<grid_of(mp * b), 256, 0, st>>>(mp, b, F, mp, fmax);
    LLS_LAUNCHED("maxabs_f32_kernel");
    f32_to_bf16_kernel<<<grid_of(mp * b), 256, 0, st>>>(mp, b, F, mp, fmax, Z16, ld16);
    LLS_LAUNCHED("f32_to_bf16_kernel");
    LLS_TRY(tc_gemm_bf16((int)np, (int)b, (int)mp, A16, ld16, Z16, ld16, F, np, tws,
                         &ds->barrier_err, st));
  }
  f32_to_f64_kernel<<<grid_of(np * b), 256, 0, st>>>(np, b, F, np, Y, ldy);
  LLS_LAUNCHED("f32_to_f64_kernel");
  return ok_status();
}

}  // namespace lls
