// Block reflectors applied to a few vectors: the replays of the solve of
// Fig. 4 (c = U^T b by steps, x = V z in reverse step order) and of its
// transpose (the refinement of the TF32 modes), for nrhs <= kThinMaxRhs.
//
// x (M x nrhs) <- (I - W op(T) W^T) x with W the M x b unit lower
// trapezoidal reflector block of one step and T its b x b upper triangular
// compact-WY factor, op(T) = T or T^T, in three launches:
//  1. thin_partials_kernel: each CTA sums W(r, j) x(r, c) over its chunk of
//     rows (the x chunk staged in shared memory, one warp per column of W);
//  2. thin_reduce_kernel: one CTA per right-hand side adds the chunks'
//     partial sums in chunk order and forms p2 = op(T) (W^T x);
//  3. thin_update_kernel: x(r, c) -= sum_j W(r, j) p2(j, c) on every row.
// The general GEMM path launches several split-K products per step and
// spends most of its time in launches for nrhs = 1; this reads W twice per
// step at HBM speed.  Every sum runs in a fixed order, so results are
// bit-identical run to run.
#include <algorithm>

#include "internal.h"

namespace lls {
namespace {

constexpr int TH_THREADS = 256;
constexpr int TH_ROWS = 256;  // rows per CTA chunk

__device__ __forceinline__ double w_unit_lower(const double* W, int64_t ldw, int64_t r, int j) {
  if (r < j) return 0.0;
  if (r == j) return 1.0;
  return W[r + (int64_t)j * ldw];
}

__global__ void __launch_bounds__(TH_THREADS) thin_partials_kernel(int64_t M, int b, int nrhs,
                                                                    const double* __restrict__ W,
                                                                    int64_t ldw,
                                                                    const double* __restrict__ x,
                                                                    int64_t ldx,
                                                                    double* __restrict__ part) {
  __shared__ double xs[TH_ROWS * kThinMaxRhs];
  const int64_t r0 = (int64_t)blockIdx.x * TH_ROWS;
  const int rows = (int)(M - r0 < TH_ROWS ? M - r0 : TH_ROWS);
  for (int e = threadIdx.x; e < rows * nrhs; e += TH_THREADS)
    xs[(e % rows) + (e / rows) * TH_ROWS] = x[r0 + (e % rows) + (int64_t)(e / rows) * ldx];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* out = part + (int64_t)blockIdx.x * b * nrhs;
  for (int j = warp; j < b; j += TH_THREADS / 32) {
    double acc[kThinMaxRhs];
#pragma unroll
    for (int c = 0; c < kThinMaxRhs; ++c) acc[c] = 0.0;
    for (int rr = lane; rr < rows; rr += 32) {
      const double w = w_unit_lower(W, ldw, r0 + rr, j);
#pragma unroll
      for (int c = 0; c < kThinMaxRhs; ++c)
        if (c < nrhs) acc[c] = fma(w, xs[rr + c * TH_ROWS], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kThinMaxRhs; ++c) {
      if (c >= nrhs) break;
      double s = acc[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) out[j + c * b] = s;
    }
  }
}

// One CTA per right-hand side c: p = sum over chunks of the partials (chunk
// order), p2 = op(T) p.
__global__ void __launch_bounds__(TH_THREADS) thin_reduce_kernel(int b, int nrhs, int chunks,
                                                                  const double* __restrict__ part,
                                                                  const double* __restrict__ T,
                                                                  int64_t ldt, int transT,
                                                                  double* __restrict__ p2) {
  __shared__ double p[128];
  const int c = blockIdx.x;
  for (int j = threadIdx.x; j < b; j += TH_THREADS) {
    double s = 0.0;
    for (int g = 0; g < chunks; ++g) s += part[(int64_t)g * b * nrhs + j + c * b];
    p[j] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < b; i += TH_THREADS) {
    double s = 0.0;
    if (!transT) {
      for (int l = i; l < b; ++l) s = fma(T[i + (int64_t)l * ldt], p[l], s);
    } else {
      for (int l = 0; l <= i; ++l) s = fma(T[l + (int64_t)i * ldt], p[l], s);
    }
    p2[i + c * b] = s;
  }
}

__global__ void __launch_bounds__(TH_THREADS) thin_update_kernel(int64_t M, int b, int nrhs,
                                                                  const double* __restrict__ W,
                                                                  int64_t ldw,
                                                                  const double* __restrict__ p2,
                                                                  double* __restrict__ x,
                                                                  int64_t ldx) {
  __shared__ double ps[128 * kThinMaxRhs];
  for (int e = threadIdx.x; e < b * nrhs; e += TH_THREADS) ps[e] = p2[e];
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * TH_THREADS + threadIdx.x;
  if (r >= M) return;
  double acc[kThinMaxRhs];
#pragma unroll
  for (int c = 0; c < kThinMaxRhs; ++c) acc[c] = 0.0;
  const int jmax = (int)(r + 1 < b ? r + 1 : b);  // W(r, j) = 0 for j > r
  for (int j = 0; j < jmax; ++j) {
    const double w = w_unit_lower(W, ldw, r, j);
#pragma unroll
    for (int c = 0; c < kThinMaxRhs; ++c)
      if (c < nrhs) acc[c] = fma(w, ps[j + c * b], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < kThinMaxRhs; ++c)
    if (c < nrhs) x[r + (int64_t)c * ldx] -= acc[c];
}

// x(0:b) <- op(S) x(0:b) for a b x b block S, one CTA per right-hand side.
__global__ void __launch_bounds__(128) thin_small_mul_kernel(int b, const double* __restrict__ S,
                                                             int64_t lds, int transS, double* x,
                                                             int64_t ldx) {
  __shared__ double xs[128];
  double* xc = x + (int64_t)blockIdx.x * ldx;
  for (int i = threadIdx.x; i < b; i += 128) xs[i] = xc[i];
  __syncthreads();
  for (int i = threadIdx.x; i < b; i += 128) {
    double s = 0.0;
    for (int l = 0; l < b; ++l)
      s = fma(transS ? S[l + (int64_t)i * lds] : S[i + (int64_t)l * lds], xs[l], s);
    xc[i] = s;
  }
}

}  // namespace

size_t thin_scratch_bytes(int64_t M, int64_t b, int64_t nrhs) {
  return sizeof(double) * ((size_t)ceil_div(M, TH_ROWS) * b * nrhs + (size_t)b * nrhs);
}

Status apply_reflectors_thin(int64_t M, int64_t b, int64_t nrhs, const double* W, int64_t ldw,
                             const double* T, int64_t ldt, bool transT, double* x, int64_t ldx,
                             Scratch scratch, cudaStream_t st) {
  if (M <= 0 || b <= 0 || nrhs <= 0) return ok_status();
  if (b > 128 || nrhs > kThinMaxRhs)
    return make_error(LLS_ERR_ARG, "apply_reflectors_thin: b <= 128 and nrhs <= 16");
  if (scratch.bytes < thin_scratch_bytes(M, b, nrhs))
    return make_error(LLS_ERR_NOMEM, "apply_reflectors_thin: scratch too small");
  const int64_t chunks = ceil_div(M, TH_ROWS);
  if (chunks > INT32_MAX) return make_error(LLS_ERR_ARG, "apply_reflectors_thin: too many rows");
  double* part = static_cast<double*>(scratch.ptr);
  double* p2 = part + (size_t)chunks * b * nrhs;
  TraceScope ts(kTrSmall, st, 4.0 * M * b * nrhs, 16.0 * M * b);
  thin_partials_kernel<<<(unsigned)chunks, TH_THREADS, 0, st>>>(M, (int)b, (int)nrhs, W, ldw, x,
                                                                 ldx, part);
  LLS_LAUNCHED("thin_partials_kernel");
  thin_reduce_kernel<<<(unsigned)nrhs, TH_THREADS, 0, st>>>((int)b, (int)nrhs, (int)chunks, part, T,
                                                            ldt, transT ? 1 : 0, p2);
  LLS_LAUNCHED("thin_reduce_kernel");
  thin_update_kernel<<<(unsigned)ceil_div(M, TH_THREADS), TH_THREADS, 0, st>>>(M, (int)b, (int)nrhs,
                                                                               W, ldw, p2, x, ldx);
  LLS_LAUNCHED("thin_update_kernel");
  return ok_status();
}

Status small_block_mul(int64_t b, int64_t nrhs, const double* S, int64_t lds, bool transS,
                       double* x, int64_t ldx, cudaStream_t st) {
  if (b <= 0 || nrhs <= 0) return ok_status();
  if (b > 128) return make_error(LLS_ERR_ARG, "small_block_mul: b <= 128");
  TraceScope ts(kTrSmall, st);
  thin_small_mul_kernel<<<(unsigned)nrhs, 128, 0, st>>>((int)b, S, lds, transS ? 1 : 0, x, ldx);
  LLS_LAUNCHED("thin_small_mul_kernel");
  return ok_status();
}

}  // namespace lls
