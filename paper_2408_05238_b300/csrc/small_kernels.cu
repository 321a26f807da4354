// Memory-bound helpers of the solver: input copy with the finiteness check,
// block copies and reversals used by Nullify, the diagonal-block write of the
// SVD step, Compute_rank, and the blocked triangular solve of Fig. 4.
#include <algorithm>

#include "internal.h"
#include "lls_kernels.h"

namespace lls {
namespace {

constexpr int EW = 256;  // threads per CTA for elementwise kernels

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, EW), 1 << 20)); }

__global__ void copy_check_kernel(int64_t m, int64_t n, const double* __restrict__ src, int64_t lds,
                                  double* __restrict__ dst, int64_t ldd, int* flag) {
  int bad = 0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % m, j = idx / m;
    double v = src[i + j * lds];
    bad |= !isfinite(v);
    if (dst) dst[i + j * ldd] = v;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

__global__ void copy_kernel(int64_t m, int64_t n, const double* __restrict__ src, int64_t lds,
                            double* __restrict__ dst, int64_t ldd) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % m, j = idx / m;
    dst[i + j * ldd] = src[i + j * lds];
  }
}

__global__ void axpy_kernel(int64_t m, int64_t n, double alpha, const double* __restrict__ X,
                            int64_t ldx, double* __restrict__ Y, int64_t ldy) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % m, j = idx / m;
    Y[i + j * ldy] = fma(alpha, X[i + j * ldx], Y[i + j * ldy]);
  }
}

__global__ void zero_kernel(int64_t m, int64_t n, double* dst, int64_t ldd) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
       idx += (int64_t)gridDim.x * blockDim.x)
    dst[(idx % m) + (idx / m) * ldd] = 0.0;
}

__global__ void copy_upper_kernel(int64_t k, const double* __restrict__ src, int64_t lds,
                                  double* __restrict__ dst, int64_t ldd) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < k * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % k, j = idx / k;
    dst[i + j * ldd] = (i <= j) ? src[i + j * lds] : 0.0;
  }
}

__global__ void set_diag_block_kernel(int64_t k, const double* __restrict__ sigma, double* D,
                                      int64_t ldd) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < k * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % k, j = idx / k;
    if (i == j) D[i + j * ldd] = sigma[i];
    else if (i < j) D[i + j * ldd] = 0.0;
  }
}

__global__ void rank_kernel(int64_t len, const double* __restrict__ T, int64_t ldt, double tol_val,
                            const double* __restrict__ tol_dev, int64_t* out) {
  __shared__ long long s_first;
  __shared__ unsigned long long s_count;
  __shared__ int s_nan;
  if (threadIdx.x == 0) {
    s_first = len;
    s_count = 0;
    s_nan = 0;
  }
  __syncthreads();
  const double tol = tol_dev ? *tol_dev : tol_val;
  long long first = len;
  unsigned long long cnt = 0;
  int nan = 0;
  for (int64_t j = threadIdx.x; j < len; j += blockDim.x) {
    double d = fabs(T[j + j * ldt]);
    bool nz = d > tol;
    cnt += nz;
    nan |= isnan(d);
    if (!nz && j < first) first = j;
  }
  atomicMin(&s_first, first);
  atomicAdd(&s_count, cnt);
  if (nan) s_nan = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = s_first;
    out[1] = (int64_t)s_count;
    out[2] = s_nan;
  }
}

__global__ void resolve_tol_kernel(double tol, int64_t mn, const double* T00, double* tol_dev) {
  *tol_dev = tol >= 0.0 ? tol : (double)mn * 2.220446049250313e-16 * fabs(*T00);
}

// Nullify block gather (see the comment of nullify in solver.cu): M is
// (bsz + L) x bsz, column j <-> row j1-1-j of T, row p' < bsz <-> column
// j1-1-p' of T (upper triangle of C_11 only), row bsz+p <-> column r+p.
__global__ void rz_gather_kernel(int64_t bsz, int64_t L, const double* __restrict__ T, int64_t ldt,
                                 int64_t j0, int64_t r, double* __restrict__ M, int64_t ldm) {
  const int64_t rows = bsz + L, j1 = j0 + bsz;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < rows * bsz;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t pp = idx % rows, j = idx / rows;
    int64_t trow = j1 - 1 - j;
    double v;
    if (pp < bsz) v = (pp <= j) ? T[trow + (j1 - 1 - pp) * ldt] : 0.0;
    else v = T[trow + (r + pp - bsz) * ldt];
    M[pp + j * ldm] = v;
  }
}

__global__ void rz_scatter_kernel(int64_t bsz, const double* __restrict__ M, int64_t ldm,
                                  double* __restrict__ T, int64_t ldt, int64_t j0, int64_t r,
                                  int64_t L) {
  const int64_t j1 = j0 + bsz;
  const int64_t rows = bsz + L;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < rows * bsz;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t pp = idx % rows, j = idx / rows;
    int64_t trow = j1 - 1 - j;
    if (pp < bsz) {
      if (pp <= j) T[trow + (j1 - 1 - pp) * ldt] = M[pp + j * ldm];
    } else {
      T[trow + (r + pp - bsz) * ldt] = 0.0;
    }
  }
}

__global__ void rows_reversed_kernel(int64_t rows, int64_t cols, const double* __restrict__ src,
                                     int64_t lds, double* __restrict__ dst, int64_t ldd) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < rows * cols;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % rows, j = idx / rows;
    dst[i + j * ldd] = src[(rows - 1 - i) + j * lds];
  }
}

__global__ void cols_reversed_kernel(int64_t rows, int64_t cols, const double* __restrict__ src,
                                     int64_t lds, double* __restrict__ dst, int64_t ldd) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < rows * cols;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % rows, j = idx / rows;
    dst[i + j * ldd] = src[i + (cols - 1 - j) * lds];
  }
}

__global__ void upper_into_kernel(int64_t k, const double* __restrict__ src, int64_t lds,
                                  double* __restrict__ dst, int64_t ldd) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < k * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % k, j = idx / k;
    if (i <= j) dst[i + j * ldd] = src[i + j * lds];
  }
}

__global__ void identity_kernel(int64_t n, double* V, int64_t ldv) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % n, j = idx / n;
    V[i + j * ldv] = (i == j) ? 1.0 : 0.0;
  }
}

__global__ void upper_trapezoid_kernel(int64_t m, int64_t n, const double* __restrict__ src,
                                       int64_t lds, double* __restrict__ dst, int64_t ldd) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % m, j = idx / m;
    dst[i + j * ldd] = (i <= j) ? src[i + j * lds] : 0.0;
  }
}

// Refinement update, one CTA per column j: x_j <- x_j + d_j, and
// norms[2j] = ||d_j||^2, norms[2j+1] = ||x_j (new)||^2.  Each thread sums a
// fixed strided subset, then a fixed-shape tree: the result is the same on
// every run.
constexpr int RF_THREADS = 256;
__global__ void __launch_bounds__(RF_THREADS)
refine_update_kernel(int64_t n, const double* __restrict__ D, int64_t ldd, double* __restrict__ X,
                     int64_t ldx, double* __restrict__ norms) {
  __shared__ double s_d[RF_THREADS], s_x[RF_THREADS];
  const double* d = D + (int64_t)blockIdx.x * ldd;
  double* x = X + (int64_t)blockIdx.x * ldx;
  double sd = 0.0, sx = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += RF_THREADS) {
    double di = d[i];
    double xi = x[i] + di;
    x[i] = xi;
    sd = fma(di, di, sd);
    sx = fma(xi, xi, sx);
  }
  s_d[threadIdx.x] = sd;
  s_x[threadIdx.x] = sx;
  __syncthreads();
  for (int w = RF_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_d[threadIdx.x] += s_d[threadIdx.x + w];
      s_x[threadIdx.x] += s_x[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    norms[2 * blockIdx.x] = s_d[0];
    norms[2 * blockIdx.x + 1] = s_x[0];
  }
}

// Back substitution on one diagonal block, one CTA per right-hand side:
// y_i = b_i / R(i,i), then b_l -= R(l,i) y_i for l < i, from the bottom.
__global__ void trsm_block_kernel(int64_t k, const double* __restrict__ R, int64_t ldr, double* B,
                                  int64_t ldb) {
  extern __shared__ double x[];
  double* b = B + (int64_t)blockIdx.x * ldb;
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) x[i] = b[i];
  __syncthreads();
  for (int64_t i = k - 1; i >= 0; --i) {
    double yi = x[i] / R[i + i * ldr];
    for (int64_t l = threadIdx.x; l < i; l += blockDim.x) x[l] = fma(-R[l + i * ldr], yi, x[l]);
    __syncthreads();
    if (threadIdx.x == 0) x[i] = yi;
    __syncthreads();
  }
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) b[i] = x[i];
}

// y (M x nrhs) -= op(A) x for op(A) M x K (A[i + k lda], or A^T: A[k + i lda]),
// x K x nrhs: the off-diagonal block updates of a blocked triangular solve
// with few right-hand sides (K <= kTrsmBlock, nrhs <= kThinMaxRhs), one thread
// per row.  The general FP64 GEMM pads N to its 16-column tile, which costs
// 16 times the FP64 work for one right-hand side on this part.
__global__ void __launch_bounds__(256) gemv_thin_sub_kernel(int64_t M, int K, int nrhs,
                                                            const double* __restrict__ A,
                                                            int64_t lda, int trans,
                                                            const double* __restrict__ x,
                                                            int64_t ldx, double* y, int64_t ldy) {
  __shared__ double xs[64 * 16];
  for (int e = threadIdx.x; e < K * nrhs; e += blockDim.x) xs[e] = x[(e % K) + (int64_t)(e / K) * ldx];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = 0.0;
  for (int k = 0; k < K; ++k) {
    const double a = trans ? A[k + i * lda] : A[i + (int64_t)k * lda];
#pragma unroll
    for (int c = 0; c < 16; ++c)
      if (c < nrhs) acc[c] = fma(a, xs[k + c * K], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < 16; ++c)
    if (c < nrhs) y[i + (int64_t)c * ldy] -= acc[c];
}

// B <- R^{-T} B for one k x k diagonal block: forward substitution with the
// transpose of the upper triangular R (R^T(l, i) = R(i, l)), one CTA per
// right-hand side.
__global__ void trsm_block_trans_kernel(int64_t k, const double* __restrict__ R, int64_t ldr,
                                        double* B, int64_t ldb) {
  extern __shared__ double x[];
  double* b = B + (int64_t)blockIdx.x * ldb;
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) x[i] = b[i];
  __syncthreads();
  for (int64_t i = 0; i < k; ++i) {
    double yi = x[i] / R[i + i * ldr];
    for (int64_t l = i + 1 + threadIdx.x; l < k; l += blockDim.x) x[l] = fma(-R[i + l * ldr], yi, x[l]);
    __syncthreads();
    if (threadIdx.x == 0) x[i] = yi;
    __syncthreads();
  }
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) b[i] = x[i];
}

// out[0] = min_{j < r} |d_j|, out[1] = max_{r <= j < len} |d_j| (0 when the
// range is empty), one CTA.
__global__ void diag_gap_kernel(int64_t len, const double* __restrict__ d, int64_t r,
                                double* out) {
  __shared__ double smin[32], smax[32];
  double mn = INFINITY, mx = 0.0;
  for (int64_t j = threadIdx.x; j < len; j += blockDim.x) {
    const double v = fabs(d[j]);
    if (j < r) mn = fmin(mn, v);
    else mx = fmax(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    smin[threadIdx.x >> 5] = mn;
    smax[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mn = fmin(mn, smin[w]);
      mx = fmax(mx, smax[w]);
    }
    out[0] = r > 0 ? mn : 0.0;
    out[1] = mx;
  }
}

}  // namespace

Status diag_gap(int64_t len, const double* d, int64_t r, double* out, cudaStream_t st) {
  TraceScope ts(kTrSmall, st);
  diag_gap_kernel<<<1, 1024, 0, st>>>(len, d, r, out);
  LLS_LAUNCHED("diag_gap_kernel");
  return ok_status();
}

Status copy_check(int64_t m, int64_t n, const double* src, int64_t lds, double* dst, int64_t ldd,
                  int* flag, cudaStream_t st) {
  if (m <= 0 || n <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  copy_check_kernel<<<grid_for(m * n), EW, 0, st>>>(m, n, src, lds, dst, ldd, flag);
  LLS_LAUNCHED("copy_check_kernel");
  return ok_status();
}

Status copy_matrix(int64_t m, int64_t n, const double* src, int64_t lds, double* dst, int64_t ldd,
                   cudaStream_t st) {
  if (m <= 0 || n <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  copy_kernel<<<grid_for(m * n), EW, 0, st>>>(m, n, src, lds, dst, ldd);
  LLS_LAUNCHED("copy_kernel");
  return ok_status();
}

Status axpy_matrix(int64_t m, int64_t n, double alpha, const double* X, int64_t ldx, double* Y,
                   int64_t ldy, cudaStream_t st) {
  if (m <= 0 || n <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  axpy_kernel<<<grid_for(m * n), EW, 0, st>>>(m, n, alpha, X, ldx, Y, ldy);
  LLS_LAUNCHED("axpy_kernel");
  return ok_status();
}

Status fill_zero(int64_t m, int64_t n, double* dst, int64_t ldd, cudaStream_t st) {
  if (m <= 0 || n <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  zero_kernel<<<grid_for(m * n), EW, 0, st>>>(m, n, dst, ldd);
  LLS_LAUNCHED("zero_kernel");
  return ok_status();
}

Status copy_upper(int64_t k, const double* src, int64_t lds, double* dst, int64_t ldd,
                  cudaStream_t st) {
  if (k <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  copy_upper_kernel<<<grid_for(k * k), EW, 0, st>>>(k, src, lds, dst, ldd);
  LLS_LAUNCHED("copy_upper_kernel");
  return ok_status();
}

Status copy_upper_into(int64_t k, const double* src, int64_t lds, double* dst, int64_t ldd,
                       cudaStream_t st) {
  if (k <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  upper_into_kernel<<<grid_for(k * k), EW, 0, st>>>(k, src, lds, dst, ldd);
  LLS_LAUNCHED("upper_into_kernel");
  return ok_status();
}

Status set_identity(int64_t n, double* V, int64_t ldv, cudaStream_t st) {
  if (n <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  identity_kernel<<<grid_for(n * n), EW, 0, st>>>(n, V, ldv);
  LLS_LAUNCHED("identity_kernel");
  return ok_status();
}

Status copy_upper_trapezoid(int64_t m, int64_t n, const double* src, int64_t lds, double* dst,
                            int64_t ldd, cudaStream_t st) {
  if (m <= 0 || n <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  upper_trapezoid_kernel<<<grid_for(m * n), EW, 0, st>>>(m, n, src, lds, dst, ldd);
  LLS_LAUNCHED("upper_trapezoid_kernel");
  return ok_status();
}

Status refine_update(int64_t n, int64_t nrhs, const double* D, int64_t ldd, double* X, int64_t ldx,
                     double* norms, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return ok_status();
  if (nrhs > (1 << 20)) return make_error(LLS_ERR_ARG, "too many right-hand sides");
  TraceScope ts(kTrSmall, st);
  refine_update_kernel<<<(unsigned)nrhs, RF_THREADS, 0, st>>>(n, D, ldd, X, ldx, norms);
  LLS_LAUNCHED("refine_update_kernel");
  return ok_status();
}

Status set_diag_block(int64_t k, const double* sigma, double* D, int64_t ldd, cudaStream_t st) {
  if (k <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  set_diag_block_kernel<<<grid_for(k * k), EW, 0, st>>>(k, sigma, D, ldd);
  LLS_LAUNCHED("set_diag_block_kernel");
  return ok_status();
}

Status rank_scan(int64_t len, const double* T, int64_t ldt, double tol, int64_t* out,
                 cudaStream_t st) {
  TraceScope ts(kTrSmall, st);
  rank_kernel<<<1, 1024, 0, st>>>(len, T, ldt, tol, nullptr, out);
  LLS_LAUNCHED("rank_kernel");
  return ok_status();
}

Status resolve_tol(double tol, int64_t mn, const double* T00, double* tol_dev, cudaStream_t st) {
  TraceScope ts(kTrSmall, st);
  resolve_tol_kernel<<<1, 1, 0, st>>>(tol, mn, T00, tol_dev);
  LLS_LAUNCHED("resolve_tol_kernel");
  return ok_status();
}

Status rank_scan_dev(int64_t len, const double* T, int64_t ldt, const double* tol_dev,
                     int64_t* out, cudaStream_t st) {
  TraceScope ts(kTrSmall, st);
  rank_kernel<<<1, 1024, 0, st>>>(len, T, ldt, 0.0, tol_dev, out);
  LLS_LAUNCHED("rank_kernel");
  return ok_status();
}

Status rz_gather(int64_t bsz, int64_t L, const double* T, int64_t ldt, int64_t j0, int64_t r,
                 double* M, int64_t ldm, cudaStream_t st) {
  if (bsz <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  rz_gather_kernel<<<grid_for((bsz + L) * bsz), EW, 0, st>>>(bsz, L, T, ldt, j0, r, M, ldm);
  LLS_LAUNCHED("rz_gather_kernel");
  return ok_status();
}

Status rz_scatter(int64_t bsz, const double* M, int64_t ldm, double* T, int64_t ldt, int64_t j0,
                  int64_t r, int64_t L, cudaStream_t st) {
  if (bsz <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  rz_scatter_kernel<<<grid_for((bsz + L) * bsz), EW, 0, st>>>(bsz, M, ldm, T, ldt, j0, r, L);
  LLS_LAUNCHED("rz_scatter_kernel");
  return ok_status();
}

Status copy_rows_reversed(int64_t rows, int64_t cols, const double* src, int64_t lds, double* dst,
                          int64_t ldd, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  rows_reversed_kernel<<<grid_for(rows * cols), EW, 0, st>>>(rows, cols, src, lds, dst, ldd);
  LLS_LAUNCHED("rows_reversed_kernel");
  return ok_status();
}

Status copy_cols_reversed(int64_t rows, int64_t cols, const double* src, int64_t lds, double* dst,
                          int64_t ldd, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  cols_reversed_kernel<<<grid_for(rows * cols), EW, 0, st>>>(rows, cols, src, lds, dst, ldd);
  LLS_LAUNCHED("cols_reversed_kernel");
  return ok_status();
}

Status trsm_block(int64_t k, int64_t nrhs, const double* R, int64_t ldr, double* B, int64_t ldb,
                  cudaStream_t st) {
  if (k <= 0 || nrhs <= 0) return ok_status();
  if (nrhs > 2147483647) return make_error(LLS_ERR_ARG, "trsm: too many right-hand sides");
  TraceScope ts(kTrSmall, st);
  trsm_block_kernel<<<(unsigned)nrhs, 128, sizeof(double) * k, st>>>(k, R, ldr, B, ldb);
  LLS_LAUNCHED("trsm_block_kernel");
  return ok_status();
}

constexpr int64_t kTrsmBlock = 64;
static_assert(kTrsmBlock <= 64 && kThinMaxRhs <= 16, "gemv_thin_sub_kernel's shared x");

// y (M x nrhs) -= op(A) x, thin: see gemv_thin_sub_kernel.
Status gemv_thin_sub(int64_t M, int64_t K, int64_t nrhs, const double* A, int64_t lda, bool trans,
                     const double* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t st) {
  if (M <= 0 || K <= 0 || nrhs <= 0) return ok_status();
  TraceScope ts(kTrSmall, st, 2.0 * M * K * nrhs, 8.0 * M * K);
  gemv_thin_sub_kernel<<<(unsigned)ceil_div(M, 256), 256, 0, st>>>(M, (int)K, (int)nrhs, A, lda,
                                                                    trans ? 1 : 0, x, ldx, y, ldy);
  LLS_LAUNCHED("gemv_thin_sub_kernel");
  return ok_status();
}

size_t trsm_upper_scratch_bytes(int64_t r, int64_t nrhs) {
  size_t need = 0;
  for (int64_t j1 = r; j1 > 0; j1 -= kTrsmBlock) {
    const int64_t j0 = std::max<int64_t>(0, j1 - kTrsmBlock);
    if (j0 > 0) need = std::max(need, gemm_scratch_bytes(j0, nrhs, j1 - j0));
  }
  return need;
}

Status trsm_upper(int64_t r, int64_t nrhs, const double* R, int64_t ldr, double* B, int64_t ldb,
                  Scratch scratch, cudaStream_t st) {
  const int64_t TB = kTrsmBlock;
  int64_t j1 = r;
  while (j1 > 0) {
    int64_t j0 = std::max<int64_t>(0, j1 - TB);
    LLS_TRY(trsm_block(j1 - j0, nrhs, R + j0 + j0 * ldr, ldr, B + j0, ldb, st));
    if (j0 > 0 && nrhs <= kThinMaxRhs)
      LLS_TRY(gemv_thin_sub(j0, j1 - j0, nrhs, R + j0 * ldr, ldr, false, B + j0, ldb, B, ldb, st));
    else if (j0 > 0)
      LLS_TRY(gemm(false, false, kDense, kDense, j0, nrhs, j1 - j0, -1.0, R + j0 * ldr, ldr,
                   B + j0, ldb, 1.0, B, ldb, scratch, st));
    j1 = j0;
  }
  return ok_status();
}

size_t trsm_upper_trans_scratch_bytes(int64_t r, int64_t nrhs) {
  size_t need = 0;
  for (int64_t j0 = 0; j0 < r; j0 += kTrsmBlock) {
    const int64_t j1 = std::min(r, j0 + kTrsmBlock);
    if (j1 < r) need = std::max(need, gemm_scratch_bytes(r - j1, nrhs, j1 - j0));
  }
  return need;
}

Status trsm_upper_trans(int64_t r, int64_t nrhs, const double* R, int64_t ldr, double* B,
                        int64_t ldb, Scratch scratch, cudaStream_t st) {
  if (r <= 0 || nrhs <= 0) return ok_status();
  if (nrhs > 2147483647) return make_error(LLS_ERR_ARG, "trsm: too many right-hand sides");
  for (int64_t j0 = 0; j0 < r; j0 += kTrsmBlock) {
    const int64_t j1 = std::min(r, j0 + kTrsmBlock);
    {
      TraceScope ts(kTrSmall, st);
      trsm_block_trans_kernel<<<(unsigned)nrhs, 128, sizeof(double) * (j1 - j0), st>>>(
          j1 - j0, R + j0 + j0 * ldr, ldr, B + j0, ldb);
      LLS_LAUNCHED("trsm_block_trans_kernel");
    }
    // B(j1:r) -= R(j0:j1, j1:r)^T B(j0:j1)
    if (j1 < r && nrhs <= kThinMaxRhs)
      LLS_TRY(gemv_thin_sub(r - j1, j1 - j0, nrhs, R + j0 + j1 * ldr, ldr, true, B + j0, ldb, B + j1,
                            ldb, st));
    else if (j1 < r)
      LLS_TRY(gemm(true, false, kDense, kDense, r - j1, nrhs, j1 - j0, -1.0, R + j0 + j1 * ldr, ldr,
                   B + j0, ldb, 1.0, B + j1, ldb, scratch, st));
  }
  return ok_status();
}

}  // namespace lls

extern "C" int lls_k_trsm_upper_trans(int64_t r, int64_t nrhs, const double* R, int64_t ldr,
                                      double* B, int64_t ldb, void* stream) {
  if (r < 0 || nrhs < 0 || ldr < (r > 1 ? r : 1) || ldb < (r > 1 ? r : 1)) return LLS_ERR_ARG;
  if (r * nrhs > 0 && (!R || !B)) return LLS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  lls::Scratch s;
  s.bytes = lls::trsm_upper_trans_scratch_bytes(r, nrhs);
  if (s.bytes && cudaMallocAsync(&s.ptr, s.bytes, st) != cudaSuccess) return LLS_ERR_NOMEM;
  int code = lls::trsm_upper_trans(r, nrhs, R, ldr, B, ldb, s, st).code;
  if (s.ptr) cudaFreeAsync(s.ptr, st);
  return code;
}

extern "C" int lls_k_trsm_upper(int64_t r, int64_t nrhs, const double* R, int64_t ldr, double* B,
                                int64_t ldb, void* stream) {
  if (r < 0 || nrhs < 0 || ldr < (r > 1 ? r : 1) || ldb < (r > 1 ? r : 1)) return LLS_ERR_ARG;
  if (r * nrhs > 0 && (!R || !B)) return LLS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  lls::Scratch s;
  s.bytes = lls::trsm_upper_scratch_bytes(r, nrhs);
  if (s.bytes && cudaMallocAsync(&s.ptr, s.bytes, st) != cudaSuccess) return LLS_ERR_NOMEM;
  int code = lls::trsm_upper(r, nrhs, R, ldr, B, ldb, s, st).code;
  if (s.ptr) cudaFreeAsync(s.ptr, st);
  return code;
}

extern "C" int lls_k_rank(int64_t len, const double* T, int64_t ldt, double tol, int64_t* out,
                          void* stream) {
  if (len < 0 || ldt < 1 || !out || (len > 0 && !T)) return LLS_ERR_ARG;
  return lls::rank_scan(len, T, ldt, tol, out, (cudaStream_t)stream).code;
}
