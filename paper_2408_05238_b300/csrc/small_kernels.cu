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

// dst(rows - 1 - i, j) += alpha src(i, j).
__global__ void axpy_rows_reversed_kernel(int64_t rows, int64_t cols, double alpha,
                                          const double* __restrict__ src, int64_t lds, double* dst,
                                          int64_t ldd) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < rows * cols;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % rows, j = idx / rows;
    double* d = dst + (rows - 1 - i) + j * ldd;
    *d = fma(alpha, src[i + j * lds], *d);
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

// One k x k diagonal block (k <= 128) of an upper triangular R, one CTA per
// right-hand side: B <- R^{-1} B (back substitution) or, trans, B <- R^{-T} B
// (forward substitution with R^T(l, i) = R(i, l)).  The block is staged in
// shared memory with coalesced loads (k^2 / blockDim in flight per thread);
// thread l owns x_l in a register and 1 / R(l, l); step i publishes
// y_i = x_i / R(i, i) (as x_i times the reciprocal, computed off the serial
// chain) and every thread still to be solved subtracts R(l, i) y_i.  One
// barrier per step: each y_i has its own shared slot.
__global__ void __launch_bounds__(128) trsm_diag_kernel(int k, const double* __restrict__ R,
                                                        int64_t ldr, double* B, int64_t ldb,
                                                        int trans) {
  extern __shared__ double sm[];
  double* Rs = sm;                      // k x k, ld k + 1
  double* ys = sm + (size_t)k * (k + 1);  // k
  const int ld = k + 1, l = threadIdx.x;
  double* b = B + (int64_t)blockIdx.x * ldb;
#pragma unroll 16
  for (int e = l; e < k * k; e += blockDim.x) Rs[(e % k) + ld * (e / k)] = __ldg(R + (e % k) + (int64_t)(e / k) * ldr);
  double xl = l < k ? b[l] : 0.0;
  __syncthreads();
  const double rinv = l < k ? 1.0 / Rs[l + ld * l] : 0.0;
  if (!trans) {
    for (int i = k - 1; i >= 0; --i) {
      if (l == i) ys[i] = xl * rinv;
      __syncthreads();
      if (l < i) xl = fma(-Rs[l + ld * i], ys[i], xl);
    }
  } else {
    for (int i = 0; i < k; ++i) {
      if (l == i) ys[i] = xl * rinv;
      __syncthreads();
      if (l > i && l < k) xl = fma(-Rs[i + ld * l], ys[i], xl);
    }
  }
  if (l < k) b[l] = ys[l];
}

// Inverses of the 64 x 64 diagonal blocks of an upper triangular r x r
// matrix R, blocks aligned from the top ([64 q, 64 q + 64), the last one
// partial): one CTA of 64 threads per block, thread j forms column j of the
// inverse by back substitution on e_j (X(j, j) = 1 / R(j, j), then
// X(i, j) = -(sum_{l = i+1..j} R(i, l) X(l, j)) / R(i, i) for i < j).  Dinv
// holds the blocks one after another, 64 x 64 column-major, zero below the
// diagonal and outside a partial block.
constexpr int kInvBlk = 64;
__global__ void __launch_bounds__(kInvBlk) trsm_blockinv_kernel(int64_t r,
                                                                const double* __restrict__ R,
                                                                int64_t ldr, double* Dinv) {
  extern __shared__ double sm[];
  constexpr int LD = kInvBlk + 1;
  double* Rs = sm;                        // kb x kb
  double* Xs = sm + kInvBlk * LD;         // kb x kb
  double* rinv = sm + 2 * kInvBlk * LD;   // kb
  const int64_t j0 = (int64_t)blockIdx.x * kInvBlk;
  const int kb = (int)(r - j0 < kInvBlk ? r - j0 : kInvBlk);
  const int j = threadIdx.x;
  const double* Rb = R + j0 + j0 * ldr;
#pragma unroll 8
  for (int e = j; e < kb * kb; e += kInvBlk) Rs[(e % kb) + LD * (e / kb)] = __ldg(Rb + (e % kb) + (int64_t)(e / kb) * ldr);
  __syncthreads();
  if (j < kb) rinv[j] = 1.0 / Rs[j + LD * j];
  __syncthreads();
  if (j < kb) {
    Xs[j + LD * j] = rinv[j];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1; l <= j; ++l) s = fma(Rs[i + LD * l], Xs[l + LD * j], s);
      Xs[i + LD * j] = -s * rinv[i];
    }
  }
  __syncthreads();
  double* D = Dinv + (int64_t)blockIdx.x * kInvBlk * kInvBlk;
  for (int e = j; e < kInvBlk * kInvBlk; e += kInvBlk) {
    const int ii = e % kInvBlk, jj = e / kInvBlk;
    D[e] = (ii <= jj && jj < kb) ? Xs[ii + LD * jj] : 0.0;
  }
}

// x(0:kb) <- op(D) x(0:kb) for one 64 x 64 upper triangular block inverse D
// (op(D) = D^T when trans), one CTA per right-hand side, four threads per
// entry (every fourth l each, then two shuffle adds).
__global__ void __launch_bounds__(256) blk_inv_apply_kernel(int kb, const double* __restrict__ D,
                                                            int trans, double* B, int64_t ldb) {
  __shared__ double xs[kInvBlk];
  double* b = B + (int64_t)blockIdx.x * ldb;
  const int t = threadIdx.x, i = t >> 2, lg = t & 3;
  if (t < kb) xs[t] = b[t];
  __syncthreads();
  double s = 0.0;
  if (i < kb) {
    if (!trans) {
      for (int l = i + ((lg - i) & 3); l < kb; l += 4) s = fma(__ldg(D + i + kInvBlk * l), xs[l], s);
    } else {
      for (int l = lg; l <= i; l += 4) s = fma(__ldg(D + l + kInvBlk * i), xs[l], s);
    }
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  __syncthreads();
  if (i < kb && lg == 0) b[i] = s;
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

Status axpy_rows_reversed(int64_t rows, int64_t cols, double alpha, const double* src, int64_t lds,
                          double* dst, int64_t ldd, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return ok_status();
  TraceScope ts(kTrSmall, st);
  axpy_rows_reversed_kernel<<<grid_for(rows * cols), EW, 0, st>>>(rows, cols, alpha, src, lds, dst,
                                                                  ldd);
  LLS_LAUNCHED("axpy_rows_reversed_kernel");
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

namespace {

Status trsm_diag(int64_t k, int64_t nrhs, const double* R, int64_t ldr, double* B, int64_t ldb,
                 bool trans, cudaStream_t st) {
  if (k <= 0 || nrhs <= 0) return ok_status();
  if (k > 128) return make_error(LLS_ERR_ARG, "trsm: diagonal blocks of at most 128");
  if (nrhs > 2147483647) return make_error(LLS_ERR_ARG, "trsm: too many right-hand sides");
  const size_t smem = sizeof(double) * (size_t)(k * (k + 1) + k);
  if (smem > 48 * 1024) LLS_TRY(allow_max_dyn_smem((const void*)trsm_diag_kernel));
  TraceScope ts(kTrTrsmDiag, st);
  trsm_diag_kernel<<<(unsigned)nrhs, 128, smem, st>>>((int)k, R, ldr, B, ldb, trans ? 1 : 0);
  LLS_LAUNCHED("trsm_diag_kernel");
  return ok_status();
}

}  // namespace

Status trsm_block(int64_t k, int64_t nrhs, const double* R, int64_t ldr, double* B, int64_t ldb,
                  cudaStream_t st) {
  return trsm_diag(k, nrhs, R, ldr, B, ldb, false, st);
}

constexpr int64_t kTrsmBlock = 64;

// The off-diagonal updates use thin_gemv for nrhs <= kThinMaxRhs (K = 64: no
// split, no scratch) and the FP64 GEMM otherwise.
size_t trsm_upper_scratch_bytes(int64_t r, int64_t nrhs) {
  size_t need = 0;
  if (nrhs <= kThinMaxRhs) return 0;
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
    LLS_TRY(trsm_diag(j1 - j0, nrhs, R + j0 + j0 * ldr, ldr, B + j0, ldb, false, st));
    // B(0:j0) -= R(0:j0, j0:j1) B(j0:j1)
    if (j0 > 0 && nrhs <= kThinMaxRhs)
      LLS_TRY(thin_gemv(false, false, j0, j1 - j0, nrhs, -1.0, R + j0 * ldr, ldr, B + j0, ldb, 1.0, B,
                        ldb, Scratch{}, st));
    else if (j0 > 0)
      LLS_TRY(gemm(false, false, kDense, kDense, j0, nrhs, j1 - j0, -1.0, R + j0 * ldr, ldr,
                   B + j0, ldb, 1.0, B, ldb, scratch, st));
    j1 = j0;
  }
  return ok_status();
}

size_t trsm_upper_trans_scratch_bytes(int64_t r, int64_t nrhs) {
  size_t need = 0;
  if (nrhs <= kThinMaxRhs) return 0;
  for (int64_t j0 = 0; j0 < r; j0 += kTrsmBlock) {
    const int64_t j1 = std::min(r, j0 + kTrsmBlock);
    if (j1 < r) need = std::max(need, gemm_scratch_bytes(r - j1, nrhs, j1 - j0));
  }
  return need;
}

Status trsm_upper_trans(int64_t r, int64_t nrhs, const double* R, int64_t ldr, double* B,
                        int64_t ldb, Scratch scratch, cudaStream_t st) {
  if (r <= 0 || nrhs <= 0) return ok_status();
  for (int64_t j0 = 0; j0 < r; j0 += kTrsmBlock) {
    const int64_t j1 = std::min(r, j0 + kTrsmBlock);
    LLS_TRY(trsm_diag(j1 - j0, nrhs, R + j0 + j0 * ldr, ldr, B + j0, ldb, true, st));
    // B(j1:r) -= R(j0:j1, j1:r)^T B(j0:j1)
    if (j1 < r && nrhs <= kThinMaxRhs)
      LLS_TRY(thin_gemv(true, false, r - j1, j1 - j0, nrhs, -1.0, R + j0 + j1 * ldr, ldr, B + j0, ldb,
                        1.0, B + j1, ldb, Scratch{}, st));
    else if (j1 < r)
      LLS_TRY(gemm(true, false, kDense, kDense, r - j1, nrhs, j1 - j0, -1.0, R + j0 + j1 * ldr, ldr,
                   B + j0, ldb, 1.0, B + j1, ldb, scratch, st));
  }
  return ok_status();
}

}  // namespace lls

namespace lls {

size_t trsm_inverse_bytes(int64_t r) {
  return sizeof(double) * (size_t)ceil_div(std::max<int64_t>(r, 0), kInvBlk) * kInvBlk * kInvBlk;
}

Status trsm_block_inverses(int64_t r, const double* R, int64_t ldr, double* Dinv, cudaStream_t st) {
  if (r <= 0) return ok_status();
  const int64_t nblk = ceil_div(r, kInvBlk);
  if (nblk > INT32_MAX) return make_error(LLS_ERR_ARG, "trsm_block_inverses: r too large");
  const size_t smem = sizeof(double) * (2 * kInvBlk * (kInvBlk + 1) + kInvBlk);
  LLS_TRY(allow_max_dyn_smem((const void*)trsm_blockinv_kernel));
  TraceScope ts(kTrTrsmDiag, st);
  trsm_blockinv_kernel<<<(unsigned)nblk, kInvBlk, smem, st>>>(r, R, ldr, Dinv);
  LLS_LAUNCHED("trsm_blockinv_kernel");
  return ok_status();
}

Status trsm_upper_inv(int64_t r, int64_t nrhs, const double* R, int64_t ldr, const double* Dinv,
                      double* B, int64_t ldb, bool trans, cudaStream_t st) {
  if (r <= 0 || nrhs <= 0) return ok_status();
  if (nrhs > kThinMaxRhs) return make_error(LLS_ERR_ARG, "trsm_upper_inv: nrhs <= 16");
  const int64_t nblk = ceil_div(r, kInvBlk);
  auto apply = [&](int64_t q, int64_t kb, bool tr) -> Status {
    TraceScope ts(kTrTrsmDiag, st);
    blk_inv_apply_kernel<<<(unsigned)nrhs, 256, 0, st>>>((int)kb, Dinv + q * kInvBlk * kInvBlk,
                                                         tr ? 1 : 0, B + q * kInvBlk, ldb);
    LLS_LAUNCHED("blk_inv_apply_kernel");
    return ok_status();
  };
  if (!trans) {  // R y = c, bottom block first
    for (int64_t q = nblk - 1; q >= 0; --q) {
      const int64_t j0 = q * kInvBlk, kb = std::min<int64_t>(kInvBlk, r - j0);
      LLS_TRY(apply(q, kb, false));
      if (j0 > 0)  // c(0:j0) -= R(0:j0, j0:j0+kb) y_q
        LLS_TRY(thin_gemv(false, false, j0, kb, nrhs, -1.0, R + j0 * ldr, ldr, B + j0, ldb, 1.0, B,
                          ldb, Scratch{}, st));
    }
  } else {  // R^T y = c, top block first
    for (int64_t q = 0; q < nblk; ++q) {
      const int64_t j0 = q * kInvBlk, j1 = std::min(r, j0 + kInvBlk);
      LLS_TRY(apply(q, j1 - j0, true));
      if (j1 < r)  // c(j1:r) -= R(j0:j1, j1:r)^T y_q
        LLS_TRY(thin_gemv(true, false, r - j1, j1 - j0, nrhs, -1.0, R + j0 + j1 * ldr, ldr, B + j0,
                          ldb, 1.0, B + j1, ldb, Scratch{}, st));
    }
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
