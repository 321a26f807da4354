// Host stand-ins for the library's launchers (test infrastructure, never
// loaded by the package).  Linked with the library's host-side orchestration
// (solver.cu, ooc_solve.cu, ooc_plan.cu) and stand_in_runtime.cpp, they let
// the CPU tests run the solver's and the out-of-core executor's sequence of
// launches, pointers, leading dimensions and copies against the oracle.
// Each stand-in is a plain loop version of what its launcher computes:
// column-major GEMM with the unit-lower operand mode, Householder QR in the
// LAPACK sign convention, the compact-WY T factor, one-sided Jacobi SVD,
// copies, the Nullify gather/scatter index maps, back substitution.  The
// sketch is a fixed deterministic hash matrix (the tests give the oracle the
// same one).  Fresh allocations are filled with NaN so that a read of memory
// nothing wrote shows up in the result.
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "batched_factor.h"
#include "solver.h"
#include "lls.h"

namespace lls {

size_t gemm_scratch_bytes(int64_t, int64_t, int64_t) { return 0; }
size_t panel_qr_scratch_bytes(int64_t, int64_t) { return 0; }

static double rd(const double* A, int64_t lda, OperandMode md, int64_t r, int64_t c) {
  if (md == kUnitLower) return r > c ? A[r + c * lda] : (r == c ? 1.0 : 0.0);
  return A[r + c * lda];
}
Status gemm(bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t m, int64_t n, int64_t k,
            double alpha, const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
            double* C, int64_t ldc, Scratch, cudaStream_t) {
  std::vector<double> out((size_t)(m * n), 0.0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      double s = 0.0;
      for (int64_t p = 0; p < k; ++p) {
        double a = ta ? rd(A, lda, ma, p, i) : rd(A, lda, ma, i, p);
        double b = tb ? rd(B, ldb, mb, j, p) : rd(B, ldb, mb, p, j);
        s += a * b;
      }
      out[i + j * m] = alpha * s + (beta == 0.0 ? 0.0 : beta * C[i + j * ldc]);
    }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) C[i + j * ldc] = out[i + j * m];
  return ok_status();
}
Status panel_qr(int64_t m, int64_t n, double* A, int64_t lda, double* tau, Scratch, int*,
                cudaStream_t, bool) {
  const int64_t k = std::min(m, n);
  for (int64_t j = 0; j < k; ++j) {
    double alpha = A[j + j * lda], sig = 0.0;
    for (int64_t i = j + 1; i < m; ++i) sig += A[i + j * lda] * A[i + j * lda];
    sig = std::sqrt(sig);
    if (sig == 0.0) { tau[j] = 0.0; continue; }
    double beta = -std::copysign(std::hypot(alpha, sig), alpha);
    double t = (beta - alpha) / beta, sc = 1.0 / (alpha - beta);
    for (int64_t i = j + 1; i < m; ++i) A[i + j * lda] *= sc;
    A[j + j * lda] = beta;
    tau[j] = t;
    for (int64_t c = j + 1; c < n; ++c) {
      double d = A[j + c * lda];
      for (int64_t i = j + 1; i < m; ++i) d += A[i + j * lda] * A[i + c * lda];
      d *= t;
      A[j + c * lda] -= d;
      for (int64_t i = j + 1; i < m; ++i) A[i + c * lda] -= d * A[i + j * lda];
    }
  }
  return ok_status();
}
Status wy_tfactor(int64_t k, const double* S, int64_t lds, const double* tau, double* T,
                  int64_t ldt, cudaStream_t) {
  for (int64_t j = 0; j < k; ++j)
    for (int64_t i = 0; i < k; ++i) T[i + j * ldt] = 0.0;
  for (int64_t j = 0; j < k; ++j) {
    T[j + j * ldt] = tau[j];
    for (int64_t i = 0; i < j; ++i) {
      double s = 0.0;
      for (int64_t l = i; l < j; ++l) s += T[i + l * ldt] * S[l + j * lds];
      T[i + j * ldt] = -tau[j] * s;
    }
  }
  return ok_status();
}
// one-sided Jacobi SVD of a b x b block, sigma descending
static void svd_block(int64_t b, const double* R, int64_t ldr, double* s, double* U, int64_t ldu,
                      double* V, int64_t ldv) {
  std::vector<double> A((size_t)(b * b)), W((size_t)(b * b), 0.0);
  for (int64_t j = 0; j < b; ++j)
    for (int64_t i = 0; i < b; ++i) A[i + j * b] = R[i + j * ldr];
  for (int64_t i = 0; i < b; ++i) W[i + i * b] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rot = false;
    for (int64_t p = 0; p < b; ++p)
      for (int64_t q = p + 1; q < b; ++q) {
        double a = 0, bb = 0, c = 0;
        for (int64_t i = 0; i < b; ++i) {
          a += A[i + p * b] * A[i + p * b];
          bb += A[i + q * b] * A[i + q * b];
          c += A[i + p * b] * A[i + q * b];
        }
        if (std::fabs(c) <= 1e-16 * std::sqrt(a * bb)) continue;
        rot = true;
        double z = (bb - a) / (2 * c), t = std::copysign(1.0, z) / (std::fabs(z) + std::hypot(1.0, z));
        double cs = 1 / std::hypot(1.0, t), sn = cs * t;
        for (int64_t i = 0; i < b; ++i) {
          double x = A[i + p * b], y = A[i + q * b];
          A[i + p * b] = cs * x - sn * y;
          A[i + q * b] = sn * x + cs * y;
          x = W[i + p * b];
          y = W[i + q * b];
          W[i + p * b] = cs * x - sn * y;
          W[i + q * b] = sn * x + cs * y;
        }
      }
    if (!rot) break;
  }
  std::vector<int64_t> ord((size_t)b);
  std::vector<double> nrm((size_t)b);
  for (int64_t j = 0; j < b; ++j) {
    double s2 = 0;
    for (int64_t i = 0; i < b; ++i) s2 += A[i + j * b] * A[i + j * b];
    nrm[(size_t)j] = std::sqrt(s2);
    ord[(size_t)j] = j;
  }
  std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return nrm[x] > nrm[y]; });
  for (int64_t jj = 0; jj < b; ++jj) {
    int64_t j = ord[(size_t)jj];
    s[jj] = nrm[(size_t)j];
    for (int64_t i = 0; i < b; ++i) {
      V[i + jj * ldv] = W[i + j * b];
      U[i + jj * ldu] = nrm[(size_t)j] > 0 ? A[i + j * b] / nrm[(size_t)j] : (i == jj ? 1.0 : 0.0);
    }
  }
}
Status jacobi_svd_batched(int count, int b, int b_last, const double* R, int64_t ldr,
                          int64_t strideR, double* sigma, int64_t strideS, double* U, int64_t ldu,
                          int64_t strideU, double* V, int64_t ldv, int64_t strideV, int*,
                          cudaStream_t) {
  for (int i = 0; i < count; ++i)
    svd_block(i == count - 1 ? b_last : b, R + i * strideR, ldr, sigma + i * strideS,
              U + i * strideU, ldu, V + i * strideV, ldv);
  return ok_status();
}
Status launch_sketch(uint64_t seed, int64_t step, int64_t rows, int64_t cols, double* G,
                     int64_t ldg, cudaStream_t) {
  for (int64_t j = 0; j < cols; ++j)
    for (int64_t i = 0; i < rows; ++i) {
      double v = std::sin(12.9898 * i + 78.233 * j + 37.719 * step + (double)(seed % 1000)) * 43758.5453;
      G[i + j * ldg] = v - std::floor(v) - 0.5;
    }
  return ok_status();
}
Status copy_matrix(int64_t m, int64_t n, const double* s, int64_t lds, double* d, int64_t ldd,
                   cudaStream_t) {
  std::vector<double> t((size_t)(m * n));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) t[i + j * m] = s[i + j * lds];
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) d[i + j * ldd] = t[i + j * m];
  return ok_status();
}
Status copy_upper(int64_t k, const double* s, int64_t lds, double* d, int64_t ldd, cudaStream_t) {
  for (int64_t j = 0; j < k; ++j)
    for (int64_t i = 0; i < k; ++i) d[i + j * ldd] = i <= j ? s[i + j * lds] : 0.0;
  return ok_status();
}
Status copy_upper_into(int64_t k, const double* s, int64_t lds, double* d, int64_t ldd,
                       cudaStream_t) {
  for (int64_t j = 0; j < k; ++j)
    for (int64_t i = 0; i <= j; ++i) d[i + j * ldd] = s[i + j * lds];
  return ok_status();
}
Status set_diag_block(int64_t k, const double* sigma, double* D, int64_t ldd, cudaStream_t) {
  for (int64_t j = 0; j < k; ++j)
    for (int64_t i = 0; i <= j; ++i) D[i + j * ldd] = i == j ? sigma[i] : 0.0;
  return ok_status();
}
Status fill_zero(int64_t m, int64_t n, double* d, int64_t ldd, cudaStream_t) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) d[i + j * ldd] = 0.0;
  return ok_status();
}
Status axpy_matrix(int64_t m, int64_t n, double a, const double* X, int64_t ldx, double* Y,
                   int64_t ldy, cudaStream_t) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) Y[i + j * ldy] += a * X[i + j * ldx];
  return ok_status();
}
Status copy_cols_reversed(int64_t rows, int64_t cols, const double* s, int64_t lds, double* d,
                          int64_t ldd, cudaStream_t) {
  for (int64_t j = 0; j < cols; ++j)
    for (int64_t i = 0; i < rows; ++i) d[i + j * ldd] = s[i + (cols - 1 - j) * lds];
  return ok_status();
}
Status copy_rows_reversed(int64_t rows, int64_t cols, const double* s, int64_t lds, double* d,
                          int64_t ldd, cudaStream_t) {
  for (int64_t j = 0; j < cols; ++j)
    for (int64_t i = 0; i < rows; ++i) d[i + j * ldd] = s[(rows - 1 - i) + j * lds];
  return ok_status();
}
Status rz_gather(int64_t bsz, int64_t L, const double* T, int64_t ldt, int64_t j0, int64_t r,
                 double* M, int64_t ldm, cudaStream_t) {
  const int64_t rows = bsz + L, j1 = j0 + bsz;
  for (int64_t j = 0; j < bsz; ++j)
    for (int64_t pp = 0; pp < rows; ++pp) {
      int64_t trow = j1 - 1 - j;
      double v;
      if (pp < bsz) v = (pp <= j) ? T[trow + (j1 - 1 - pp) * ldt] : 0.0;
      else v = T[trow + (r + pp - bsz) * ldt];
      M[pp + j * ldm] = v;
    }
  return ok_status();
}
Status rz_scatter(int64_t bsz, const double* M, int64_t ldm, double* T, int64_t ldt, int64_t j0,
                  int64_t r, int64_t L, cudaStream_t) {
  const int64_t j1 = j0 + bsz, rows = bsz + L;
  for (int64_t j = 0; j < bsz; ++j)
    for (int64_t pp = 0; pp < rows; ++pp) {
      int64_t trow = j1 - 1 - j;
      if (pp < bsz) {
        if (pp <= j) T[trow + (j1 - 1 - pp) * ldt] = M[pp + j * ldm];
      } else {
        T[trow + (r + pp - bsz) * ldt] = 0.0;
      }
    }
  return ok_status();
}
Status trsm_block(int64_t k, int64_t nrhs, const double* R, int64_t ldr, double* B, int64_t ldb,
                  cudaStream_t) {
  for (int64_t c = 0; c < nrhs; ++c)
    for (int64_t i = k - 1; i >= 0; --i) {
      double y = B[i + c * ldb] / R[i + i * ldr];
      B[i + c * ldb] = y;
      for (int64_t l = 0; l < i; ++l) B[l + c * ldb] -= R[l + i * ldr] * y;
    }
  return ok_status();
}
}  // namespace lls

namespace lls {
Status copy_check(int64_t m, int64_t n, const double* src, int64_t lds, double* dst, int64_t ldd,
                  int* flag, cudaStream_t) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      double v = src[i + j * lds];
      if (!std::isfinite(v)) *flag = 1;
      if (dst) dst[i + j * ldd] = v;
    }
  return ok_status();
}
size_t oz_gemm_workspace_bytes(int64_t, int64_t, int64_t) { return 0; }
Status oz_gemm(bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t m, int64_t n, int64_t k,
               double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
               double beta, double* C, int64_t ldc, bool, Scratch s, int*, cudaStream_t st) {
  return gemm(ta, tb, ma, mb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s, st);
}
// The mixed-precision sample, in FP64 here (the BF16 products are a kernel
// matter): Y = (A^T A)^q A^T G with the harness's sketch, so the mixed path's
// orchestration around it runs with exact products.
Status sample_bf16(Handle&, const double* A, int64_t lda, int64_t mp, int64_t np, int64_t b, int q,
                   uint64_t seed, int64_t step, double* Y, int64_t ldy) {
  std::vector<double> G((size_t)std::max<int64_t>(mp * b, 1)), W((size_t)std::max<int64_t>(mp * b, 1));
  LLS_TRY(launch_sketch(seed, step, mp, b, G.data(), std::max<int64_t>(mp, 1), nullptr));
  const int64_t ldg = std::max<int64_t>(mp, 1);
  LLS_TRY(gemm(true, false, kDense, kDense, np, b, mp, 1.0, A, lda, G.data(), ldg, 0.0, Y, ldy,
               Scratch{}, nullptr));
  for (int it = 0; it < q; ++it) {
    LLS_TRY(gemm(false, false, kDense, kDense, mp, b, np, 1.0, A, lda, Y, ldy, 0.0, W.data(), ldg,
                 Scratch{}, nullptr));
    LLS_TRY(gemm(true, false, kDense, kDense, np, b, mp, 1.0, A, lda, W.data(), ldg, 0.0, Y, ldy,
                 Scratch{}, nullptr));
  }
  return ok_status();
}
Status resolve_tol(double tol, int64_t mn, const double* T00, double* tol_dev, cudaStream_t) {
  *tol_dev = tol >= 0.0 ? tol : (double)mn * 2.220446049250313e-16 * std::fabs(*T00);
  return ok_status();
}
Status rank_scan_dev(int64_t len, const double* T, int64_t ldt, const double* tol_dev,
                     int64_t* out, cudaStream_t) {
  int64_t first = len, cnt = 0, nan = 0;
  for (int64_t j = 0; j < len; ++j) {
    double d = std::fabs(T[j + j * ldt]);
    bool nz = d > *tol_dev;
    cnt += nz;
    nan |= std::isnan(d);
    if (!nz && j < first) first = j;
  }
  out[0] = first;
  out[1] = cnt;
  out[2] = nan;
  return ok_status();
}
Status refine_update(int64_t n, int64_t nrhs, const double* D, int64_t ldd, double* X, int64_t ldx,
                     double* norms, cudaStream_t) {
  for (int64_t c = 0; c < nrhs; ++c) {
    double sd = 0, sx = 0;
    for (int64_t i = 0; i < n; ++i) {
      X[i + c * ldx] += D[i + c * ldd];
      sd += D[i + c * ldd] * D[i + c * ldd];
      sx += X[i + c * ldx] * X[i + c * ldx];
    }
    norms[2 * c] = sd;
    norms[2 * c + 1] = sx;
  }
  return ok_status();
}
Status copy_upper_trapezoid(int64_t m, int64_t n, const double* s, int64_t lds, double* d,
                            int64_t ldd, cudaStream_t) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) d[i + j * ldd] = i <= j ? s[i + j * lds] : 0.0;
  return ok_status();
}
Status set_identity(int64_t n, double* V, int64_t ldv, cudaStream_t) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) V[i + j * ldv] = i == j ? 1.0 : 0.0;
  return ok_status();
}
size_t trsm_upper_scratch_bytes(int64_t, int64_t) { return 0; }
Status trsm_upper(int64_t r, int64_t nrhs, const double* R, int64_t ldr, double* B, int64_t ldb,
                  Scratch, cudaStream_t st) {
  return trsm_block(r, nrhs, R, ldr, B, ldb, st);
}
Status diag_gap(int64_t len, const double* d, int64_t r, double* out, cudaStream_t) {
  double mn = INFINITY, mx = 0.0;
  for (int64_t j = 0; j < len; ++j) {
    if (j < r) mn = std::min(mn, std::fabs(d[j]));
    else mx = std::max(mx, std::fabs(d[j]));
  }
  out[0] = r > 0 ? mn : 0.0;
  out[1] = mx;
  return ok_status();
}
size_t thin_scratch_bytes(int64_t, int64_t, int64_t) { return 0; }
size_t thin_gemv_scratch_bytes(bool, int64_t, int64_t, int64_t) { return 0; }
// y = beta y + alpha op(A) x, plainly (unit_lower: 0 above, 1 on the diagonal).
Status thin_gemv(bool trans, bool unit_lower, int64_t M, int64_t K, int64_t nrhs, double alpha,
                 const double* A, int64_t lda, const double* x, int64_t ldx, double beta, double* y,
                 int64_t ldy, Scratch, cudaStream_t) {
  auto a = [&](int64_t i, int64_t k) {  // stored A(i, k)
    if (unit_lower && i <= k) return i == k ? 1.0 : 0.0;
    return A[i + k * lda];
  };
  for (int64_t c = 0; c < nrhs; ++c)
    for (int64_t i = 0; i < M; ++i) {
      double s = 0.0;
      for (int64_t k = 0; k < K; ++k) s += (trans ? a(k, i) : a(i, k)) * x[k + c * ldx];
      double& out = y[i + c * ldy];
      out = beta == 0.0 ? alpha * s : beta * out + alpha * s;
    }
  return ok_status();
}
// x <- (I - W op(T) W^T) x with unit lower W, plainly.
Status apply_reflectors_thin(int64_t M, int64_t b, int64_t nrhs, const double* W, int64_t ldw,
                             const double* T, int64_t ldt, bool transT, double* x, int64_t ldx,
                             Scratch, cudaStream_t) {
  auto w = [&](int64_t r, int64_t j) { return r < j ? 0.0 : (r == j ? 1.0 : W[r + j * ldw]); };
  for (int64_t c = 0; c < nrhs; ++c) {
    double* xc = x + c * ldx;
    std::vector<double> p((size_t)b, 0.0), p2((size_t)b, 0.0);
    for (int64_t j = 0; j < b; ++j)
      for (int64_t r = 0; r < M; ++r) p[j] += w(r, j) * xc[r];
    for (int64_t i = 0; i < b; ++i)
      for (int64_t l = 0; l < b; ++l) {
        const double t = transT ? (l <= i ? T[l + i * ldt] : 0.0) : (l >= i ? T[i + l * ldt] : 0.0);
        p2[i] += t * p[l];
      }
    for (int64_t r = 0; r < M; ++r)
      for (int64_t j = 0; j < b; ++j) xc[r] -= w(r, j) * p2[j];
  }
  return ok_status();
}
size_t replay_persistent_scratch_bytes(int64_t, int64_t) { return 0; }
bool replay_persistent_fits(int64_t nb, int64_t nrhs, const double* W, int64_t ldw, int64_t,
                            int64_t) {
  return nrhs >= 1 && nrhs <= 4 && nb >= 1 && nb <= 128 && ldw % 2 == 0 &&
         reinterpret_cast<uintptr_t>(W) % 16 == 0;
}
// The replay's steps one after another, each as the plain thin step above.
Status replay_persistent(bool forward, int64_t M, int64_t nb, int64_t nsteps, int64_t kmax,
                         const double* W, int64_t ldw, const double* T, double* x, int64_t ldx,
                         int64_t nrhs, Scratch, int*, cudaStream_t st) {
  for (int64_t s = 0; s < nsteps; ++s) {
    const int64_t i = forward ? s : nsteps - 1 - s, k = i * nb, b = std::min(nb, kmax - k);
    LLS_TRY(apply_reflectors_thin(M - k, b, nrhs, W + k + k * ldw, ldw, T + i * nb * nb, nb, forward,
                                  x + k, ldx, {}, st));
  }
  return ok_status();
}
Status axpy_rows_reversed(int64_t rows, int64_t cols, double alpha, const double* src, int64_t lds,
                          double* dst, int64_t ldd, cudaStream_t) {
  for (int64_t j = 0; j < cols; ++j)
    for (int64_t i = 0; i < rows; ++i) dst[(rows - 1 - i) + j * ldd] += alpha * src[i + j * lds];
  return ok_status();
}
Status small_blocks_batched(int64_t nblk, int64_t nb, int64_t kmax, int64_t nrhs, const double* S,
                            bool transS, const double* x, int64_t ldx, double* xo, int64_t ldxo,
                            cudaStream_t) {
  for (int64_t i = 0; i < nblk; ++i) {
    const int64_t k = i * nb, b = std::min(nb, kmax - k);
    const double* Si = S + i * nb * nb;
    for (int64_t c = 0; c < nrhs; ++c)
      for (int64_t r = 0; r < b; ++r) {
        double s = 0.0;
        for (int64_t l = 0; l < b; ++l)
          s += (transS ? Si[l + r * nb] : Si[r + l * nb]) * x[k + l + c * ldx];
        xo[k + r + c * ldxo] = s;
      }
  }
  return ok_status();
}
Status small_block_mul(int64_t b, int64_t nrhs, const double* S, int64_t lds, bool transS,
                       double* x, int64_t ldx, cudaStream_t) {
  for (int64_t c = 0; c < nrhs; ++c) {
    double* xc = x + c * ldx;
    std::vector<double> y((size_t)b, 0.0);
    for (int64_t i = 0; i < b; ++i)
      for (int64_t l = 0; l < b; ++l) y[i] += (transS ? S[l + i * lds] : S[i + l * lds]) * xc[l];
    for (int64_t i = 0; i < b; ++i) xc[i] = y[i];
  }
  return ok_status();
}
// The block-inverse solves: the inverses are not formed here, the solves
// substitute (the inverses are a kernel matter).
size_t trsm_inverse_bytes(int64_t r) { return sizeof(double) * (size_t)std::max<int64_t>(r, 1); }
Status trsm_block_inverses(int64_t, const double*, int64_t, double*, cudaStream_t) {
  return ok_status();
}
Status trsm_upper_inv(int64_t r, int64_t nrhs, const double* R, int64_t ldr, const double*,
                      double* B, int64_t ldb, bool trans, cudaStream_t st) {
  if (trans) return trsm_upper_trans(r, nrhs, R, ldr, B, ldb, Scratch{}, st);
  return trsm_upper(r, nrhs, R, ldr, B, ldb, Scratch{}, st);
}
Status trsm_upper_inv_persistent(int64_t r, int64_t nrhs, const double* R, int64_t ldr,
                                 const double* Dinv, double* B, int64_t ldb, bool trans, Scratch,
                                 int*, cudaStream_t st) {
  return trsm_upper_inv(r, nrhs, R, ldr, Dinv, B, ldb, trans, st);
}
size_t trsm_upper_trans_scratch_bytes(int64_t, int64_t) { return 0; }
// R^T Y = B by forward substitution, one column at a time.
Status trsm_upper_trans(int64_t r, int64_t nrhs, const double* R, int64_t ldr, double* B,
                        int64_t ldb, Scratch, cudaStream_t) {
  for (int64_t j = 0; j < nrhs; ++j) {
    double* b = B + j * ldb;
    for (int64_t i = 0; i < r; ++i) {
      double s = b[i];
      for (int64_t l = 0; l < i; ++l) s -= R[l + i * ldr] * b[l];
      b[i] = s / R[i + i * ldr];
    }
  }
  return ok_status();
}
// The split-TF32 products, exact here (their rounding is a kernel matter):
// the TF32 modes' orchestration -- the minimum-norm refinement and the
// transposed solve operator -- runs with exact products.
size_t tf32_gemm_workspace_bytes(int64_t, int64_t, int64_t, int) { return 0; }
Status tf32_gemm(bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t m, int64_t n, int64_t k,
                 double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                 double beta, double* C, int64_t ldc, int, Scratch s, int*, cudaStream_t st) {
  return gemm(ta, tb, ma, mb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s, st);
}
// The persistent batched factorization, emulated: every problem's phases in
// the kernel's order with the plain-loop launchers above, writing the
// problem's buffers as the kernel does (so the driver's arena layout, the
// factor views and the finishing path run here).
bool batched_factor_available() { return true; }
int pb_num_phases(int m, int n, int nb, int q) {
  return 1 + (int)ceil_div(std::min(m, n), nb) * (8 + 2 * q) + 3;
}
size_t pb_workspace_doubles(int64_t m, int64_t n, int nb) {
  return 4 * (size_t)m * nb + 2 * (size_t)nb * n + (size_t)nb * nb;
}
Status batched_factor_launch(const PBArgs& a, cudaStream_t st) {
  for (int j = 0; j < a.count; ++j) {
    const PBProblem& p = a.probs[j];
    const int64_t m = p.m, n = p.n, nb = p.nb, ldt = p.ldt, ldw = p.ldw;
    const size_t blk = (size_t)nb * nb;
    LLS_TRY(copy_check(m, n, p.A, p.lda, p.T, ldt, p.flags, st));
    for (int i = 0; i < p.steps; ++i) {
      const int64_t k = i * nb, mp = m - k, np = n - k, b = std::min(nb, std::min(mp, np));
      double* ABR = p.T + k + k * ldt;
      double* Y = p.WV + k + k * ldw;
      LLS_TRY(launch_sketch(p.seed, i, mp, b, p.G, m, st));
      LLS_TRY(gemm(true, false, kDense, kDense, np, b, mp, 1.0, ABR, ldt, p.G, m, 0.0, Y, ldw, {}, st));
      for (int it = 0; it < p.q; ++it) {
        LLS_TRY(gemm(false, false, kDense, kDense, mp, b, np, 1.0, ABR, ldt, Y, ldw, 0.0, p.W, m, {}, st));
        LLS_TRY(gemm(true, false, kDense, kDense, np, b, mp, 1.0, ABR, ldt, p.W, m, 0.0, Y, ldw, {}, st));
      }
      LLS_TRY(panel_qr(np, b, Y, ldw, p.tauV + i * nb, {}, p.flags, st));
      LLS_TRY(gemm(true, false, kUnitLower, kUnitLower, b, b, np, 1.0, Y, ldw, Y, ldw, 0.0, p.S, nb, {}, st));
      LLS_TRY(wy_tfactor(b, p.S, nb, p.tauV + i * nb, p.TV + i * blk, nb, st));
      double* Tk = p.T + k * ldt;
      LLS_TRY(gemm(false, false, kDense, kUnitLower, m, b, np, 1.0, Tk, ldt, Y, ldw, 0.0, p.P, m, {}, st));
      LLS_TRY(gemm(false, false, kDense, kDense, m, b, b, 1.0, p.P, m, p.TV + i * blk, nb, 0.0, p.P2, m, {}, st));
      LLS_TRY(gemm(false, true, kDense, kUnitLower, m, np, b, -1.0, p.P2, m, Y, ldw, 1.0, Tk, ldt, {}, st));
      LLS_TRY(panel_qr(mp, b, ABR, ldt, p.tauU + i * nb, {}, p.flags, st));
      LLS_TRY(copy_upper(b, ABR, ldt, p.Rblk + i * blk, nb, st));
      LLS_TRY(gemm(true, false, kUnitLower, kUnitLower, b, b, mp, 1.0, ABR, ldt, ABR, ldt, 0.0, p.S, nb, {}, st));
      LLS_TRY(wy_tfactor(b, p.S, nb, p.tauU + i * nb, p.TU + i * blk, nb, st));
      if (np > b) {
        double* A12 = ABR + b * ldt;
        LLS_TRY(gemm(true, false, kUnitLower, kDense, b, np - b, mp, 1.0, ABR, ldt, A12, ldt, 0.0, p.Q, nb, {}, st));
        LLS_TRY(gemm(true, false, kDense, kDense, b, np - b, b, 1.0, p.TU + i * blk, nb, p.Q, nb, 0.0, p.Q2, nb, {}, st));
        LLS_TRY(gemm(false, false, kUnitLower, kDense, mp, np - b, b, -1.0, ABR, ldt, p.Q2, nb, 1.0, A12, ldt, {}, st));
      }
    }
    const int64_t bl = std::min(nb, std::min(m, n) - (int64_t)(p.steps - 1) * nb);
    LLS_TRY(jacobi_svd_batched(p.steps, (int)nb, (int)bl, p.Rblk, nb, blk, p.sigma, nb, p.US, nb, blk,
                               p.VS, nb, blk, p.flags + 1, st));
    for (int i = 0; i < p.steps; ++i) {
      const int64_t k = i * nb, b = std::min(nb, std::min(m - k, n - k));
      LLS_TRY(set_diag_block(b, p.sigma + i * nb, p.T + k + k * ldt, ldt, st));
      if (k > 0) {
        LLS_TRY(gemm(false, false, kDense, kDense, k, b, b, 1.0, p.T + k * ldt, ldt, p.VS + i * blk, nb, 0.0, p.P, k, {}, st));
        LLS_TRY(copy_matrix(k, b, p.P, k, p.T + k * ldt, ldt, st));
      }
    }
    for (int i = 0; i < p.steps; ++i) {
      const int64_t k = i * nb, b = std::min(nb, std::min(m - k, n - k)), np = n - k;
      if (np > b) {
        double* A12 = p.T + k + (k + b) * ldt;
        LLS_TRY(gemm(true, false, kDense, kDense, b, np - b, b, 1.0, p.US + i * blk, nb, A12, ldt, 0.0, p.Q, nb, {}, st));
        LLS_TRY(copy_matrix(b, np - b, p.Q, nb, A12, ldt, st));
      }
    }
  }
  return ok_status();
}
}  // namespace lls

