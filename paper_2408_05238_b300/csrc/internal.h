// Launchers shared between the library's translation units.  All matrices
// are column-major FP64; all pointers are device pointers; every launcher
// only enqueues work on `st`.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"

namespace lls {

// Operand layout flag for the GEMM loader: the stored matrix is read as
// unit lower trapezoidal (0 above the diagonal, 1 on it).
enum OperandMode { kDense = 0, kUnitLower = 1 };

// Raises fn's dynamic shared-memory limit to the device maximum, once per
// device and kernel.  The limit is a property of the kernel, not of a
// launch, so setting it per launch to that launch's size would race between
// host threads (worker handles) launching the same kernel with different
// sizes: one thread's smaller value could land between another's set and
// launch.  Raising it once, to the maximum, is safe for every launch.
Status allow_max_dyn_smem(const void* fn);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no
// link-time libcuda dependency); nullptr when the driver lacks it.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder();

// Reusable device scratch owned by the caller of a launcher.
struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// sketch.cu -----------------------------------------------------------------
Status launch_philox_raw(uint64_t seed, int64_t step, int64_t groups, int64_t cols,
                         uint64_t* out, cudaStream_t st);
Status launch_sketch(uint64_t seed, int64_t step, int64_t rows, int64_t cols,
                     double* G, int64_t ldg, cudaStream_t st);
// Same sketch written as bf16 (mixed-precision sampling).
Status launch_sketch_bf16(uint64_t seed, int64_t step, int64_t rows, int64_t cols,
                          void* G, int64_t ldg, cudaStream_t st);

// gemm_f64.cu ----------------------------------------------------------------
// Scratch bytes the GEMM may use for split-K partial sums (0 = no split).
size_t gemm_scratch_bytes(int64_t m, int64_t n, int64_t k);
Status gemm(bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t m, int64_t n,
            int64_t k, double alpha, const double* A, int64_t lda, const double* B,
            int64_t ldb, double beta, double* C, int64_t ldc, Scratch scratch,
            cudaStream_t st);

// panel_qr.cu ----------------------------------------------------------------
// Most CTAs a cooperative panel kernel uses.
constexpr int kPanelMaxCtas = 256;
// Scratch of the cooperative panel kernels with G CTAs and n columns: the
// grid-barrier arrival counter (first 64 bytes), then the partial sums of
// the larger of the two kernels' layouts (global-memory kernel: one norm
// per CTA, one dot per CTA and column, one reduced dot per column;
// shared-memory kernel: two buffers of one value per CTA and column, two
// copies of one row, two of the column totals).
constexpr size_t panel_qr_scratch_layout_bytes(int64_t G, int64_t n) {
  return 64 + sizeof(double) * (size_t)std::max(G + G * n + n, 2 * G * n + 2 * n + 2 * (n + 4));
}
size_t panel_qr_scratch_bytes(int64_t m, int64_t n);
// Householder QR of the m x n panel in place; tau[min(m,n)]; err (device
// int) is raised if a grid barrier timed out.  shared_device: panels of other
// streams of this process may run at the same time (batched and served work):
// a panel that fits one thread-block cluster then always takes the cluster
// kernel, which needs no cooperative launch and so no library-wide gate;
// otherwise the cluster kernel is kept for panels of at most kClusterPanelRows
// rows, beyond which its FP64 work on <= 16 SMs outlasts the grid-wide slab
// kernel's barriers.
constexpr int64_t kClusterPanelRows = 1024;
Status panel_qr(int64_t m, int64_t n, double* A, int64_t lda, double* tau, Scratch scratch,
                int* err, cudaStream_t st, bool shared_device = false);
// Cooperative launch (all G CTAs resident at once, as the grid barrier
// needs) behind a library-wide gate that orders cooperative kernels of
// different streams, so two of them never wait on each other's CTAs.
Status coop_launch(const void* fn, int G, int threads, void** args, size_t smem,
                   cudaStream_t st);

// replay_persistent.cu -------------------------------------------------------
// The steps of one replay of stored block reflectors as one cooperative
// launch (nrhs <= 4, nb <= 128): step i (k = i nb, b = min(nb, kmax - k))
// applies I - W_i op(T_i) W_i^T to rows k..M-1 of x (ldx, nrhs columns),
// W_i the unit lower reflectors at W + k + k ldw, T_i the b x b upper factor
// at T + i nb^2 (ld nb); forward: steps 0..nsteps-1 with op(T) = T^T,
// otherwise nsteps-1..0 with op(T) = T.  err (device int) is raised if a
// grid barrier timed out.  The reflector chunks are TMA tensor loads, so W
// must be 16-byte aligned with an even ldw (replay_persistent_fits).
size_t replay_persistent_scratch_bytes(int64_t nb, int64_t nrhs);
bool replay_persistent_fits(int64_t nb, int64_t nrhs, const double* W, int64_t ldw, int64_t M,
                            int64_t kmax);
Status replay_persistent(bool forward, int64_t M, int64_t nb, int64_t nsteps, int64_t kmax,
                         const double* W, int64_t ldw, const double* T, double* x, int64_t ldx,
                         int64_t nrhs, Scratch scratch, int* err, cudaStream_t st);

// trsm_persistent.cu ----------------------------------------------------------
// trsm_upper_inv (below) for nrhs <= 4 as one cooperative launch, a grid
// barrier per 64-row block; scratch: 8 bytes (the barrier's counter); err
// (device int) is raised if a barrier timed out.
Status trsm_upper_inv_persistent(int64_t r, int64_t nrhs, const double* R, int64_t ldr,
                                 const double* Dinv, double* B, int64_t ldb, bool trans,
                                 Scratch scratch, int* err, cudaStream_t st);

// T factor (k x k, ldt) of H_0 ... H_{k-1} = I - W T W^T from the Gram
// matrix S = W^T W (k x k, lds) and tau.
Status wy_tfactor(int64_t k, const double* S, int64_t lds, const double* tau, double* T,
                  int64_t ldt, cudaStream_t st);

// jacobi_svd.cu --------------------------------------------------------------
// SVD of b x b R (b <= 128).  status: device int (0 / LLS_ERR_SVD_NOCONV).
Status jacobi_svd(int64_t b, const double* R, int64_t ldr, double* sigma, double* Us,
                  int64_t ldu, double* Vs, int64_t ldv, int* status, cudaStream_t st);

// small_kernels.cu -----------------------------------------------------------
// Copy src (m x n) to dst and raise *flag if any entry is not finite.
Status copy_check(int64_t m, int64_t n, const double* src, int64_t lds, double* dst,
                  int64_t ldd, int* flag, cudaStream_t st);
Status copy_matrix(int64_t m, int64_t n, const double* src, int64_t lds, double* dst,
                   int64_t ldd, cudaStream_t st);
Status fill_zero(int64_t m, int64_t n, double* dst, int64_t ldd, cudaStream_t st);
// dst (k x k) = upper triangle of src, zeros below.
Status copy_upper(int64_t k, const double* src, int64_t lds, double* dst, int64_t ldd,
                  cudaStream_t st);
// Upper triangle (diagonal included) of src (k x k) into dst; dst's strictly
// lower part is left as it is.
Status copy_upper_into(int64_t k, const double* src, int64_t lds, double* dst, int64_t ldd,
                       cudaStream_t st);
// V (n x n) = I.
Status set_identity(int64_t n, double* V, int64_t ldv, cudaStream_t st);
// dst (m x n) = upper trapezoid of src, zeros below the diagonal.
Status copy_upper_trapezoid(int64_t m, int64_t n, const double* src, int64_t lds, double* dst,
                            int64_t ldd, cudaStream_t st);
// X (n x nrhs) += D; norms (device, 2 nrhs) = per column ||d_j||^2, ||x_j||^2
// of the updated X, each summed in a fixed order.
Status refine_update(int64_t n, int64_t nrhs, const double* D, int64_t ldd, double* X, int64_t ldx,
                     double* norms, cudaStream_t st);
// Block (k x k) at D: diagonal = sigma, strictly upper part = 0, strictly
// lower part untouched (it holds Householder vectors).
Status set_diag_block(int64_t k, const double* sigma, double* D, int64_t ldd, cudaStream_t st);
// Compute_rank on diag(T).  out: device int64[3] = {prefix, count, nan}.
Status rank_scan(int64_t len, const double* T, int64_t ldt, double tol, int64_t* out,
                 cudaStream_t st);
// Default tolerance max(m,n) * eps * |T_00| written to *tol_dev if tol < 0.
Status resolve_tol(double tol, int64_t mn, const double* T00, double* tol_dev, cudaStream_t st);
// Rank scan with a device tolerance.
Status rank_scan_dev(int64_t len, const double* T, int64_t ldt, const double* tol_dev,
                     int64_t* out, cudaStream_t st);
// reflector_thin.cu: products with at most kThinMaxRhs right-hand sides.
constexpr int kThinMaxRhs = 16;
// y (M x nrhs) = beta y + alpha op(A) x with op(A) M x K: A (M x K, ld lda)
// or, trans, A^T for A K x M; unit_lower: the stored A reads as unit lower
// trapezoidal (0 above the diagonal, 1 on it).  The K split, and so the
// order of every sum, is a function of (trans, M, K, nrhs) only; split sums
// need thin_gemv_scratch_bytes of scratch (0 when there is no split).
size_t thin_gemv_scratch_bytes(bool trans, int64_t M, int64_t K, int64_t nrhs);
Status thin_gemv(bool trans, bool unit_lower, int64_t M, int64_t K, int64_t nrhs, double alpha,
                 const double* A, int64_t lda, const double* x, int64_t ldx, double beta, double* y,
                 int64_t ldy, Scratch scratch, cudaStream_t st);
size_t thin_scratch_bytes(int64_t M, int64_t b, int64_t nrhs);
// x (M x nrhs) <- (I - W op(T) W^T) x, W M x b unit lower trapezoidal (ld
// ldw), T b x b upper triangular, op(T) = T^T when transT; b <= 128.
Status apply_reflectors_thin(int64_t M, int64_t b, int64_t nrhs, const double* W, int64_t ldw,
                             const double* T, int64_t ldt, bool transT, double* x, int64_t ldx,
                             Scratch scratch, cudaStream_t st);
// xo(k_i + r) = sum_l op(S_i)(r, l) x(k_i + l) for every block i of a replay
// at once (k_i = i nb, b_i = min(nb, kmax - k_i), S_i = S + i nb^2, ld nb;
// nb <= 128, nrhs <= 65535), out of place.
Status small_blocks_batched(int64_t nblk, int64_t nb, int64_t kmax, int64_t nrhs, const double* S,
                            bool transS, const double* x, int64_t ldx, double* xo, int64_t ldxo,
                            cudaStream_t st);
// x(0:b, :) <- op(S) x(0:b, :) for a b x b block S (b <= 128).
Status small_block_mul(int64_t b, int64_t nrhs, const double* S, int64_t lds, bool transS,
                       double* x, int64_t ldx, cudaStream_t st);
// Gap at the rank of a diagonal d (len entries, contiguous): out (device,
// 2 doubles) = {min_{j < r} |d_j|, max_{j >= r} |d_j|}.
Status diag_gap(int64_t len, const double* d, int64_t r, double* out, cudaStream_t st);
// Reversed-index gather / scatter used by Nullify (see nullify in solver.cu).
Status rz_gather(int64_t bsz, int64_t L, const double* T, int64_t ldt, int64_t j0,
                 int64_t r, double* M, int64_t ldm, cudaStream_t st);
Status rz_scatter(int64_t bsz, const double* M, int64_t ldm, double* T, int64_t ldt,
                  int64_t j0, int64_t r, int64_t L, cudaStream_t st);
// Y <- Y + alpha X (m x n blocks).
Status axpy_matrix(int64_t m, int64_t n, double alpha, const double* X, int64_t ldx, double* Y,
                   int64_t ldy, cudaStream_t st);
// dst(i, :) = src(rows - 1 - i, :) for a rows x cols block.
Status copy_rows_reversed(int64_t rows, int64_t cols, const double* src, int64_t lds,
                          double* dst, int64_t ldd, cudaStream_t st);
// dst(rows - 1 - i, :) += alpha src(i, :).
Status axpy_rows_reversed(int64_t rows, int64_t cols, double alpha, const double* src, int64_t lds,
                          double* dst, int64_t ldd, cudaStream_t st);
// dst(:, j) = src(:, cols - 1 - j).
Status copy_cols_reversed(int64_t rows, int64_t cols, const double* src, int64_t lds,
                          double* dst, int64_t ldd, cudaStream_t st);
// Back substitution for one diagonal block: B (k x nrhs) <- R^{-1} B.
Status trsm_block(int64_t k, int64_t nrhs, const double* R, int64_t ldr, double* B,
                  int64_t ldb, cudaStream_t st);
// Scratch bytes trsm_upper needs for its split-K GEMM updates.
size_t trsm_upper_scratch_bytes(int64_t r, int64_t nrhs);
// B <- R^{-T} B (forward substitution with the transpose of the upper
// triangular r x r matrix R), blocked like trsm_upper.
size_t trsm_upper_trans_scratch_bytes(int64_t r, int64_t nrhs);
Status trsm_upper_trans(int64_t r, int64_t nrhs, const double* R, int64_t ldr, double* B,
                        int64_t ldb, Scratch scratch, cudaStream_t st);
Status trsm_upper(int64_t r, int64_t nrhs, const double* R, int64_t ldr, double* B,
                  int64_t ldb, Scratch scratch, cudaStream_t st);
// Inverses of the 64 x 64 diagonal blocks of an upper triangular r x r R
// (blocks from the top, the last one partial), trsm_inverse_bytes(r) bytes;
// then B <- R^{-1} B or, trans, R^{-T} B with them (nrhs <= kThinMaxRhs):
// each diagonal block is a product with its inverse instead of a serial
// substitution (the refinement's preconditioner applies T_11^{-1} and
// T_11^{-T} many times with the same factor).
size_t trsm_inverse_bytes(int64_t r);
Status trsm_block_inverses(int64_t r, const double* R, int64_t ldr, double* Dinv, cudaStream_t st);
Status trsm_upper_inv(int64_t r, int64_t nrhs, const double* R, int64_t ldr, const double* Dinv,
                      double* B, int64_t ldb, bool trans, cudaStream_t st);

}  // namespace lls
