/*
 * lls_kernels.h -- step-level entry points of the randUTV library.
 *
 * Each call runs one step of the method on caller-owned DEVICE buffers, on
 * the given cudaStream_t (NULL = legacy default stream), and returns after
 * enqueueing (no synchronization unless stated).  They exist so that every
 * kernel of the solver can be checked on its own; lls_solve chains the same
 * launchers.  Matrices are column-major FP64.  Return values follow lls.h:
 * LLS_OK, LLS_ERR_ARG (bad size / leading dimension / NULL pointer, nothing
 * launched), LLS_ERR_CUDA (launch failed) or LLS_ERR_NOMEM (scratch).
 */
#ifndef LLS_KERNELS_H
#define LLS_KERNELS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Raw Philox4x64-10 blocks (Salmon et al., SC'11) used by the sketch of
 * Fig. 2: block (g, j) has counter (g, j, step, 0) and key (seed, 0); its
 * four words go to out[4 * (g + groups * j) + w], w = 0..3. */
int lls_k_philox(uint64_t seed, int64_t step, int64_t groups, int64_t cols,
                 uint64_t* out, void* stream);

/* Gaussian sketch G (rows x cols, leading dimension ldg) of step `step`
 * (Fig. 2, generate_iid_stdnorm_matrix): entry (p, j) is normal number
 * p % 4 of the Box-Muller pairs of block (p / 4, j):
 *   u = ((w >> 11) + 1) 2^-53, t = (w >> 11) 2^-53,
 *   (G(4g, j), G(4g+1, j)) = sqrt(-2 ln u0) (cos 2 pi t1, sin 2 pi t1),
 *   (G(4g+2, j), G(4g+3, j)) = sqrt(-2 ln u2) (cos 2 pi t3, sin 2 pi t3). */
int lls_k_sketch(uint64_t seed, int64_t step, int64_t rows, int64_t cols,
                 double* G, int64_t ldg, void* stream);

/* C = alpha op(A) op(B) + beta C in FP64 (op(X) = X or X^T for trans = 0/1).
 * op(A) is m x k, op(B) is k x n.  unit_lower_a / unit_lower_b = 1 reads
 * the stored matrix as unit lower trapezoidal (entries above the diagonal
 * read as 0, the diagonal as 1), the layout of Householder vectors kept
 * below a QR's R (the "W" of Fig. 2).  beta = 0 ignores the old C. */
int lls_k_gemm(int transa, int transb, int unit_lower_a, int unit_lower_b,
               int64_t m, int64_t n, int64_t k, double alpha,
               const double* A, int64_t lda, const double* B, int64_t ldb,
               double beta, double* C, int64_t ldc, void* stream);

/* Householder QR of the m x n panel A in place (unpivoted_QR of Fig. 2):
 * on return R is in the upper trapezoid and the Householder vectors W (unit
 * diagonal implied) below the diagonal, tau[min(m,n)] holds the scalars and
 * T (min(m,n) x min(m,n), ldt) the upper triangular compact-WY factor with
 * H_0 H_1 ... H_{k-1} = I - W T W^T.  LAPACK xLARFG sign convention. */
int lls_k_geqrf(int64_t m, int64_t n, double* A, int64_t lda, double* tau,
                double* T, int64_t ldt, void* stream);

/* SVD of the b x b block R (b <= 128) by one-sided Jacobi (Fig. 2,
 * SVD(A_11)): R = Us diag(sigma) Vs^T, sigma descending >= 0.  One CTA for
 * b < 32, else a thread-block cluster of 4 (b <= 64) or 8 CTAs.
 * status (device int, may be NULL) receives 0, or LLS_ERR_SVD_NOCONV when
 * the sweep limit was hit. */
int lls_k_jacobi_svd(int64_t b, const double* R, int64_t ldr, double* sigma,
                     double* Us, int64_t ldu, double* Vs, int64_t ldv,
                     int* status, void* stream);

/* B <- R^{-1} B for the upper triangular r x r matrix R (only its upper
 * triangle is read), B r x nrhs: the T_tl^{-1} of Fig. 4. */
int lls_k_trsm_upper(int64_t r, int64_t nrhs, const double* R, int64_t ldr,
                     double* B, int64_t ldb, void* stream);

/* B <- R^{-T} B for the upper triangular r x r matrix R (only its upper
 * triangle is read), B r x nrhs: the T_11^{-T} of the transposed solve
 * operator P^T = U_1 T_11^{-T} V_1^T used by the refinement of the TF32
 * modes (see lls_options.max_refine). */
int lls_k_trsm_upper_trans(int64_t r, int64_t nrhs, const double* R, int64_t ldr,
                           double* B, int64_t ldb, void* stream);

/* B <- R^{-1} B (trans = 0) or R^{-T} B (trans = 1) for the upper
 * triangular r x r matrix R through the inverses of its 64 x 64 diagonal
 * blocks, the triangular solves of the refinement of the TF32 modes
 * (T_11^{-1} and T_11^{-T} of Fig. 4's solve operator): with nrhs <= 4 one
 * cooperative launch with a grid barrier per block (LLS_ERR_TIMEOUT if a
 * barrier wait ran out; R and B stay valid device memory), with nrhs <= 16
 * two launches a block; LLS_ERR_ARG for nrhs > 16.  Scratch is allocated
 * stream-ordered on `stream` and freed before returning; the call waits for
 * the stream. */
int lls_k_trsm_upper_blockinv(int64_t r, int64_t nrhs, const double* R, int64_t ldr,
                              double* B, int64_t ldb, int trans, void* stream);

/* Compute_rank (Fig. 4) of diag(T) (len entries, T with leading dimension
 * ldt): out[0] = length of the leading run of |T_jj| > tol, out[1] = number
 * of |T_jj| > tol, out[2] = 1 if a diagonal entry is NaN (device int64[3]). */
int lls_k_rank(int64_t len, const double* T, int64_t ldt, double tol,
               int64_t* out, void* stream);

/* D = X^T Z on the tcgen05 tensor cores: X is K x M and Z is K x N, both
 * column-major BF16 (ldx, ldz multiples of 8, 16-byte aligned base), D is
 * M x N column-major FP32 (ldd >= M), N <= 128.  BF16 products, FP32
 * accumulation.  This is the sampling product Y = A^T G (and A^T (A Y)) of
 * Fig. 2 in mixed precision.  status (device int) becomes nonzero if a
 * device-side wait timed out.  Scratch for split-K partial sums is
 * allocated and freed on the stream inside the call. */
int lls_k_gemm_bf16_tn(int64_t M, int64_t N, int64_t K, const void* X, int64_t ldx,
                       const void* Z, int64_t ldz, float* D, int64_t ldd, int* status,
                       void* stream);

/* C = alpha op(A) op(B) + beta C with FP64 operands and result, computed on
 * the BF16 tensor cores by exact slicing (Ozaki-style): each row of op(A)
 * and column of op(B) is scaled by a power of two and split into 8 signed
 * base-128 integer digit planes stored as BF16; the 36 digit-plane products
 * with s + t <= 9 accumulate exactly in FP32 (at most 256 K entries per
 * partial product), are recombined exactly in 64-bit integers (one rounding
 * at 2^-55 of the row/column scale) and summed in FP64.
 * Same operand conventions as lls_k_gemm.  Accuracy: at least that of an
 * FP64 GEMM relative to max_k |op(A)_ik| max_k |op(B)_kj|.  status (device
 * int) becomes nonzero if a device-side wait timed out.  Workspace is
 * allocated and freed on the stream inside the call. */
int lls_k_gemm_oz(int transa, int transb, int unit_lower_a, int unit_lower_b,
                  int64_t m, int64_t n, int64_t k, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb,
                  double beta, double* C, int64_t ldc, int* status, void* stream);

/* C = alpha op(A) op(B) + beta C with FP64 operands and result on the TF32
 * tensor cores (tcgen05 kind::tf32), the product of the trailing WY updates
 * of the TF32 precision modes (Fig. 2, right and left updates; Fig. 3,
 * Nullify's updates).  Every entry x of op(A) and op(B) is split into TF32
 * terms hi = x rounded to 11 significant bits and lo = (x - hi) rounded to
 * 11 bits; terms = 3 sums hi*hi + hi*lo + lo*hi (3xTF32, about 2^-21
 * relative to sum_k |a_k b_k|), terms = 1 only hi*hi (plain TF32, about
 * 2^-11).  FP32 accumulation in tensor memory over K ranges of 1024, the
 * ranges summed in FP64.  Entries must lie inside FP32's range (|x| <
 * 2^128, else the result is not finite; below 2^-126 they count as zero).
 * Same operand conventions as lls_k_gemm; LLS_ERR_ARG for terms other than
 * 1 or 3.  status (device int) becomes nonzero if a device-side wait timed
 * out.  Workspace is allocated and freed on the stream inside the call. */
int lls_k_gemm_tf32(int transa, int transb, int unit_lower_a, int unit_lower_b,
                    int64_t m, int64_t n, int64_t k, double alpha,
                    const double* A, int64_t lda, const double* B, int64_t ldb,
                    double beta, double* C, int64_t ldc, int terms, int* status,
                    void* stream);

/* The Householder panel QR of lls_k_geqrf (R, W and tau in place; no T
 * factor) for callers that cannot allocate device memory: code whose device
 * memory is owned by another allocator (a framework's pool, a fixed budget
 * set at start-up), or loops that must not block, since cudaMalloc/cudaFree
 * can synchronize the device.  The paper has no counterpart; this is a
 * library convenience.
 *
 * The kernel's scratch (the grid barrier's arrival counter and per-CTA
 * partial sums) lives in one fixed array of the library (528,512 bytes,
 * about 516 KiB, held by every GPU that loads the library until the process
 * exits), so this call allocates nothing.  n may be at most 128; larger n returns LLS_ERR_CAPACITY and
 * launches nothing.  status is a caller-owned device int: it is set to 0 and
 * becomes nonzero if a grid barrier of the kernel timed out (then A and tau
 * are not valid).  The call only enqueues work on `stream`; it does not
 * synchronize.  The first call on each device looks up the array's device
 * address (once, with that device current), so make that first call before
 * any stream capture.  All calls share the one array, which keeps the last
 * call's contents (the barrier counter is cleared by each call): calls that
 * overlap on the GPU -- on different streams, or from several threads --
 * race on it, so issue them one after another. */
int lls_k_panel_qr_noalloc(int64_t m, int64_t n, double* A, int64_t lda, double* tau,
                           int* status, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LLS_KERNELS_H */
