/*
 * lls.h -- C ABI of the B300 (sm_103a) randUTV least-squares library.
 *
 * The library computes the least-squares solution of A x = b that
 * (1) minimizes ||A x - b||_2 and (2) among the minimizers has the smallest
 * ||x||_2 (Chillaron, Quintana-Orti, Vidal, Martinsson, arXiv 2408.05238,
 * Sec. 2, conditions (1)-(2)).  It factors A V = U T with randUTV (Fig. 2),
 * decides the numerical rank r against a tolerance (Compute_rank, Fig. 4),
 * annihilates T(0:r, r:n) (Nullify, Fig. 3) and returns
 * x = V T(0:r,0:r)^{-1} U(:,0:r)^T b (Fig. 4; Eq. (4) when r = n).
 *
 * Conventions shared by every call:
 *  - Matrices are column-major FP64.  A is m x n with leading dimension
 *    lda >= max(1, m); B is m x nrhs (ldb >= max(1, m)); X is n x nrhs
 *    (ldx >= max(1, n)).  Sizes are int64.
 *  - Pointers passed to lls_solve / lls_factor / lls_solve_factored /
 *    lls_solve_batched / lls_submit are DEVICE pointers on the handle's
 *    device; lls_solve_host takes HOST pointers.  The caller owns every
 *    buffer it passes and must keep it alive until the call returns (or, for
 *    lls_submit, until lls_poll reports completion).  The library never
 *    frees or retains caller memory; A and B are only read.
 *  - The handle owns its stream (or borrows the one given to lls_create),
 *    its workspace and every resident factorization.  A handle is not
 *    thread-safe: one host thread at a time.
 *  - Return value: LLS_OK (0), a positive warning (the result is valid) or
 *    a negative error.  After LLS_ERR_ARG, lls_last_error() reports the
 *    1-based index of the offending argument (LAPACK's info = -i).
 *  - m = 0, n = 0 or nrhs = 0 are valid and do nothing (rank 0, X = 0).
 *  - Non-finite entries in A or B give LLS_ERR_NONFINITE (no result).
 */
#ifndef LLS_H
#define LLS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
enum {
  LLS_OK = 0,
  LLS_PENDING = 1,              /* lls_poll: request not finished yet */
  LLS_WARN_RANK_NONPREFIX = 2,  /* some |T_jj| > tol after the first |T_jj| <= tol */
  LLS_WARN_REFINE_NOCONV = 3,   /* refinement stopped with its last correction
                                   above refine_tol (x is still the refined one) */
  LLS_ERR_ARG = -1,             /* invalid argument (see lls_last_error) */
  LLS_ERR_NOMEM = -2,           /* device or host allocation failed */
  LLS_ERR_CUDA = -3,            /* a CUDA runtime call failed */
  LLS_ERR_NONFINITE = -4,       /* NaN or Inf in A or B */
  LLS_ERR_SVD_NOCONV = -5,      /* block SVD hit its sweep limit */
  LLS_ERR_TIMEOUT = -6,         /* a device-side wait hit its iteration limit */
  LLS_ERR_NOT_FOUND = -7,       /* unknown factor id or ticket */
  LLS_ERR_CAPACITY = -8         /* request larger than the serving memory cap */
};

/* ---- precision modes --------------------------------------------------- */
enum {
  LLS_FP64 = 0,        /* every step in FP64 */
  LLS_MIXED_BF16 = 1,  /* sampling products (step a2) in BF16 on the tcgen05
                          tensor cores with FP32 accumulation; the trailing
                          WY updates and Nullify's products as FP64-accurate
                          tensor-core GEMMs (exact BF16 digit slices, FP32
                          accumulation, FP64 recombination, see
                          lls_k_gemm_oz); panels, block SVDs, rank and the
                          solve in FP64 */
  LLS_MIXED_BF16_3xTF32 = 2,  /* BF16 sampling as above; the trailing WY
                          updates and Nullify's products on the TF32 tensor
                          cores with split operands, hi*hi + hi*lo + lo*hi,
                          FP32 accumulation (lls_k_gemm_tf32, terms = 3), so
                          the factorization carries errors of about 2^-21
                          ||A||; panels, block SVDs, rank and the solve in
                          FP64.  The accuracy of x is won back by max_refine
                          steps of the minimum-norm refinement (see
                          max_refine); the rank is revealed when tol and the
                          kept singular values lie well above that noise
                          (e.g. tol = 1e-6 ||A||) */
  LLS_MIXED_BF16_TF32 = 3     /* the same with plain TF32 products (terms = 1):
                          errors of about 2^-11 ||A||, which hide singular
                          values below about 1e-3 ||A|| -- the rank of such
                          matrices is not revealed and refinement cannot
                          repair it; kept as the baseline of the split */
};

typedef struct lls_handle_s* lls_handle;

/* Options (lls_default_options fills the defaults in brackets). */
typedef struct {
  int32_t nb;          /* block size n_b of Fig. 2, 1..128 [64]; 0: n_b and q
                          from the handle's tuning table (lls_autotune) */
  int32_t q;           /* power iterations of Y = (A^T A)^q A^T G, 0..4 [1] */
  int32_t precision;   /* LLS_FP64 | LLS_MIXED_BF16 | LLS_MIXED_BF16_3xTF32 |
                          LLS_MIXED_BF16_TF32 [LLS_FP64] */
  int32_t nullify;     /* 1: run Nullify (minimum-norm x, Fig. 3) [1];
                          0: fast option (Remark after Fig. 4, Eq. (7)): a
                          least-squares x whose excess norm is of the size
                          of T_12, only with precision LLS_FP64 (LLS_ERR_ARG,
                          index 2, otherwise: a BF16 sample fixes V_1 only to
                          BF16 accuracy, so T_12 and the excess norm would be
                          of order 1e-4..1e-2 relative) */
  uint64_t seed;       /* key of the Gaussian sketch generator [2001] */
  int32_t explicit_v;  /* 1: accumulate V (n x n) during the factorization
                          (V <- V (I - W_V T_V W_V^T), V_01 <- V_01 V_SVD,
                          Nullify's reflectors from the right, Fig. 2-3);
                          solves then apply V as one GEMM and
                          lls_factor_get can return it; 0: V is kept as its
                          reflectors and applied by replaying them [0] */
  int32_t max_refine;  /* iterative refinement steps after the solve, 0..16
                          [0] (see lls_refinement_info).  LLS_FP64 and
                          LLS_MIXED_BF16 (FP64-accurate factors):
                          x <- x + P (b - A x) with the FP64 residual and
                          P = V_1 T_11^{-1} U_1^T the factorization's solve
                          operator.  The TF32 modes (factors accurate to the
                          TF32 split only) refine in two stages from
                          x_0 = P b: (1) least squares,
                          x <- x + N N^T A^T (b - A x) with N = V_1 T_11^{-1},
                          then (2) the projection onto range(A^T):
                          x <- x + L L^T (x_ls - x) from 0 with
                          L = A^T U_1 T_11^{-T}; each stage contracts by
                          about the factors' relative error times the
                          condition number of T_11 (kappa eps < 1), and
                          max_refine bounds each stage's steps.  When the
                          largest dropped |T(i,i)| is above 1e-2 times the
                          smallest kept one the split is not reliable and
                          no refinement runs (LLS_WARN_REFINE_NOCONV).
                          With max_refine = 0 these modes return x = P b at
                          TF32 accuracy */
  double refine_tol;   /* refinement stops once every column has
                          ||dx_j|| <= refine_tol ||x_j||, >= 0 [1e-12] */
  int32_t reserved[2]; /* must be zero */
} lls_options;

/* One problem of lls_solve_batched / one request of lls_submit (device
 * pointers).  rank_out, if not NULL, is a HOST pointer written when the
 * problem is done. */
typedef struct {
  const double* A; int64_t m, n, lda;
  const double* B; int64_t nrhs, ldb;
  double tol;
  double* X; int64_t ldx;
  int64_t* rank_out;
  int64_t factor_id;   /* lls_submit only: >= 0 reuses a resident factor
                          (A ignored; m, n must match), -1 factors A; with
                          keep_factor = 1 the new factor stays resident */
  int32_t keep_factor;
  int32_t status;      /* written by lls_solve_batched: per-problem status */
} lls_problem;

/* ---- autotuning of n_b and q ---------------------------------------------
 * With opt.nb == 0 a factorization of an m x n matrix takes n_b and q from
 * the handle's tuning table entry for its bucket (ceil(log2 m), ceil(log2 n));
 * a bucket without an entry uses n_b = 64, q = 1.  Worker handles of
 * lls_solve_batched / lls_submit share the table.
 *
 * lls_autotune fills the entry of the bucket of (m, n).  On a synthetic m x n
 * matrix X Y of rank min(m, n)/2 (X, Y Gaussian from the library's Philox
 * generator, X's columns scaled so the singular values spread over four
 * decades) with one Gaussian right-hand side and the default tol, it runs the
 * reference choice n_b = 32, q = 2, then, for each n_b in {32, 64, 128}
 * (n_b <= min(m, n) beyond 32; not above 64 when the handle's batches run in
 * the persistent launch) and q in {0, 1, 2}, checks one solve against the
 * reference and times `trials` copies of the problem solved together by
 * lls_solve_batched (host wall clock, the handle's batched mode and
 * precision) -- the concurrency batched and served work runs with -- and
 * keeps the fastest candidate whose rank equals the reference's and whose x
 * agrees with the reference x to 1e-9 relative.  nb_out, q_out (host, may be NULL)
 * receive the choice.  Errors: LLS_ERR_ARG (m, n outside 1..2^20, trials < 1,
 * or requests of this handle queued or running), LLS_ERR_NOMEM, and those of
 * lls_solve. */
int lls_autotune(lls_handle h, int64_t m, int64_t n, int32_t trials, int32_t* nb_out,
                 int32_t* q_out);
/* The (n_b, q) a tuned solve (opt.nb == 0) of an m x n matrix would use. */
int lls_tuning_lookup(lls_handle h, int64_t m, int64_t n, int32_t* nb, int32_t* q);
/* Write the table as text, one "bucket_m bucket_n n_b q" line per entry;
 * read such a file and merge it into the table.  LLS_ERR_ARG when the file
 * cannot be opened or a line is malformed (nothing is merged then). */
int lls_tuning_save(lls_handle h, const char* path);
int lls_tuning_load(lls_handle h, const char* path);

/* Fill *opt with the defaults.  Returns LLS_OK or LLS_ERR_ARG (opt NULL). */
int lls_default_options(lls_options* opt);

/* Create a handle on the current CUDA device.  opt NULL = defaults.
 * cuda_stream: a cudaStream_t to borrow, or NULL for a handle-owned stream.
 * A borrowed stream must outlive the handle: the handle's workspace is
 * allocated and freed in stream order on it (cudaMallocAsync /
 * cudaFreeAsync), up to lls_destroy.
 * Errors: LLS_ERR_ARG (bad option; index 2), LLS_ERR_CUDA, LLS_ERR_NOMEM. */
int lls_create(lls_handle* h, const lls_options* opt, void* cuda_stream);

/* Free the handle, its workspace and all resident factors. */
int lls_destroy(lls_handle h);

/* Change the options (every field of lls_options) for later calls. */
int lls_set_options(lls_handle h, const lls_options* opt);

/* Solve min ||A X - B|| with minimum ||X|| (per column) by the method of
 * Sec. 3.2: A = U T V^T by randUTV (Fig. 2), the numerical rank r from
 * diag(T) (Compute_rank), Nullify of T(0:r, r:n) (Fig. 3), then
 * X = V(:, 0:r) T(0:r, 0:r)^{-1} U(:, 0:r)^T B (Fig. 4).  tol absolute:
 * diagonal entries of T with |T_jj| <= tol count as zero (tol < 0 selects
 * max(m,n) * eps * |T_00|).  Synchronous: returns when X is written.
 * rank (host pointer, may be NULL) receives r.  A is not modified. */
int lls_solve(lls_handle h, const double* A, int64_t m, int64_t n, int64_t lda,
              const double* B, int64_t nrhs, int64_t ldb, double tol,
              double* X, int64_t ldx, int64_t* rank);

/* As lls_solve with HOST pointers: A and B are copied to the device, X is
 * copied back, all inside the call (pinned host memory is fastest). */
int lls_solve_host(lls_handle h, const double* A, int64_t m, int64_t n, int64_t lda,
                   const double* B, int64_t nrhs, int64_t ldb, double tol,
                   double* X, int64_t ldx, int64_t* rank);

/* Factor A and keep the factorization resident (the paper's variants that
 * keep U and V for later right-hand sides, Sec. 3.5).
 * *factor_id receives a handle-local id (>= 0). */
int lls_factor(lls_handle h, const double* A, int64_t m, int64_t n, int64_t lda,
               double tol, int64_t* factor_id, int64_t* rank);

/* Solve with a resident factorization and new right-hand sides. */
int lls_solve_factored(lls_handle h, int64_t factor_id, const double* B, int64_t nrhs,
                       int64_t ldb, double* X, int64_t ldx);

/* Release a resident factorization. */
int lls_factor_release(lls_handle h, int64_t factor_id);

/* What lls_factor_get copies. */
enum {
  LLS_FACTOR_T = 0,  /* T (m x n): upper trapezoid, zeros below the
                        diagonal; after Nullify T(0:r, r:n) = 0 */
  LLS_FACTOR_V = 1   /* V (n x n, orthogonal, A V = U T; after Nullify it
                        includes Nullify's reflectors); needs a factor made
                        with explicit_v = 1 */
};

/* Copy a resident factor's T or V (which = LLS_FACTOR_T / LLS_FACTOR_V) to
 * the DEVICE buffer dst (column-major, ld >= max(1, rows)).  Synchronous.
 * LLS_ERR_ARG: unknown `which`, ld too small, NULL dst, or V of a factor
 * made without explicit_v (index 3); LLS_ERR_NOT_FOUND: unknown id. */
int lls_factor_get(lls_handle h, int64_t factor_id, int32_t which, double* dst, int64_t ld);

/* Refinement of the last lls_solve / lls_solve_host / lls_solve_factored on
 * h: *steps (host, may be NULL) receives the number of corrections applied
 * (0 when max_refine = 0 or the factor kept no copy of A), *correction
 * (host, may be NULL) the last one's max_j ||dx_j|| / ||x_j||.  Refinement
 * stops at max_refine steps, once the correction is <= refine_tol, or when
 * a correction is not below half the previous one (the FP64 residual's
 * rounding floor); the call returns LLS_WARN_REFINE_NOCONV when that last
 * correction is still above refine_tol.  lls_solve refines with the
 * caller's A; lls_solve_factored and requests with a resident factor refine
 * only when the factor was made with max_refine > 0, in which case it holds
 * a copy of A (m x n more device memory).  Batched and served requests
 * refine the same way (their status carries the warning). */
int lls_refinement_info(lls_handle h, int32_t* steps, double* correction);

/* Copy |diag(T)| (min(m,n) values) of a resident factor to a HOST buffer;
 * rank_count (host, may be NULL) receives the number of entries > tol. */
int lls_factor_diag(lls_handle h, int64_t factor_id, double* diag, int64_t len,
                    int64_t* rank_count);

/* Solve count independent problems (device pointers in each entry).
 * Blocks until all are done.  Returns the first error; each entry's status
 * field holds its own result.  Two ways to run the batch (lls_set_batched_mode):
 *  - persistent: the randUTV step loop and block SVDs (Fig. 2) of every
 *    problem run in ONE kernel launch -- the paper's algorithm-by-blocks
 *    idea (Sec. 3.4): each problem's factorization is cut into tasks on
 *    64 x 64 blocks (sketch rows, sample and update tiles, the panel QRs with
 *    their T factors, the block SVDs and their updates), a device task queue
 *    holds one (phase, tasks claimed) word per problem, any CTA of the
 *    persistent grid claims a ready task (largest problems first) and the
 *    last task of a phase releases the next one (per-problem dependency
 *    counters).  Then the worker pool decides each rank, runs Nullify and the
 *    solve.  The factors are those of lls_solve up to the order of
 *    floating-point sums.  FP64 only, explicit_v = 0, 1 <= m, n <= 16384,
 *    n_b <= 64; the factors and workspace of all problems are held at once
 *    (about 8 (m n + n^2 + 6 m n_b) bytes each).  A waiting CTA polls the
 *    queue a bounded number of times (lls_debug_barrier_limit sets the same
 *    limit) and then ends the launch with LLS_ERR_TIMEOUT for every problem.
 *  - workers: each problem runs lls_solve's launch sequence on one of the
 *    pool's worker streams (lls_set_workers), largest first, several at a
 *    time. */
int lls_solve_batched(lls_handle h, int64_t count, lls_problem* problems);

/* How lls_solve_batched runs a batch: LLS_BATCHED_AUTO (persistent when
 * every problem and the options allow it, else workers; the default),
 * LLS_BATCHED_WORKERS, or LLS_BATCHED_PERSISTENT (lls_solve_batched then
 * returns LLS_ERR_ARG, index 3, for a batch it cannot take).  LLS_ERR_ARG
 * for another mode. */
enum { LLS_BATCHED_AUTO = 0, LLS_BATCHED_WORKERS = 1, LLS_BATCHED_PERSISTENT = 2 };
int lls_set_batched_mode(lls_handle h, int mode);

/* Serving: enqueue one request (copied; buffers must stay alive until it
 * completes) and return at once; *ticket receives its id.  Each request is
 * one solve of lls_solve (Sec. 3.2, Figs. 2-4), or with a resident factor
 * the solve of Fig. 4 alone.  Requests start in
 * arrival order as soon as a worker of the pool is free and the estimated
 * device memory of the running requests stays under the cap
 * (lls_set_memory_cap), and run concurrently on separate streams.
 * LLS_ERR_CAPACITY if the request alone exceeds the cap. */
int lls_submit(lls_handle h, const lls_problem* request, int64_t* ticket);

/* Serving: report a ticket's state in *status without blocking:
 * LLS_PENDING, or the request's final status.  A finished ticket is
 * forgotten after it has been reported once. */
int lls_poll(lls_handle h, int64_t ticket, int* status);

/* Serving: device-memory cap in bytes for admitted work (0 = no cap). */
int lls_set_memory_cap(lls_handle h, int64_t bytes);

/* Serving: for a request submitted with keep_factor = 1, *factor_id
 * receives the id of its resident factorization once it has finished
 * (LLS_PENDING before; call it before lls_poll forgets the ticket). */
int lls_ticket_factor(lls_handle h, int64_t ticket, int64_t* factor_id);

/* Withdraw a request that has not started: LLS_OK, and the ticket is
 * forgotten (lls_poll then returns LLS_ERR_NOT_FOUND); LLS_ERR_NOT_FOUND when
 * the ticket is unknown or its request has already started or finished
 * (poll it as usual). */
int lls_cancel(lls_handle h, int64_t ticket);

/* Number of worker streams (1..64, default 4) used by lls_solve_batched and
 * lls_submit; waits for running requests and drops queued ones. */
int lls_set_workers(lls_handle h, int workers);

/* ---- out-of-core planning ---------------------------------------------
 * The host<->device traffic of a solve whose m x n matrix stays in host
 * memory and moves through a device cache of `cache_panels` whole column
 * panels (nb columns, all m rows; the paper's block cache, Sec. 3.5, with
 * device memory as the cache and host memory as the disk).  The plan visits
 * the trailing panels in passes: per step of Fig. 2 the sampling passes
 * (the first product A^T G taken in the previous step's update pass; q + 1
 * passes for q >= 1), the pass forming T(:, k:n) W_V, and the update pass
 * (right and left updates, modifying the panels); then one pass for the
 * block-SVD updates; with nullify = 1 and 0 < rank < n, per panel-aligned
 * row block of Nullify (Fig. 3) a read and a write pass over its own panel
 * and the panels of T(0:r, r:n) (plus one gathering pass before the first
 * block); and the solve's reads (Fig. 4).  Consecutive passes alternate
 * direction.  policy LLS_OOC_FARTHEST evicts the panel whose next use lies
 * latest in the future (the paper's "LFU" policy, Belady's MIN: the access
 * list is known before the solve starts), LLS_OOC_LRU the least recently
 * used one; a modified panel is written back when evicted and at the end.
 * Host computation only (no device is touched).  LLS_ERR_ARG for m, n < 0,
 * nb < 1, q outside 0..4, rank outside 0..min(m, n), nullify not 0/1,
 * cache_panels < 1, an unknown policy, more than 2^24 panels or out NULL. */
enum { LLS_OOC_FARTHEST = 0, LLS_OOC_LRU = 1 };
typedef struct {
  int64_t panels;      /* column panels of nb columns (the last may be narrower) */
  int64_t passes;      /* passes over panels in the plan */
  int64_t accesses;    /* panel visits */
  int64_t hits;        /* visits that found the panel on the device */
  int64_t loads;       /* host->device panel copies (the other visits) */
  int64_t stores;      /* device->host write-backs of modified panels */
  double load_bytes;   /* bytes of those copies (whole panels, m rows) */
  double store_bytes;
  double side_bytes;   /* W_V of every step and Nullify's reflector panels:
                          written to host memory once, read back once */
} lls_ooc_stats;
int lls_ooc_plan(int64_t m, int64_t n, int32_t nb, int32_t q, int64_t rank, int32_t nullify,
                 int64_t cache_panels, int32_t policy, lls_ooc_stats* out);

/* What a planned access does (the kinds named in lls_ooc_plan's passes). */
enum {
  LLS_OOC_K_SAMPLE_ATG = 0,     /* step 0: Y_j = A_j^T G */
  LLS_OOC_K_SAMPLE_AY = 1,      /* W += A_j Y_j */
  LLS_OOC_K_SAMPLE_ATW_AY = 2,  /* Y_j = A_j^T W, then W' += A_j Y_j */
  LLS_OOC_K_SAMPLE_ATW = 3,     /* Y_j = A_j^T W */
  LLS_OOC_K_PRODUCT_TWV = 4,    /* P += T(:, panel) W_V(panel rows) */
  LLS_OOC_K_UPDATE = 5,         /* right update; panel QR (panel = step) or left update;
                                   the next step's A_j^T G */
  LLS_OOC_K_SVD = 6,            /* the block SVDs' V_s and U_s^T updates */
  LLS_OOC_K_NULL_GATHER = 7,    /* rows of D = T(0:r, r:n) of the first Nullify block */
  LLS_OOC_K_NULL_READ = 8,      /* Nullify block `step`: reflectors (its own panel), P */
  LLS_OOC_K_NULL_WRITE = 9,     /* Nullify block `step`: updates, the next block's rows */
  LLS_OOC_K_SOLVE_UTB = 10,     /* c = U^T b with the panel's W_U */
  LLS_OOC_K_SOLVE_TRSM = 11,    /* back substitution with the panel's columns of T_11 */
  LLS_OOC_K_FLUSH = 12          /* final write-back of a modified panel */
};

/* One entry of an out-of-core schedule: before the access, the panel in
 * `slot` (evict, or -1) is written back to host memory if store = 1, then
 * `panel` is copied into `slot` if load = 1; the access (kind, for step or
 * Nullify row block `step`, in pass number `pass` of the schedule) then works
 * on the panel in `slot`, modifying it if write = 1.  FLUSH entries (pass -1)
 * write back `panel` from `slot`. */
typedef struct {
  int32_t kind;
  int32_t write;
  int64_t step;
  int64_t pass;
  int64_t panel;
  int64_t slot;
  int64_t evict;
  int32_t store;
  int32_t load;
} lls_ooc_action;

/* The schedule behind lls_ooc_plan (same arguments): *count receives the
 * number of entries; with actions not NULL they are copied there
 * (LLS_ERR_CAPACITY, nothing copied, when max_actions is smaller).  Slots
 * are numbered 0..min(cache_panels, panels)-1.  phase 0 is the whole solve;
 * phase 1 the factorization (step loop and block-SVD pass, which do not
 * depend on the rank), ending with every modified panel written back; phase
 * 2 Nullify and the solve's reads for the given rank, starting from an empty
 * cache -- the split lls_solve_ooc runs, since the rank is known only after
 * phase 1.  LLS_ERR_ARG also for phase outside 0..2. */
int lls_ooc_schedule(int64_t m, int64_t n, int32_t nb, int32_t q, int64_t rank,
                     int32_t nullify, int64_t cache_panels, int32_t policy, int32_t phase,
                     lls_ooc_action* actions, int64_t max_actions, int64_t* count);

/* Out-of-core solve: as lls_solve_host (A m x n, B m x nrhs and X n x nrhs
 * in HOST memory, column-major; pinned memory is not required), with A
 * copied into a pinned host store and at most cache_panels column panels of
 * nb columns of it on the device at any time, moved by the schedule of
 * lls_ooc_schedule (phase 1, then phase 2 once the rank is known) under
 * `policy`.  Device memory used: cache_panels * m * nb doubles plus
 * O((m + n) nb + nb^2 s) for the sketch, the samples, the WY products and
 * the per-step factors; each step's W_V and Nullify's reflector panels go to
 * pinned host memory (host memory used: m n for the copy of A, n^2 for the
 * W_V and (r / nb)(nb + n - r) nb for the reflector panels, in doubles).  Same arithmetic as lls_solve (FP64; the handle's nb,
 * q, nullify and seed), so x agrees with lls_solve's to rounding.  Copies
 * and compute run in stream order on the handle's stream.
 * Errors: those of lls_solve_host; LLS_ERR_ARG also for cache_panels < 1
 * (index 13), an unknown policy (14), or a handle whose options ask for
 * LLS_MIXED_BF16, explicit_v or max_refine (index 1). */
int lls_solve_ooc(lls_handle h, const double* A, int64_t m, int64_t n, int64_t lda,
                  const double* B, int64_t nrhs, int64_t ldb, double tol, double* X,
                  int64_t ldx, int64_t* rank, int64_t cache_panels, int32_t policy);

/* The cache of lls_ooc_plan run over any access list: access t touches panel
 * panels[t] (0 <= panels[t] < num_panels) and modifies it when writes[t] is
 * nonzero (writes may be NULL: no modification); every panel is rows x cols
 * FP64.  Fills loads, stores, hits, accesses, panels and the byte counts
 * (passes and side_bytes are 0).  LLS_ERR_ARG on a bad argument. */
int lls_ooc_simulate(const int64_t* panels, const int8_t* writes, int64_t count,
                     int64_t num_panels, int64_t rows, int64_t cols, int64_t cache_panels,
                     int32_t policy, lls_ooc_stats* out);

/* ---- tracing (per-kernel-family CUDA-event timing) --------------------- */
typedef struct {
  char name[32];     /* kernel family, e.g. "dgemm_kernel" */
  int64_t launches;  /* launches recorded while tracing was on */
  double seconds;    /* summed device time between the events around them */
  double flops;      /* summed algorithmic flops of those launches */
  double bytes;      /* summed algorithmic bytes moved by those launches */
} lls_trace_stat;

/* Turn tracing on (1) or off (0) for later calls on h; turning it on clears
 * the counters.  Events are recorded on the handle's stream around every
 * kernel launch the calls make (the paper's per-task time table), and
 * around each phase of the method: entries named "phase:sample",
 * "phase:qr_y", "phase:right_update", "phase:panel", "phase:left_update",
 * "phase:block_svd", "phase:rank", "phase:nullify" and "phase:solve" (steps
 * a1/a2 .. a10), and "phase:refine" (the iterative refinement after the
 * solve); a phase's time includes the kernels it launches, so phases and
 * kernel families are two views of the same time. */
int lls_trace_enable(lls_handle h, int on);

/* Copy up to max per-family and per-phase counters to out (host array);
 * *count receives the number of entries with launches (phases count their
 * instances).  Waits for the recorded events. */
int lls_trace_read(lls_handle h, lls_trace_stat* out, int64_t max, int64_t* count);

/* Number of kernels this library has launched since it was loaded (all
 * handles and threads). */
int64_t lls_launch_count(void);

/* Number of device allocations (workspace and factor buffers growing) this
 * library has made since it was loaded.  A steady-state loop of solves of
 * shapes seen before makes none. */
int64_t lls_alloc_count(void);

/* Testing hook (failure injection on the host): the (after + 1)-th device
 * workspace allocation from now, in any handle, fails as if the device were
 * out of memory (the call returns LLS_ERR_NOMEM and the handle stays usable);
 * after = -1 turns the injection off.  Allocations inside the lls_k_* step
 * entry points are not covered. */
int lls_debug_fail_allocation(int64_t after);

/* Testing hook (failure detection without a GPU fault): a CTA of the
 * cooperative panel kernels waiting at their grid barrier, or a CTA of the
 * persistent batched factorization finding no ready task, gives up after
 * `polls` polls (default about 4 million, a few seconds) instead of
 * hanging; the kernel then exits and the call that launched it returns
 * LLS_ERR_TIMEOUT.  polls = 0 makes every wait that does not pass at once
 * run out; polls < 0 restores the default.  Applies to kernels launched
 * after the call, by every handle. */
int lls_debug_barrier_limit(int64_t polls);

/* Debug mode (guard words; for tests on small shapes).  With on = 1, every
 * device buffer the library allocates from then on (solver workspace,
 * factors, batched and serving workers; not the lls_k_* entry points'
 * temporaries) carries 512 bytes of a fixed pattern before and after it,
 * inside the same allocation.  After every kernel launch the library
 * synchronizes the device and checks every live buffer's guards, and checks
 * a buffer again when it is freed: a kernel that writes past either end of
 * its buffer is reported (reads are not).  Turning it on clears the report;
 * buffers allocated while it was off stay unguarded.  LLS_ERR_ARG unless on
 * is 0 or 1. */
int lls_debug_guard(int on);

/* Number of guard violations seen since lls_debug_guard(1); msg (host, may
 * be NULL) receives the first one: which guard, the buffer size, the offset
 * and the kernel after which it was seen. */
int64_t lls_debug_guard_report(char* msg, int64_t len);

/* Checks the guard machinery itself: writes one byte just past the end and
 * two bytes just before the start of a guarded buffer with cudaMemset (inside
 * its allocation) and returns LLS_OK iff both writes are reported with the
 * right offsets and an intact buffer is not. */
int lls_debug_guard_selftest(void);

/* Static text for a status code. */
const char* lls_status_string(int status);

/* Details of the last error on h: 1-based argument index (0 if none) and a
 * message copied into msg (NUL-terminated, up to len bytes). */
int lls_last_error(lls_handle h, int* arg_index, char* msg, int64_t len);

#ifdef __cplusplus
}
#endif
#endif /* LLS_H */
