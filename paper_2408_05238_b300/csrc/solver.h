// Host driver of the solver: handle, resident factors and the step loop.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "lls.h"
#include "trace.h"

namespace lls {

// Allocation-failure injection for tests (lls_debug_fail_allocation): while
// >= 0, each workspace allocation decrements it and the one that finds it
// at 0 fails as if the device were out of memory.
extern std::atomic<int64_t> g_fail_alloc_countdown;
inline bool injected_alloc_failure() {
  int64_t c = g_fail_alloc_countdown.load(std::memory_order_relaxed);
  while (c >= 0) {
    if (g_fail_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 0;
  }
  return false;
}

// Owning device buffer (with guard words while lls_debug_guard is on).
//
// A buffer bound to a stream (bind) is only ever used by work on that
// stream: it is allocated and freed stream-ordered (cudaMallocAsync /
// cudaFreeAsync), so growing it never waits for other streams.  An unbound
// buffer may be used from any stream (resident factors shared by the
// worker pool): freeing it first waits for the whole device.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  bool guarded = false;
  cudaStream_t stream = nullptr;
  bool ordered = false;
  bool borrowed = false;  // a view into memory owned elsewhere (never freed here)
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  // Only while empty.
  void bind(cudaStream_t s) {
    stream = s;
    ordered = true;
  }
  // Points the buffer at `n` bytes owned by someone else (a batch arena).
  void borrow(void* ptr, size_t n) {
    release();
    p = ptr;
    bytes = n;
    borrowed = true;
  }
  void release() {
    if (borrowed) {
      p = nullptr;
      bytes = 0;
      borrowed = false;
      return;
    }
    if (p) {
      if (guarded) {
        cudaDeviceSynchronize();
        guard_free(p);
      } else if (ordered) {
        cudaFreeAsync(p, stream);  // after the work queued on `stream` that uses it
      } else {
        cudaDeviceSynchronize();  // work queued on any stream may still use it
        cudaFree(p);
      }
    }
    p = nullptr;
    bytes = 0;
    guarded = false;
  }
  // Grow to at least `need` bytes (contents are not kept).
  Status reserve(size_t need) {
    if (need <= bytes) return ok_status();
    if (borrowed) return make_error(LLS_ERR_NOMEM, "borrowed buffer smaller than needed");
    release();
    if (need == 0) return ok_status();
    if (injected_alloc_failure())
      return make_error(LLS_ERR_NOMEM, "device allocation of " + std::to_string(need) +
                                           " bytes failed (injected)");
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    if (g_guard_mode.load(std::memory_order_relaxed)) {
      Status s = guard_alloc(need, &p);
      if (!s.ok()) {
        p = nullptr;
        return s;
      }
      guarded = true;
      bytes = need;
      return ok_status();
    }
    cudaError_t e = ordered ? cudaMallocAsync(&p, need, stream) : cudaMalloc(&p, need);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return make_error(LLS_ERR_NOMEM, "device allocation of " + std::to_string(need) + " bytes failed");
    }
    bytes = need;
    return ok_status();
  }
  double* d() const { return static_cast<double*>(p); }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// Small device-side status block read back once per factorization.
struct DevStatus {
  int nonfinite;    // copy_check flag
  int barrier_err;  // grid-barrier timeout in a cooperative kernel
  int svd_status;   // LLS_ERR_SVD_NOCONV or 0
  int pad;
  int64_t rank[3];  // prefix, count, nan
  double tol;
};
static_assert(offsetof(DevStatus, barrier_err) == offsetof(DevStatus, nonfinite) + sizeof(int),
              "nonfinite and barrier_err are read back as one pair");

// A randUTV factorization A V = U T kept on the device.
//  T       m x n (ld = m): T's upper trapezoid; below the diagonal of each
//          step's block column the Householder vectors W_U (unit diagonal
//          implied).
//  WV      n x n (ld = n): step i's W_V in rows k..n-1, columns k..k+b-1.
//  TV, TU  per step nb x nb compact-WY factors (ld nb).
//  US, VS  per step nb x nb singular vectors of the diagonal block (ld nb).
//  Rz*     Nullify: per row block, the (bsz + n - r) x bsz reflector panel
//          M (Householder vectors below its diagonal) and its T factor.
//  Vx      with explicit_v: V itself (n x n, ld n), Nullify's reflectors
//          included.
//  A0      with max_refine > 0 on a factor kept for reuse: a copy of A
//          (m x n, ld m) for the refinement residual.
struct Factor {
  int64_t m = 0, n = 0, ldt = 0;
  int nb = 0, q = 0, precision = 0;
  bool nullified = false;
  bool has_v = false, has_a = false;
  DevBuf Vx, A0;
  std::vector<int64_t> ks, bs;
  DevBuf T, WV, TV, TU, US, VS, tauV, tauU, Rblk, sigma;
  int64_t rank = 0, rank_count = 0;
  double tol = 0.0;
  struct RzBlock {
    int64_t j0, bsz;
    size_t off_m, off_t, off_tau;
  };
  std::vector<RzBlock> rz;
  DevBuf RzM, RzT, RzTau;
  // Stream-ordered allocation for a factor that only one stream uses (a
  // handle's reusable scratch factor); only while empty.
  void bind(cudaStream_t s) {
    for (DevBuf* b : {&T, &WV, &TV, &TU, &US, &VS, &tauV, &tauU, &Rblk, &sigma, &RzM, &RzT, &RzTau,
                      &Vx, &A0})
      b->bind(s);
  }
  size_t bytes() const {
    return T.bytes + WV.bytes + TV.bytes + TU.bytes + US.bytes + VS.bytes + tauV.bytes +
           tauU.bytes + Rblk.bytes + sigma.bytes + RzM.bytes + RzT.bytes + RzTau.bytes +
           Vx.bytes + A0.bytes;
  }
};

// Block size and power-iteration count per (m, n) bucket (ceil(log2 m),
// ceil(log2 n)), filled by lls_autotune or lls_tuning_load and read when
// opt.nb == 0.  Shared by a handle and its workers.
struct TuneTable {
  std::mutex mu;
  std::map<std::pair<int, int>, std::pair<int, int>> entries;  // bucket -> (nb, q)
};
int tune_bucket(int64_t x);
// (nb, q) a factorization of an m x n matrix uses: opt.nb and opt.q, or,
// when opt.nb == 0, the table's entry for the bucket (nb 64, q 1 if none).
void effective_nb_q(const lls_options& opt, const TuneTable* table, int64_t m, int64_t n,
                    int* nb, int* q);

struct Handle {
  lls_options opt{};
  std::shared_ptr<TuneTable> tune;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // workspace
  DevBuf G, Wt, P, P2, Q, Q2, S, gemm_ws, panel_ws, bw, z, sp, sp2, xc;
  // iterative refinement: residual, correction, per-column norms; what the
  // last refined solve did (lls_refinement_info)
  DevBuf rr, dd, nrm;
  // the minimum-norm refinement of the TF32 modes: n x nrhs products and
  // the least-squares solution of its first stage
  DevBuf rs, z2, dinv;  // dinv: inverses of T_11's 64 x 64 diagonal blocks
  DevBuf sbat;          // a replay's batched singular-vector block products
  int refine_steps = 0;
  double refine_corr = 0.0;
  bool in_refine = false;  // solves inside the refinement trace as phase:refine only
  bool shares_device = false;  // a worker of a pool: other streams run panels meanwhile
  int bf16_scale_extra = 0;    // BF16 sample scaling: log2 of sqrt(m n), set at step 0
  DevBuf dstat;           // DevStatus
  // mixed precision sampling: bf16 copies of A_BR and A_BR^T, bf16 sketch /
  // product, fp32 product, tensor-core split-K partials, scalars
  DevBuf G16, A16, A16t, Z16, F32, tc_ws, mixed_misc;
  // workspace of the tensor-core update GEMMs (exact-slice or TF32 split)
  DevBuf oz_ws;
  DevStatus* hstat = nullptr;  // pinned host mirror
  // lls_solve reuses one factor object between calls of the same shape
  std::unique_ptr<Factor> scratch_factor;
  // batched solves: a factor whose T, W_V and per-step blocks are views into
  // the parent's batch arena (its own Nullify buffers grow on this stream)
  std::unique_ptr<Factor> batch_view;
  // lls_solve_batched: the persistent launch's arena (factors and workspace
  // of every problem) and its scheduler state; how the batch runs
  DevBuf batch_arena, batch_meta;
  int batched_mode = 0;  // LLS_BATCHED_AUTO / _WORKERS / _PERSISTENT
  // resident factors, shared with the worker pool (guarded by factors_mu)
  std::map<int64_t, std::shared_ptr<Factor>> factors;
  int64_t next_factor = 0;
  std::mutex factors_mu;
  // tracing
  std::unique_ptr<Tracer> tracer;
  bool trace_on = false;
  // errors
  int last_arg = 0;
  std::string last_msg;
  // batched solves and serving: a pool of worker handles, each with its own
  // stream, workspace and host thread (serving.cu)
  int64_t mem_cap = 0;
  int num_workers = 4;
  struct Pool;
  std::unique_ptr<Pool> pool;
  Handle();  // both defined where Pool is complete (serving.cu)
  ~Handle();
  // Every workspace buffer above (all used on `stream` only).
  std::vector<DevBuf*> workspace() {
    return {&G,  &Wt, &P,  &P2,  &Q,   &Q2,  &S,   &gemm_ws, &panel_ws,   &bw,   &z,   &sp,   &sp2,
            &xc, &rr, &dd, &nrm, &dstat, &G16, &A16, &A16t,  &Z16,        &F32,  &tc_ws, &mixed_misc,
            &oz_ws, &rs, &z2, &dinv, &sbat, &batch_arena, &batch_meta};
  }
  // Binds the workspace to `stream` (call once the stream is set).
  void bind_workspace() {
    for (DevBuf* b : workspace()) b->bind(stream);
  }
  // The handle's reusable factor for lls_solve / batched problems.
  Factor& scratch() {
    if (!scratch_factor) {
      scratch_factor.reset(new Factor());
      scratch_factor->bind(stream);
    }
    return *scratch_factor;
  }
  Factor& view() {
    if (!batch_view) {
      batch_view.reset(new Factor());
      batch_view->bind(stream);
    }
    return *batch_view;
  }
};

// Makes h's tracer the active one on this thread for the duration of a call.
struct TraceGuard {
  Tracer* prev;
  explicit TraceGuard(Handle& h) : prev(g_tracer) {
    g_tracer = (h.trace_on && h.tracer) ? h.tracer.get() : nullptr;
  }
  ~TraceGuard() { g_tracer = prev; }
};

// keep_a: with opt.max_refine > 0, keep a copy of A in the factor so that
// later solves with it can refine.
Status factorize(Handle& h, Factor& f, const double* A, int64_t m, int64_t n, int64_t lda,
                 double tol, bool keep_a = false);
Status solve_factored(Handle& h, Factor& f, const double* B, int64_t nrhs, int64_t ldb, double* X,
                      int64_t ldx);
// solve_factored, then opt.max_refine refinement steps x <- x + P (b - A x)
// with A (ld lda), or f's own copy when A is NULL; no refinement when
// max_refine = 0 or neither is there.  Records the steps in h.
Status solve_refined(Handle& h, Factor& f, const double* A, int64_t lda, const double* B,
                     int64_t nrhs, int64_t ldb, double* X, int64_t ldx);
// Compute_rank and Nullify (steps a8-a9) on a factor whose step loop and
// block SVDs are done (f.T, WV, the per-step blocks, ks, bs filled): reads
// the handle's device status (which must be cleared before the factor's
// kernels ran), decides the rank against tol and annihilates T_12.
Status finish_factorization(Handle& h, Factor& f, double tol);
// The solve's replays of the stored factors on nrhs columns, in place:
// c (m rows) <- U^T c, w (m rows) <- U w, z (n rows) <- V^T z, and
// z (n rows) <- V z where rows kz.. of z are zero.
Status apply_ut(Handle& h, Factor& f, double* c, int64_t ldc, int64_t nrhs);
Status apply_u(Handle& h, Factor& f, double* w, int64_t ldw, int64_t nrhs);
Status apply_vt(Handle& h, Factor& f, double* z, int64_t ldz, int64_t nrhs);
Status apply_v(Handle& h, Factor& f, double* z, int64_t ldz, int64_t nrhs, int64_t kz);
// Device bytes a factorization of m x n (and a solve with nrhs) will hold.
size_t factor_bytes(int64_t m, int64_t n, int nb, bool explicit_v = false, bool keep_a = false);

// Whether lls_solve_batched can run these problems in one persistent launch
// with the handle's options (serving.cu); *why says why not.
bool persistent_eligible(Handle& h, int64_t count, const lls_problem* probs, std::string* why);
// Stops and joins the worker pool (serving.cu); queued requests are dropped.
void stop_pool(Handle& h);
// True while the handle's worker pool has requests queued or running.
bool pool_busy(Handle& h);

Status jacobi_svd_batched(int count, int b, int b_last, const double* R, int64_t ldr,
                          int64_t strideR, double* sigma, int64_t strideS, double* U, int64_t ldu,
                          int64_t strideU, double* V, int64_t ldv, int64_t strideV, int* status,
                          cudaStream_t st);

// Mixed precision sampling (sampling_bf16.cu): Y (n' x b, ld ldy) =
// (A^T A)^q A^T G with A = the m' x n' block at A (ld lda), products in
// BF16 on tensor cores with FP32 accumulation, results stored as FP64.
Status sample_bf16(Handle& h, const double* A, int64_t lda, int64_t mp, int64_t np, int64_t b,
                   int q, uint64_t seed, int64_t step, double* Y, int64_t ldy);

}  // namespace lls
