// C ABI entry points (include/lls.h): argument validation, handle and
// factor management.  The numerical work is in solver.cu.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "lls.h"
#include "solver.h"

using lls::Handle;
using lls::Status;

namespace {

int finish(Handle* h, const Status& s) {
  if (h) {
    if (s.code != LLS_OK) {
      h->last_arg = s.arg;
      h->last_msg = s.msg;
    } else {
      h->last_arg = 0;
      h->last_msg.clear();
    }
  }
  return s.code;
}

Status arg_error(int idx, const char* what) { return lls::make_error(LLS_ERR_ARG, what, idx); }

Status check_options(const lls_options& o) {
  if (o.nb < 0 || o.nb > 128) return arg_error(2, "nb must be in 0..128 (0: tuned)");
  if (o.q < 0 || o.q > 4) return arg_error(2, "q must be in 0..4");
  if (o.precision < LLS_FP64 || o.precision > LLS_MIXED_BF16_TF32)
    return arg_error(2, "unknown precision mode");
  if (o.nullify != 0 && o.nullify != 1) return arg_error(2, "nullify must be 0 or 1");
  // The fast option keeps T_12.  Its x is the minimum-norm one only when the
  // sample resolves range(V_1) to FP64 accuracy (T_12 at rounding level, the
  // Remark after Fig. 4); a BF16 sample leaves T_12 of BF16 size.
  if (o.nullify == 0 && o.precision != LLS_FP64)
    return arg_error(2, "the fast option (nullify = 0) needs precision LLS_FP64: a BF16 sample "
                        "leaves T_12 of BF16 size, so x would not be the minimum-norm solution");
  if (o.explicit_v != 0 && o.explicit_v != 1) return arg_error(2, "explicit_v must be 0 or 1");
  if (o.max_refine < 0 || o.max_refine > 16) return arg_error(2, "max_refine must be in 0..16");
  if (!(o.refine_tol >= 0.0) || o.refine_tol == INFINITY)
    return arg_error(2, "refine_tol must be finite and >= 0");
  for (int i = 0; i < 2; ++i)
    if (o.reserved[i] != 0) return arg_error(2, "reserved option fields must be zero");
  return lls::ok_status();
}

// Validation of (A, m, n, lda) at argument positions ia, im, in, ilda.
Status check_matrix(const void* A, int64_t m, int64_t n, int64_t lda, int ia, int im, int in,
                    int ilda) {
  if (m < 0) return arg_error(im, "m < 0");
  if (n < 0) return arg_error(in, "n < 0");
  if (lda < (m > 1 ? m : 1)) return arg_error(ilda, "leading dimension < max(1, rows)");
  if (m > 0 && n > 0 && !A) return arg_error(ia, "NULL matrix pointer");
  if (m > 0 && n > (INT64_MAX / 8) / (lda > 0 ? lda : 1)) return arg_error(in, "size overflows");
  return lls::ok_status();
}

Status do_solve(Handle& h, const double* A, int64_t m, int64_t n, int64_t lda, const double* B,
                int64_t nrhs, int64_t ldb, double tol, double* X, int64_t ldx, int64_t* rank) {
  LLS_TRY(check_matrix(A, m, n, lda, 2, 3, 4, 5));
  LLS_TRY(check_matrix(B, m, nrhs, ldb, 6, 3, 7, 8));
  if (ldx < (n > 1 ? n : 1)) return arg_error(11, "ldx < max(1, n)");
  if (n > 0 && nrhs > 0 && !X) return arg_error(10, "NULL X");
  if (tol != tol) return arg_error(9, "tol is NaN");
  if (rank) *rank = 0;
  if (n == 0 || nrhs == 0) return lls::ok_status();
  if (m == 0) return lls::fill_zero(n, nrhs, X, ldx, h.stream);
  lls::Factor& f = h.scratch();
  Status fs = lls::factorize(h, f, A, m, n, lda, tol);
  if (!fs.ok()) return fs;
  if (rank) *rank = f.rank;
  Status ss = lls::solve_refined(h, f, A, lda, B, nrhs, ldb, X, ldx);
  if (!ss.ok()) return ss;
  return fs.code != LLS_OK ? fs : ss;  // LLS_WARN_RANK_NONPREFIX, else LLS_WARN_REFINE_NOCONV
}

}  // namespace

extern "C" {

int lls_default_options(lls_options* opt) {
  if (!opt) return LLS_ERR_ARG;
  std::memset(opt, 0, sizeof(*opt));
  opt->nb = 64;
  opt->q = 1;
  opt->precision = LLS_FP64;
  opt->nullify = 1;
  opt->seed = 2001;
  opt->refine_tol = 1e-12;
  return LLS_OK;
}

int lls_create(lls_handle* out, const lls_options* opt, void* cuda_stream) {
  if (!out) return LLS_ERR_ARG;
  *out = nullptr;
  lls_options o;
  lls_default_options(&o);
  if (opt) o = *opt;
  Status s = check_options(o);
  if (!s.ok()) return s.code;
  Handle* h = new (std::nothrow) Handle();
  if (!h) return LLS_ERR_NOMEM;
  h->opt = o;
  h->tune = std::make_shared<lls::TuneTable>();
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return LLS_ERR_CUDA;
  }
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return LLS_ERR_CUDA;
    }
    h->own_stream = true;
  }
  h->bind_workspace();
  *out = reinterpret_cast<lls_handle>(h);
  return LLS_OK;
}

int lls_destroy(lls_handle hh) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  lls::stop_pool(*h);
  cudaStreamSynchronize(h->stream);
  delete h;
  return LLS_OK;
}

int lls_set_options(lls_handle hh, const lls_options* opt) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  if (!opt) return finish(h, arg_error(2, "NULL options"));
  Status s = check_options(*opt);
  if (s.ok()) h->opt = *opt;
  return finish(h, s);
}

int lls_solve(lls_handle hh, const double* A, int64_t m, int64_t n, int64_t lda, const double* B,
              int64_t nrhs, int64_t ldb, double tol, double* X, int64_t ldx, int64_t* rank) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  lls::TraceGuard tg(*h);
  return finish(h, do_solve(*h, A, m, n, lda, B, nrhs, ldb, tol, X, ldx, rank));
}

int lls_solve_host(lls_handle hh, const double* A, int64_t m, int64_t n, int64_t lda,
                   const double* B, int64_t nrhs, int64_t ldb, double tol, double* X, int64_t ldx,
                   int64_t* rank) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  lls::TraceGuard tg(*h);
  Status s = check_matrix(A, m, n, lda, 2, 3, 4, 5);
  if (s.ok()) s = check_matrix(B, m, nrhs, ldb, 6, 3, 7, 8);
  if (s.ok() && ldx < (n > 1 ? n : 1)) s = arg_error(11, "ldx < max(1, n)");
  if (s.ok() && n > 0 && nrhs > 0 && !X) s = arg_error(10, "NULL X");
  if (!s.ok()) return finish(h, s);
  if (rank) *rank = 0;
  if (n == 0 || nrhs == 0) return finish(h, lls::ok_status());
  lls::DevBuf dA, dB, dX;
  const int64_t mm = m > 1 ? m : 1, nn = n > 1 ? n : 1;
  s = dA.reserve(sizeof(double) * (size_t)mm * n);
  if (s.ok()) s = dB.reserve(sizeof(double) * (size_t)mm * nrhs);
  if (s.ok()) s = dX.reserve(sizeof(double) * (size_t)nn * nrhs);
  if (!s.ok()) return finish(h, s);
  cudaStream_t st = h->stream;
  if (m > 0) {
    s = lls::cuda_status(cudaMemcpy2DAsync(dA.p, sizeof(double) * mm, A, sizeof(double) * lda,
                                           sizeof(double) * m, n, cudaMemcpyHostToDevice, st),
                         "copy A to device");
    if (s.ok())
      s = lls::cuda_status(cudaMemcpy2DAsync(dB.p, sizeof(double) * mm, B, sizeof(double) * ldb,
                                             sizeof(double) * m, nrhs, cudaMemcpyHostToDevice, st),
                           "copy B to device");
  }
  if (s.ok())
    s = do_solve(*h, dA.d(), m, n, mm, dB.d(), nrhs, mm, tol, dX.d(), nn, rank);
  if (s.ok()) {
    Status c = lls::cuda_status(cudaMemcpy2DAsync(X, sizeof(double) * ldx, dX.p, sizeof(double) * nn,
                                                  sizeof(double) * n, nrhs, cudaMemcpyDeviceToHost,
                                                  st),
                                "copy X to host");
    if (c.ok()) c = lls::cuda_status(cudaStreamSynchronize(st), "synchronize");
    if (!c.ok()) s = c;
  }
  return finish(h, s);
}

int lls_factor(lls_handle hh, const double* A, int64_t m, int64_t n, int64_t lda, double tol,
               int64_t* factor_id, int64_t* rank) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  lls::TraceGuard tg(*h);
  Status s = check_matrix(A, m, n, lda, 2, 3, 4, 5);
  if (s.ok() && !factor_id) s = arg_error(7, "NULL factor_id");
  if (s.ok() && tol != tol) s = arg_error(6, "tol is NaN");
  if (!s.ok()) return finish(h, s);
  std::unique_ptr<lls::Factor> f(new lls::Factor());
  s = lls::factorize(*h, *f, A, m, n, lda, tol, /*keep_a=*/true);
  if (!s.ok()) return finish(h, s);
  if (rank) *rank = f->rank;
  std::lock_guard<std::mutex> lock(h->factors_mu);
  int64_t id = h->next_factor++;
  h->factors[id] = std::move(f);
  *factor_id = id;
  return finish(h, s);
}

int lls_solve_factored(lls_handle hh, int64_t factor_id, const double* B, int64_t nrhs,
                       int64_t ldb, double* X, int64_t ldx) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  lls::TraceGuard tg(*h);
  std::shared_ptr<lls::Factor> fp;
  {
    std::lock_guard<std::mutex> lock(h->factors_mu);
    auto it = h->factors.find(factor_id);
    if (it != h->factors.end()) fp = it->second;
  }
  if (!fp) return finish(h, lls::make_error(LLS_ERR_NOT_FOUND, "unknown factor id", 2));
  lls::Factor& f = *fp;
  Status s = check_matrix(B, f.m, nrhs, ldb, 3, 2, 4, 5);
  if (s.ok() && ldx < (f.n > 1 ? f.n : 1)) s = arg_error(7, "ldx < max(1, n)");
  if (s.ok() && f.n > 0 && nrhs > 0 && !X) s = arg_error(6, "NULL X");
  if (s.ok()) s = lls::solve_refined(*h, f, nullptr, 0, B, nrhs, ldb, X, ldx);
  return finish(h, s);
}

int lls_factor_release(lls_handle hh, int64_t factor_id) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  std::shared_ptr<lls::Factor> keep;  // freed outside the lock
  {
    std::lock_guard<std::mutex> lock(h->factors_mu);
    auto it = h->factors.find(factor_id);
    if (it == h->factors.end())
      return finish(h, lls::make_error(LLS_ERR_NOT_FOUND, "unknown factor id", 2));
    keep = std::move(it->second);
    h->factors.erase(it);
  }
  cudaStreamSynchronize(h->stream);
  keep.reset();
  return finish(h, lls::ok_status());
}

int lls_factor_diag(lls_handle hh, int64_t factor_id, double* diag, int64_t len,
                    int64_t* rank_count) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  std::shared_ptr<lls::Factor> fp;
  {
    std::lock_guard<std::mutex> lock(h->factors_mu);
    auto it = h->factors.find(factor_id);
    if (it != h->factors.end()) fp = it->second;
  }
  if (!fp) return finish(h, lls::make_error(LLS_ERR_NOT_FOUND, "unknown factor id", 2));
  lls::Factor& f = *fp;
  int64_t mn = f.m < f.n ? f.m : f.n;
  if (len < mn || (mn > 0 && !diag)) return finish(h, arg_error(4, "diag buffer too short"));
  // |diag(T)| is the singular values written by the SVD step (before Nullify).
  Status s = lls::ok_status();
  size_t off = 0;
  for (size_t i = 0; i < f.ks.size() && s.ok(); ++i) {
    s = lls::cuda_status(cudaMemcpyAsync(diag + f.ks[i], f.sigma.d() + i * f.nb,
                                         sizeof(double) * f.bs[i], cudaMemcpyDeviceToHost,
                                         h->stream),
                         "copy diag");
    off += f.bs[i];
  }
  if (s.ok()) s = lls::cuda_status(cudaStreamSynchronize(h->stream), "synchronize");
  if (rank_count) *rank_count = f.rank_count;
  return finish(h, s);
}

int lls_factor_get(lls_handle hh, int64_t factor_id, int32_t which, double* dst, int64_t ld) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  std::shared_ptr<lls::Factor> fp;
  {
    std::lock_guard<std::mutex> lock(h->factors_mu);
    auto it = h->factors.find(factor_id);
    if (it != h->factors.end()) fp = it->second;
  }
  if (!fp) return finish(h, lls::make_error(LLS_ERR_NOT_FOUND, "unknown factor id", 2));
  lls::Factor& f = *fp;
  if (which != LLS_FACTOR_T && which != LLS_FACTOR_V)
    return finish(h, arg_error(3, "which must be LLS_FACTOR_T or LLS_FACTOR_V"));
  if (which == LLS_FACTOR_V && !f.has_v)
    return finish(h, arg_error(3, "V is kept only by factors made with explicit_v = 1"));
  const int64_t rows = which == LLS_FACTOR_T ? f.m : f.n, cols = f.n;
  if (ld < (rows > 1 ? rows : 1)) return finish(h, arg_error(5, "ld < max(1, rows)"));
  if (rows > 0 && cols > 0 && !dst) return finish(h, arg_error(4, "NULL dst"));
  Status s = which == LLS_FACTOR_T
                 ? lls::copy_upper_trapezoid(rows, cols, f.T.d(), f.ldt, dst, ld, h->stream)
                 : lls::copy_matrix(rows, cols, f.Vx.d(), cols > 1 ? cols : 1, dst, ld, h->stream);
  if (s.ok()) s = lls::cuda_status(cudaStreamSynchronize(h->stream), "synchronize");
  return finish(h, s);
}

int lls_refinement_info(lls_handle hh, int32_t* steps, double* correction) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  if (steps) *steps = h->refine_steps;
  if (correction) *correction = h->refine_corr;
  return LLS_OK;
}

const char* lls_status_string(int status) {
  switch (status) {
    case LLS_OK: return "ok";
    case LLS_PENDING: return "pending";
    case LLS_WARN_RANK_NONPREFIX: return "warning: a diagonal entry above tol follows one below";
    case LLS_WARN_REFINE_NOCONV: return "warning: refinement stopped above refine_tol";
    case LLS_ERR_ARG: return "invalid argument";
    case LLS_ERR_NOMEM: return "out of memory";
    case LLS_ERR_CUDA: return "CUDA error";
    case LLS_ERR_NONFINITE: return "NaN or Inf in the input";
    case LLS_ERR_SVD_NOCONV: return "block SVD did not converge";
    case LLS_ERR_TIMEOUT: return "device wait timed out";
    case LLS_ERR_NOT_FOUND: return "unknown factor or ticket";
    case LLS_ERR_CAPACITY: return "request exceeds the memory cap";
    default: return "unknown status";
  }
}

int lls_last_error(lls_handle hh, int* arg_index, char* msg, int64_t len) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  if (arg_index) *arg_index = h->last_arg;
  if (msg && len > 0) {
    std::strncpy(msg, h->last_msg.c_str(), (size_t)len - 1);
    msg[len - 1] = '\0';
  }
  return LLS_OK;
}

}  // extern "C"

namespace lls {
std::atomic<int64_t> g_fail_alloc_countdown{-1};
}  // namespace lls

extern "C" int lls_debug_barrier_limit(int64_t polls) {
  lls::g_barrier_spin_limit.store(polls < 0 ? lls::kBarrierSpinLimit : (long long)polls);
  return LLS_OK;
}

extern "C" int lls_debug_fail_allocation(int64_t after) {
  if (after < -1) return LLS_ERR_ARG;
  lls::g_fail_alloc_countdown.store(after < 0 ? -1 : after);
  return LLS_OK;
}
