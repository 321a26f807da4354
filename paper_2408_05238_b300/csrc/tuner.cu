// Autotuning of the block size n_b and the power-iteration count q
// (lls_autotune, lls_tuning_lookup / save / load).
//
// The randUTV loop (Fig. 2) leaves n_b and q to the user.  n_b trades the
// number of sequential steps (panels, block SVDs) against the size of each
// product; q trades sampling work against how well the sample captures the
// dominant subspace (the Remark after Fig. 2).  The tuner checks each
// candidate's answer on one synthetic matrix of the bucket's shape and times
// it on a batch of copies solved together (lls_solve_batched), the way
// batched and served work runs, keeping the fastest candidate that still
// reaches the reference answer.
#include <cerrno>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "batched_factor.h"
#include "lls.h"
#include "solver.h"

namespace lls {

int tune_bucket(int64_t x) {
  int b = 0;
  while (b < 62 && ((int64_t)1 << b) < x) ++b;
  return b;
}

void effective_nb_q(const lls_options& opt, const TuneTable* table, int64_t m, int64_t n,
                    int* nb, int* q) {
  *nb = opt.nb;
  *q = opt.q;
  if (opt.nb != 0) return;
  *nb = 64;
  *q = 1;
  if (!table) return;
  std::lock_guard<std::mutex> lock(const_cast<TuneTable*>(table)->mu);
  auto it = table->entries.find({tune_bucket(m), tune_bucket(n)});
  if (it != table->entries.end()) {
    *nb = it->second.first;
    *q = it->second.second;
  }
}

namespace {

// X(:, j) *= 10^(-4 j / (r - 1)): singular values of X Y spread over four decades.
__global__ void decay_cols_kernel(int64_t m, int64_t r, double* X, int64_t ldx) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * r) return;
  const int64_t i = idx % m, j = idx / m;
  const double t = r > 1 ? (double)j / (double)(r - 1) : 0.0;
  X[i + j * ldx] *= exp10(-4.0 * t);
}

struct DevMem {
  void* p = nullptr;
  ~DevMem() {
    if (p) cudaFree(p);
  }
};

}  // namespace
}  // namespace lls

using lls::Handle;
using lls::Status;

extern "C" {

int lls_autotune(lls_handle hh, int64_t m, int64_t n, int32_t trials, int32_t* nb_out,
                 int32_t* q_out) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || m < 1 || n < 1 || trials < 1 || m > (1LL << 20) || n > (1LL << 20))
    return LLS_ERR_ARG;
  // the sweep changes the handle's options while it runs: not with requests in flight
  if (lls::pool_busy(*h)) {
    h->last_arg = 0;
    h->last_msg = "lls_autotune: the handle has batched or served requests in flight";
    return LLS_ERR_ARG;
  }
  if (!h->tune) h->tune = std::make_shared<lls::TuneTable>();
  cudaStream_t st = h->stream;
  const int64_t r = std::max<int64_t>(1, std::min(m, n) / 2);
  lls::DevMem X, Y, A, B, Xo, Xb, ws;
  if (cudaMalloc(&X.p, 8 * (size_t)m * r) != cudaSuccess ||
      cudaMalloc(&Y.p, 8 * (size_t)r * n) != cudaSuccess ||
      cudaMalloc(&A.p, 8 * (size_t)m * n) != cudaSuccess ||
      cudaMalloc(&B.p, 8 * (size_t)m) != cudaSuccess ||
      cudaMalloc(&Xo.p, 8 * (size_t)n) != cudaSuccess ||
      cudaMalloc(&Xb.p, 8 * (size_t)n * trials) != cudaSuccess) {
    cudaGetLastError();
    return LLS_ERR_NOMEM;
  }
  const uint64_t seed = 0x5EED7A11ull;
  Status s = lls::launch_sketch(seed, 0, m, r, (double*)X.p, m, st);
  if (s.ok()) s = lls::launch_sketch(seed, 1, r, n, (double*)Y.p, r, st);
  if (s.ok()) s = lls::launch_sketch(seed, 2, m, 1, (double*)B.p, m, st);
  if (s.ok()) {
    lls::decay_cols_kernel<<<(unsigned)lls::ceil_div(m * r, 256), 256, 0, st>>>(m, r,
                                                                               (double*)X.p, m);
    s = lls::cuda_status(cudaGetLastError(), "decay_cols_kernel");
    lls::g_launches.fetch_add(1, std::memory_order_relaxed);
    if (lls::g_guard_mode.load(std::memory_order_relaxed)) lls::guard_after_launch("decay_cols_kernel");
  }
  const size_t wsb = lls::gemm_scratch_bytes(m, n, r);
  if (s.ok() && wsb && cudaMalloc(&ws.p, wsb) != cudaSuccess) s = lls::make_error(LLS_ERR_NOMEM, "tuner");
  if (s.ok())
    s = lls::gemm(false, false, lls::kDense, lls::kDense, m, n, r, 1.0, (const double*)X.p, m,
                  (const double*)Y.p, r, 0.0, (double*)A.p, m, lls::Scratch{ws.p, wsb}, st);
  if (s.ok()) s = lls::cuda_status(cudaStreamSynchronize(st), "tuner inputs");
  if (!s.ok()) return s.code;

  const lls_options saved = h->opt;
  auto run = [&](int nb, int q, int64_t* rank, std::vector<double>* x) -> int {
    h->opt.nb = nb;
    h->opt.q = q;
    int code = lls_solve(hh, (const double*)A.p, m, n, m, (const double*)B.p, 1, m, -1.0,
                         (double*)Xo.p, n, rank);
    if (code < 0) return code;
    if (x) {
      x->resize((size_t)n);
      if (cudaMemcpy(x->data(), Xo.p, 8 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return LLS_ERR_CUDA;
    }
    return LLS_OK;
  };
  // timing: `trials` copies solved together by lls_solve_batched, so each
  // candidate is timed under the concurrency batched and served work runs
  // with (the persistent launch, or the worker pool)
  std::vector<lls_problem> batch((size_t)trials);
  for (int t = 0; t < trials; ++t) {
    lls_problem& p = batch[(size_t)t];
    std::memset(&p, 0, sizeof(p));
    p.A = (const double*)A.p;
    p.m = m;
    p.n = n;
    p.lda = m;
    p.B = (const double*)B.p;
    p.nrhs = 1;
    p.ldb = m;
    p.tol = -1.0;
    p.X = (double*)Xb.p + (size_t)t * n;
    p.ldx = n;
    p.factor_id = -1;
  }
  auto run_batch = [&](int nb, int q) -> int {
    h->opt.nb = nb;
    h->opt.q = q;
    return lls_solve_batched(hh, trials, batch.data());
  };
  // n_b above the persistent launch's limit only where the batch runs on workers
  std::string why;
  h->opt.nb = lls::kPbMaxNb;
  const bool persistent = h->batched_mode != LLS_BATCHED_WORKERS &&
                          lls::persistent_eligible(*h, trials, batch.data(), &why);
  h->opt = saved;
  // reference: the smallest block and the most power iterations
  int64_t rank_ref = -1;
  std::vector<double> x_ref, x;
  int code = run(32, 2, &rank_ref, &x_ref);
  double ref_norm = 0.0;
  for (double v : x_ref) ref_norm += v * v;
  ref_norm = std::sqrt(ref_norm);
  int best_nb = 32, best_q = 2;
  double best_t = 1e300;
  const int nbs[3] = {32, 64, 128};
  for (int a = 0; a < 3 && code >= 0; ++a) {
    const int nb = nbs[a];
    if (nb > 32 && nb > std::min(m, n)) continue;
    if (persistent && nb > lls::kPbMaxNb) continue;
    for (int q = 0; q <= 2 && code >= 0; ++q) {
      int64_t rk = -1;
      code = run(nb, q, &rk, &x);  // accuracy check
      if (code < 0) break;
      double d = 0.0;
      for (int64_t i = 0; i < n; ++i) d += (x[i] - x_ref[i]) * (x[i] - x_ref[i]);
      if (rk != rank_ref || !(std::sqrt(d) <= 1e-9 * ref_norm)) continue;
      code = run_batch(nb, q);  // warm-up (workspace)
      if (code < 0) break;
      const auto t0 = std::chrono::steady_clock::now();
      code = run_batch(nb, q);
      const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (code >= 0 && dt < best_t) {
        best_t = dt;
        best_nb = nb;
        best_q = q;
      }
    }
  }
  h->opt = saved;
  if (code < 0) return code;
  {
    std::lock_guard<std::mutex> lock(h->tune->mu);
    h->tune->entries[{lls::tune_bucket(m), lls::tune_bucket(n)}] = {best_nb, best_q};
  }
  if (nb_out) *nb_out = best_nb;
  if (q_out) *q_out = best_q;
  return LLS_OK;
}

int lls_tuning_lookup(lls_handle hh, int64_t m, int64_t n, int32_t* nb, int32_t* q) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || m < 0 || n < 0 || !nb || !q) return LLS_ERR_ARG;
  lls_options o = h->opt;
  o.nb = 0;  // what a tuned solve would use
  int b = 0, qq = 0;
  lls::effective_nb_q(o, h->tune.get(), m, n, &b, &qq);
  *nb = b;
  *q = qq;
  return LLS_OK;
}

int lls_tuning_save(lls_handle hh, const char* path) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !path) return LLS_ERR_ARG;
  FILE* f = std::fopen(path, "w");
  if (!f) return LLS_ERR_ARG;
  std::fprintf(f, "# lls tuning table: ceil(log2 m) ceil(log2 n) nb q\n");
  if (h->tune) {
    std::lock_guard<std::mutex> lock(h->tune->mu);
    for (const auto& e : h->tune->entries)
      std::fprintf(f, "%d %d %d %d\n", e.first.first, e.first.second, e.second.first,
                   e.second.second);
  }
  const bool ok = std::fclose(f) == 0;
  return ok ? LLS_OK : LLS_ERR_ARG;
}

int lls_tuning_load(lls_handle hh, const char* path) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !path) return LLS_ERR_ARG;
  FILE* f = std::fopen(path, "r");
  if (!f) return LLS_ERR_ARG;
  if (!h->tune) h->tune = std::make_shared<lls::TuneTable>();
  char line[256];
  int bad = 0;
  std::vector<std::pair<std::pair<int, int>, std::pair<int, int>>> rows;
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    int a, b, nb, q;
    if (std::sscanf(line, "%d %d %d %d", &a, &b, &nb, &q) != 4 || a < 0 || a > 62 || b < 0 ||
        b > 62 || nb < 1 || nb > 128 || q < 0 || q > 4) {
      bad = 1;
      break;
    }
    rows.push_back({{a, b}, {nb, q}});
  }
  std::fclose(f);
  if (bad) return LLS_ERR_ARG;
  std::lock_guard<std::mutex> lock(h->tune->mu);
  for (const auto& r : rows) h->tune->entries[r.first] = r.second;
  return LLS_OK;
}

}  // extern "C"
