// Batched solves and the serving queue (lls_solve_batched, lls_submit,
// lls_poll, lls_set_memory_cap, lls_set_workers).
//
// A handle owns a pool of worker handles.  Each worker has its own stream,
// its own workspace and one host thread, and runs whole requests
// (factorization and solve, or a solve with a resident factor) one after
// another; different workers' requests overlap on the device.  Requests wait
// in one FIFO queue and are admitted, in arrival order, when a worker is
// free and the estimated device memory of the admitted requests stays under
// the handle's cap (continuous batching: a request that arrives while others
// run starts as soon as a worker and memory free up).  Every kernel reduces
// in a fixed order, so a request's result does not depend on what runs
// beside it.
#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <thread>

#include "batched_factor.h"
#include "lls.h"
#include "solver.h"

namespace lls {

struct Ticket {
  lls_problem req;
  std::function<Status(Handle&)> job;  // set: run this on the worker instead of req
  int64_t bytes = 0;
  int status = LLS_PENDING;
  int err_arg = 0;
  std::string err_msg;  // the worker's message when status < 0
  bool done = false;
};

struct Handle::Pool {
  Handle* parent = nullptr;
  std::vector<std::unique_ptr<Handle>> workers;
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queue;
  std::map<int64_t, std::shared_ptr<Ticket>> tickets;
  int64_t next_ticket = 0;
  int64_t admitted_bytes = 0;
  int running = 0;
  bool stop = false;
};

Handle::Handle() = default;

Handle::~Handle() {
  stop_pool(*this);
  // Stream-ordered frees of the workspace before the stream goes away.
  for (DevBuf* b : workspace()) b->release();
  scratch_factor.reset();
  batch_view.reset();
  if (stream) cudaStreamSynchronize(stream);
  if (hstat) cudaFreeHost(hstat);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

namespace {

// Device memory one request holds while it runs (factor + workspace).
int64_t request_bytes(const lls_problem& p, const lls_options& opt) {
  int nb = opt.nb;
  if (nb <= 0) nb = 128;  // tuned block size: bound by the largest
  const int64_t rhs = std::max<int64_t>(p.nrhs, 1);
  const int64_t refine = opt.max_refine > 0 ? 8 * (int64_t)(p.m + p.n) * rhs : 0;
  if (p.factor_id >= 0) return (int64_t)(8 * (p.m + 2 * p.n) * rhs) + refine;
  int64_t mx = std::max(p.m, p.n);
  int64_t ws = 8 * (int64_t)mx * nb * 6 + 8 * (int64_t)(p.m + p.n) * rhs + refine;
  return (int64_t)factor_bytes(p.m, p.n, nb, opt.explicit_v != 0,
                               p.keep_factor && opt.max_refine > 0) +
         ws;
}

Status run_request(Handle& parent, Handle& w, lls_problem& p) {
  if (p.factor_id >= 0) {
    std::shared_ptr<Factor> f;
    {
      std::lock_guard<std::mutex> lock(parent.factors_mu);
      auto it = parent.factors.find(p.factor_id);
      if (it != parent.factors.end()) f = it->second;
    }
    if (!f) return make_error(LLS_ERR_NOT_FOUND, "unknown factor id");
    if (p.rank_out) *p.rank_out = f->rank;
    return solve_refined(w, *f, nullptr, 0, p.B, p.nrhs, p.ldb, p.X, p.ldx);
  }
  if (p.n == 0 || p.nrhs == 0) {
    if (p.rank_out) *p.rank_out = 0;
    return ok_status();
  }
  if (p.m == 0) {
    if (p.rank_out) *p.rank_out = 0;
    Status s = fill_zero(p.n, p.nrhs, p.X, p.ldx, w.stream);
    if (s.ok()) s = cuda_status(cudaStreamSynchronize(w.stream), "synchronize");
    return s;
  }
  std::shared_ptr<Factor> f;
  if (p.keep_factor) f = std::make_shared<Factor>();  // shared later: not stream-bound
  Factor& fr = p.keep_factor ? *f : w.scratch();
  Status fs = factorize(w, fr, p.A, p.m, p.n, p.lda, p.tol, p.keep_factor != 0);
  if (!fs.ok()) return fs;
  if (p.rank_out) *p.rank_out = fr.rank;
  Status ss = solve_refined(w, fr, p.A, p.lda, p.B, p.nrhs, p.ldb, p.X, p.ldx);
  if (!ss.ok()) return ss;
  if (p.keep_factor) {
    std::lock_guard<std::mutex> lock(parent.factors_mu);
    int64_t id = parent.next_factor++;
    parent.factors[id] = f;
    p.factor_id = id;
  }
  return fs.code != LLS_OK ? fs : ss;
}

void worker_loop(Handle::Pool* pool, int wi) {
  Handle& w = *pool->workers[wi];
  cudaSetDevice(w.device);
  for (;;) {
    std::shared_ptr<Ticket> t;
    {
      std::unique_lock<std::mutex> lock(pool->mu);
      pool->cv_work.wait(lock, [&] {
        if (pool->stop) return true;
        if (pool->queue.empty()) return false;
        auto& head = pool->tickets[pool->queue.front()];
        int64_t cap = pool->parent->mem_cap;
        return cap <= 0 || pool->running == 0 || pool->admitted_bytes + head->bytes <= cap;
      });
      if (pool->stop) return;
      t = pool->tickets[pool->queue.front()];
      pool->queue.pop_front();
      pool->admitted_bytes += t->bytes;
      ++pool->running;
    }
    w.opt = pool->parent->opt;
    w.tune = pool->parent->tune;
    Status s = t->job ? t->job(w) : run_request(*pool->parent, w, t->req);
    {
      std::lock_guard<std::mutex> lock(pool->mu);
      pool->admitted_bytes -= t->bytes;
      --pool->running;
      t->status = s.code;
      t->err_arg = s.arg;
      t->err_msg = s.msg;
      t->done = true;
    }
    pool->cv_done.notify_all();
    pool->cv_work.notify_all();
  }
}

Status ensure_pool(Handle& h) {
  if (h.pool) return ok_status();
  std::unique_ptr<Handle::Pool> pool(new Handle::Pool());
  pool->parent = &h;
  for (int i = 0; i < h.num_workers; ++i) {
    std::unique_ptr<Handle> w(new Handle());
    w->opt = h.opt;
    w->device = h.device;
    if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess)
      return make_error(LLS_ERR_CUDA, "cannot create a worker stream");
    w->own_stream = true;
    w->shares_device = true;
    w->bind_workspace();
    pool->workers.push_back(std::move(w));
  }
  Handle::Pool* raw = pool.get();
  h.pool = std::move(pool);
  for (int i = 0; i < h.num_workers; ++i) raw->threads.emplace_back(worker_loop, raw, i);
  return ok_status();
}

int64_t enqueue(Handle& h, const lls_problem& req) {
  Handle::Pool& pool = *h.pool;
  auto t = std::make_shared<Ticket>();
  t->req = req;
  t->bytes = request_bytes(req, h.opt);
  int64_t id;
  {
    std::lock_guard<std::mutex> lock(pool.mu);
    id = pool.next_ticket++;
    pool.tickets[id] = t;
    pool.queue.push_back(id);
  }
  pool.cv_work.notify_all();
  return id;
}

int64_t enqueue_job(Handle& h, std::function<Status(Handle&)> job) {
  Handle::Pool& pool = *h.pool;
  auto t = std::make_shared<Ticket>();
  std::memset(&t->req, 0, sizeof(t->req));
  t->job = std::move(job);
  int64_t id;
  {
    std::lock_guard<std::mutex> lock(pool.mu);
    id = pool.next_ticket++;
    pool.tickets[id] = t;
    pool.queue.push_back(id);
  }
  pool.cv_work.notify_all();
  return id;
}

// ---------------------------------------------------------------------------
// lls_solve_batched in one persistent launch (batched_factor.cu): every
// problem's factors and workspace live in one arena of the handle; the
// kernel runs the step loop and block SVDs of all problems, then the worker
// pool decides each rank, runs Nullify and the solve on views of the arena.
// ---------------------------------------------------------------------------
constexpr int64_t kPbMaxDim = 16384;

// Offsets (bytes) of one problem's buffers in the arena.
struct PBLayout {
  int nb, q, steps;
  size_t T, WV, TV, TU, US, VS, R, tauV, tauU, sigma, G, W, P, P2, Q, Q2, S;
};

}  // namespace

bool persistent_eligible(Handle& h, int64_t count, const lls_problem* probs, std::string* why) {
  if (!batched_factor_available()) return (*why = "persistent kernel not in this build"), false;
  if (h.opt.precision != LLS_FP64) return (*why = "the persistent path is FP64"), false;
  if (h.opt.explicit_v) return (*why = "the persistent path keeps V implicit"), false;
  if (count > INT32_MAX / 2) return (*why = "too many problems"), false;
  for (int64_t i = 0; i < count; ++i) {
    const lls_problem& p = probs[i];
    int nb = 0, q = 0;
    effective_nb_q(h.opt, h.tune.get(), p.m, p.n, &nb, &q);
    if (!p.A || p.m < 1 || p.n < 1 || p.m > kPbMaxDim || p.n > kPbMaxDim || nb > kPbMaxNb ||
        p.lda < p.m || p.nrhs < 0)
      return (*why = "problem " + std::to_string(i) + " is outside the persistent path's range " +
                     "(1 <= m, n <= 16384, nb <= 64)"),
             false;
  }
  return true;
}

namespace {

Status solve_batched_persistent(Handle& h, int64_t count, lls_problem* probs,
                                std::vector<int>& status) {
  cudaStream_t st = h.stream;
  // largest first: the scheduler prefers problems in this order
  std::vector<int64_t> order(count);
  for (int64_t i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    const lls_problem &pa = probs[a], &pb = probs[b];
    return (double)pa.m * pa.n * std::min(pa.m, pa.n) > (double)pb.m * pb.n * std::min(pb.m, pb.n);
  });
  std::vector<PBLayout> lay(count);
  size_t total = 0;
  auto take = [&](size_t doubles) {
    const size_t o = total;
    total += (std::max<size_t>(doubles, 1) * sizeof(double) + 255) / 256 * 256;
    return o;
  };
  for (int64_t k = 0; k < count; ++k) {
    const lls_problem& p = probs[order[k]];
    PBLayout& L = lay[k];
    effective_nb_q(h.opt, h.tune.get(), p.m, p.n, &L.nb, &L.q);
    L.steps = (int)ceil_div(std::min(p.m, p.n), L.nb);
    const size_t blk = (size_t)L.nb * L.nb * L.steps, vec = (size_t)L.nb * L.steps;
    L.T = take((size_t)p.m * p.n);
    L.WV = take((size_t)p.n * p.n);
    L.TV = take(blk);
    L.TU = take(blk);
    L.US = take(blk);
    L.VS = take(blk);
    L.R = take(blk);
    L.tauV = take(vec);
    L.tauU = take(vec);
    L.sigma = take(vec);
    L.G = take((size_t)p.m * L.nb);
    L.W = take((size_t)p.m * L.nb);
    L.P = take((size_t)p.m * L.nb);
    L.P2 = take((size_t)p.m * L.nb);
    L.Q = take((size_t)L.nb * p.n);
    L.Q2 = take((size_t)L.nb * p.n);
    L.S = take((size_t)L.nb * L.nb);
  }
  LLS_TRY(h.batch_arena.reserve(total));
  // scheduler state and flags: problems, state, done, flags, finished, err
  const size_t off_probs = 0, off_state = (sizeof(PBProblem) * count + 255) / 256 * 256;
  const size_t off_done = off_state + 8 * (size_t)count;
  const size_t off_flags = off_done + 4 * (size_t)count;
  const size_t off_tail = off_flags + 8 * (size_t)count;
  const size_t meta_bytes = off_tail + 16;
  LLS_TRY(h.batch_meta.reserve(meta_bytes));
  char* arena = h.batch_arena.as<char>();
  char* meta = h.batch_meta.as<char>();
  int* flags = reinterpret_cast<int*>(meta + off_flags);
  std::vector<PBProblem> pp(count);
  for (int64_t k = 0; k < count; ++k) {
    const lls_problem& p = probs[order[k]];
    const PBLayout& L = lay[k];
    PBProblem& q = pp[k];
    auto at = [&](size_t off) { return reinterpret_cast<double*>(arena + off); };
    q.m = (int)p.m;
    q.n = (int)p.n;
    q.nb = L.nb;
    q.q = L.q;
    q.steps = L.steps;
    q.nphases = pb_num_phases(q.m, q.n, q.nb, q.q);
    q.seed = h.opt.seed;
    q.A = p.A;
    q.lda = p.lda;
    q.T = at(L.T);
    q.ldt = p.m;
    q.WV = at(L.WV);
    q.ldw = p.n;
    q.TV = at(L.TV);
    q.TU = at(L.TU);
    q.US = at(L.US);
    q.VS = at(L.VS);
    q.Rblk = at(L.R);
    q.tauV = at(L.tauV);
    q.tauU = at(L.tauU);
    q.sigma = at(L.sigma);
    q.G = at(L.G);
    q.W = at(L.W);
    q.P = at(L.P);
    q.P2 = at(L.P2);
    q.Q = at(L.Q);
    q.Q2 = at(L.Q2);
    q.S = at(L.S);
    q.flags = flags + 2 * k;
  }
  LLS_CUDA(cudaMemcpyAsync(meta + off_probs, pp.data(), sizeof(PBProblem) * count,
                           cudaMemcpyHostToDevice, st));
  LLS_CUDA(cudaMemsetAsync(meta + off_state, 0, meta_bytes - off_state, st));
  PBArgs args;
  args.count = (int)count;
  args.probs = reinterpret_cast<const PBProblem*>(meta + off_probs);
  args.state = reinterpret_cast<unsigned long long*>(meta + off_state);
  args.done = reinterpret_cast<unsigned int*>(meta + off_done);
  args.finished = reinterpret_cast<unsigned int*>(meta + off_tail);
  args.err = reinterpret_cast<int*>(meta + off_tail + 8);
  args.poll_limit = g_barrier_spin_limit.load(std::memory_order_relaxed);
  {
    TraceGuard tg(h);
    LLS_TRY(batched_factor_launch(args, st));
  }
  std::vector<int> hflags(2 * (size_t)count + 4);
  LLS_CUDA(cudaMemcpyAsync(hflags.data(), flags, (off_tail + 16 - off_flags), cudaMemcpyDeviceToHost,
                           st));
  LLS_CUDA(cudaStreamSynchronize(st));
  const int sched_err = hflags[2 * count + 2];
  // per problem: the rank, Nullify and the solve on the worker pool
  std::vector<int64_t> ids(count, -1);
  for (int64_t k = 0; k < count; ++k) {
    const int64_t j = order[k];
    if (sched_err) status[j] = LLS_ERR_TIMEOUT;
    else if (hflags[2 * k]) status[j] = LLS_ERR_NONFINITE;
    else if (hflags[2 * k + 1]) status[j] = LLS_ERR_SVD_NOCONV;
    if (status[j] != LLS_PENDING) continue;
    const lls_problem p = probs[j];
    const PBLayout L = lay[k];
    ids[k] = enqueue_job(h, [p, L, arena](Handle& w) -> Status {
      Factor& f = w.view();
      auto at = [&](size_t off) { return arena + off; };
      const size_t blk = sizeof(double) * L.nb * L.nb * L.steps, vec = sizeof(double) * L.nb * L.steps;
      f.m = p.m;
      f.n = p.n;
      f.ldt = p.m;
      f.nb = L.nb;
      f.q = L.q;
      f.precision = LLS_FP64;
      f.nullified = false;
      f.has_v = f.has_a = false;
      f.ks.clear();
      f.bs.clear();
      f.rz.clear();
      f.rank = f.rank_count = 0;
      for (int64_t k0 = 0; k0 < std::min(p.m, p.n); k0 += L.nb) {
        f.ks.push_back(k0);
        f.bs.push_back(std::min<int64_t>(L.nb, std::min(p.m - k0, p.n - k0)));
      }
      f.T.borrow(at(L.T), sizeof(double) * p.m * p.n);
      f.WV.borrow(at(L.WV), sizeof(double) * p.n * p.n);
      f.TV.borrow(at(L.TV), blk);
      f.TU.borrow(at(L.TU), blk);
      f.US.borrow(at(L.US), blk);
      f.VS.borrow(at(L.VS), blk);
      f.Rblk.borrow(at(L.R), blk);
      f.tauV.borrow(at(L.tauV), vec);
      f.tauU.borrow(at(L.tauU), vec);
      f.sigma.borrow(at(L.sigma), vec);
      LLS_TRY(w.dstat.reserve(sizeof(DevStatus)));
      LLS_CUDA(cudaMemsetAsync(w.dstat.p, 0, sizeof(DevStatus), w.stream));
      Status fs = finish_factorization(w, f, p.tol);
      if (!fs.ok()) return fs;
      if (p.rank_out) *p.rank_out = f.rank;
      Status ss = solve_refined(w, f, p.A, p.lda, p.B, p.nrhs, p.ldb, p.X, p.ldx);
      if (!ss.ok()) return ss;
      return fs.code != LLS_OK ? fs : ss;
    });
  }
  Handle::Pool& pool = *h.pool;
  std::unique_lock<std::mutex> lock(pool.mu);
  for (int64_t k = 0; k < count; ++k) {
    if (ids[k] < 0) continue;
    auto t = pool.tickets[ids[k]];
    pool.cv_done.wait(lock, [&] { return t->done; });
    status[order[k]] = t->status;
    if (t->status < 0 && h.last_msg.empty()) {
      h.last_arg = t->err_arg;
      h.last_msg = "problem " + std::to_string(order[k]) + ": " + t->err_msg;
    }
    pool.tickets.erase(ids[k]);
  }
  return ok_status();
}

}  // namespace

bool pool_busy(Handle& h) {
  if (!h.pool) return false;
  std::lock_guard<std::mutex> lock(h.pool->mu);
  return h.pool->running > 0 || !h.pool->queue.empty();
}

void stop_pool(Handle& h) {
  if (!h.pool) return;
  {
    std::lock_guard<std::mutex> lock(h.pool->mu);
    h.pool->stop = true;
  }
  h.pool->cv_work.notify_all();
  for (auto& th : h.pool->threads) th.join();
  h.pool.reset();
}

}  // namespace lls

using lls::Handle;

extern "C" {

int lls_set_workers(lls_handle hh, int workers) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || workers < 1 || workers > 64) return LLS_ERR_ARG;
  lls::stop_pool(*h);
  h->num_workers = workers;
  return LLS_OK;
}

int lls_set_batched_mode(lls_handle hh, int mode) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || mode < LLS_BATCHED_AUTO || mode > LLS_BATCHED_PERSISTENT) return LLS_ERR_ARG;
  h->batched_mode = mode;
  return LLS_OK;
}

int lls_solve_batched(lls_handle hh, int64_t count, lls_problem* problems) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || count < 0 || (count > 0 && !problems)) return LLS_ERR_ARG;
  if (count == 0) return LLS_OK;
  lls::Status ps = lls::ensure_pool(*h);
  if (!ps.ok()) return ps.code;
  if (h->batched_mode != LLS_BATCHED_WORKERS) {
    std::string why;
    if (lls::persistent_eligible(*h, count, problems, &why)) {
      std::vector<int> status(count, LLS_PENDING);
      h->last_arg = 0;
      h->last_msg.clear();
      lls::Status s = lls::solve_batched_persistent(*h, count, problems, status);
      if (!s.ok()) {
        h->last_arg = s.arg;
        h->last_msg = s.msg;
        return s.code;
      }
      int first = LLS_OK;
      for (int64_t i = 0; i < count; ++i) {
        problems[i].status = status[i];
        problems[i].factor_id = -1;
        if (first == LLS_OK && status[i] < 0) first = status[i];
      }
      return first;
    }
    if (h->batched_mode == LLS_BATCHED_PERSISTENT) {
      h->last_arg = 3;
      h->last_msg = why;
      return LLS_ERR_ARG;
    }
  }
  // Largest problems first, so the pool's tail is made of short requests.
  std::vector<int64_t> order(count);
  for (int64_t i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    const lls_problem &pa = problems[a], &pb = problems[b];
    return (double)pa.m * pa.n * std::min(pa.m, pa.n) > (double)pb.m * pb.n * std::min(pb.m, pb.n);
  });
  std::vector<int64_t> ids(count);
  for (int64_t k = 0; k < count; ++k) {
    lls_problem p = problems[order[k]];
    p.factor_id = -1;
    p.keep_factor = 0;
    ids[k] = lls::enqueue(*h, p);
  }
  Handle::Pool& pool = *h->pool;
  int first = LLS_OK;
  std::unique_lock<std::mutex> lock(pool.mu);
  for (int64_t k = 0; k < count; ++k) {
    auto t = pool.tickets[ids[k]];
    pool.cv_done.wait(lock, [&] { return t->done; });
    problems[order[k]].status = t->status;
    problems[order[k]].factor_id = -1;
    if (first == LLS_OK && t->status < 0) {
      first = t->status;
      h->last_arg = t->err_arg;
      h->last_msg = "problem " + std::to_string(order[k]) + ": " + t->err_msg;
    }
    pool.tickets.erase(ids[k]);
  }
  return first;
}

int lls_set_memory_cap(lls_handle hh, int64_t bytes) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || bytes < 0) return LLS_ERR_ARG;
  h->mem_cap = bytes;
  if (h->pool) h->pool->cv_work.notify_all();
  return LLS_OK;
}

int lls_submit(lls_handle hh, const lls_problem* req, int64_t* ticket) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !req || !ticket) return LLS_ERR_ARG;
  if (req->m < 0 || req->n < 0 || req->nrhs < 0 || req->ldb < std::max<int64_t>(1, req->m) ||
      req->ldx < std::max<int64_t>(1, req->n) ||
      (req->factor_id < 0 && req->lda < std::max<int64_t>(1, req->m)))
    return LLS_ERR_ARG;
  if (h->mem_cap > 0 && lls::request_bytes(*req, h->opt) > h->mem_cap) return LLS_ERR_CAPACITY;
  lls::Status ps = lls::ensure_pool(*h);
  if (!ps.ok()) return ps.code;
  *ticket = lls::enqueue(*h, *req);
  return LLS_OK;
}

int lls_poll(lls_handle hh, int64_t ticket, int* status) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !status) return LLS_ERR_ARG;
  if (!h->pool) return LLS_ERR_NOT_FOUND;
  std::lock_guard<std::mutex> lock(h->pool->mu);
  auto it = h->pool->tickets.find(ticket);
  if (it == h->pool->tickets.end()) return LLS_ERR_NOT_FOUND;
  if (!it->second->done) {
    *status = LLS_PENDING;
    return LLS_OK;
  }
  *status = it->second->status;
  if (*status < 0) {
    h->last_arg = it->second->err_arg;
    h->last_msg = "ticket " + std::to_string(ticket) + ": " + it->second->err_msg;
  }
  h->pool->tickets.erase(it);
  return LLS_OK;
}

int lls_cancel(lls_handle hh, int64_t ticket) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  if (!h->pool) return LLS_ERR_NOT_FOUND;
  Handle::Pool& pool = *h->pool;
  {
    std::lock_guard<std::mutex> lock(pool.mu);
    auto q = std::find(pool.queue.begin(), pool.queue.end(), ticket);
    if (q == pool.queue.end()) return LLS_ERR_NOT_FOUND;  // unknown, started or finished
    pool.queue.erase(q);
    pool.tickets.erase(ticket);
  }
  pool.cv_work.notify_all();  // the head of the queue may have changed
  return LLS_OK;
}

int lls_ticket_factor(lls_handle hh, int64_t ticket, int64_t* factor_id) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !factor_id) return LLS_ERR_ARG;
  if (!h->pool) return LLS_ERR_NOT_FOUND;
  std::lock_guard<std::mutex> lock(h->pool->mu);
  auto it = h->pool->tickets.find(ticket);
  if (it == h->pool->tickets.end()) return LLS_ERR_NOT_FOUND;
  if (!it->second->done) return LLS_PENDING;
  *factor_id = it->second->req.factor_id;
  return LLS_OK;
}

}  // extern "C"
