// Batched solves and the request queue (lls_solve_batched, lls_submit,
// lls_poll, lls_set_memory_cap).
#include <deque>

#include "lls.h"
#include "solver.h"

namespace lls {

struct Handle::Ticket {
  lls_problem req;
  int status = LLS_PENDING;
  bool done = false;
};

namespace {

Status run_one(Handle& h, lls_problem& p) {
  if (p.factor_id >= 0) {
    auto it = h.factors.find(p.factor_id);
    if (it == h.factors.end()) return make_error(LLS_ERR_NOT_FOUND, "unknown factor id");
    Factor& f = *it->second;
    if (p.rank_out) *p.rank_out = f.rank;
    return solve_factored(h, f, p.B, p.nrhs, p.ldb, p.X, p.ldx);
  }
  std::unique_ptr<Factor> f(new Factor());
  Status fs = factorize(h, *f, p.A, p.m, p.n, p.lda, p.tol);
  if (!fs.ok()) return fs;
  if (p.rank_out) *p.rank_out = f->rank;
  Status ss = solve_factored(h, *f, p.B, p.nrhs, p.ldb, p.X, p.ldx);
  if (!ss.ok()) return ss;
  if (p.keep_factor) {
    int64_t id = h.next_factor++;
    h.factors[id] = std::move(f);
    p.factor_id = id;
  }
  return fs;
}

}  // namespace
}  // namespace lls

using lls::Handle;

extern "C" {

int lls_solve_batched(lls_handle hh, int64_t count, lls_problem* problems) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || count < 0 || (count > 0 && !problems)) return LLS_ERR_ARG;
  lls::TraceGuard tg(*h);
  int first = LLS_OK;
  for (int64_t i = 0; i < count; ++i) {
    lls_problem& p = problems[i];
    p.factor_id = -1;
    lls::Status s = lls::run_one(*h, p);
    p.status = s.code;
    if (first == LLS_OK && s.code < 0) first = s.code;
  }
  return first;
}

int lls_set_memory_cap(lls_handle hh, int64_t bytes) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || bytes < 0) return LLS_ERR_ARG;
  h->mem_cap = bytes;
  return LLS_OK;
}

int lls_submit(lls_handle hh, const lls_problem* req, int64_t* ticket) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !req || !ticket) return LLS_ERR_ARG;
  if (h->mem_cap > 0 && req->factor_id < 0 &&
      (int64_t)lls::factor_bytes(req->m, req->n, h->opt.nb) > h->mem_cap)
    return LLS_ERR_CAPACITY;
  auto t = std::make_shared<Handle::Ticket>();
  t->req = *req;
  int64_t id = h->next_ticket++;
  h->tickets[id] = t;
  *ticket = id;
  return LLS_OK;
}

int lls_poll(lls_handle hh, int64_t ticket, int* status) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !status) return LLS_ERR_ARG;
  auto it = h->tickets.find(ticket);
  if (it == h->tickets.end()) return LLS_ERR_NOT_FOUND;
  lls::TraceGuard tg(*h);
  // run queued requests in arrival order up to this one
  for (auto& kv : h->tickets) {
    if (kv.second->done) continue;
    lls::Status s = lls::run_one(*h, kv.second->req);
    kv.second->status = s.code;
    kv.second->done = true;
    if (kv.first == ticket) break;
  }
  *status = it->second->done ? it->second->status : LLS_PENDING;
  if (it->second->done) h->tickets.erase(it);
  return LLS_OK;
}

}  // extern "C"
