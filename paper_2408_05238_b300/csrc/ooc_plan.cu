// Out-of-core planning: the schedule and the host<->device panel traffic of
// a randUTV solve whose matrix lives in host memory and passes through a
// device cache of whole column panels (the paper's block cache, Sec. 3.5
// variants v23c-v23e, with the GPU's memory in the role of main memory and
// host memory in the role of the disk).  Host code only: no CUDA call.
//
// The matrix T (m x n, column-major) is split into P = ceil(n / nb) column
// panels of nb columns (the last one narrower), each moved whole (all m
// rows).  The planned solve visits the panels in passes (access kinds of
// lls.h in brackets):
//
//   step i (k = i nb), trailing panels i..P-1:
//     sampling   Y = (A^T A)^q A^T G over A_BR.  Y_j = A_j^T G is taken in
//                the previous step's update pass (step 0: a pass of its own
//                [SAMPLE_ATG]); for q >= 1, q + 1 passes: W = sum_j A_j Y_j
//                [SAMPLE_AY], q - 1 passes Y_j = A_j^T W with the next
//                W += A_j Y_j in the same visit [SAMPLE_ATW_AY], and
//                Y_j = A_j^T W [SAMPLE_ATW]
//     P pass     P = T(:, k:n) W_V [PRODUCT_TWV]
//     update     panel i first (right update, panel QR), then every j > i:
//                right and left update and the next step's A_j^T G [UPDATE];
//                the panels are modified
//   after the loop one pass over all panels: the block SVDs' V_s and U_s^T
//   updates [SVD], modified.
//   Nullify (0 < r < n), per panel-aligned row block p of T(0:r, 0:r) from
//   the bottom (block rows j0 = p nb .. min(r, j0 + nb)); D = T(0:r, r:n)
//   lies in the panels r / nb .. P-1:
//     first block only: a pass gathering its rows of D [NULL_GATHER]
//     read pass: panel p first (its reflectors are formed from C_11 and the
//                gathered D_1; C_01's part of P = [C_01 | D_0] W), then the D
//                panels (D_0's part) [NULL_READ]
//     write pass: the D panels (D_0 -= P_2 W_bot^T, D_1 = 0, the next block's
//                rows of D gathered), then panel p (C_01 and C_11) [NULL_WRITE]
//   solve: panels 0..s-1 forward (U^T b from each step's W_U) [SOLVE_UTB],
//   then the panels of T_11 backward (T_11^{-1}) [SOLVE_TRSM].
//   Modified panels still on the device are written back at the end [FLUSH].
//
// Consecutive passes alternate direction where the method allows, so that
// the panels used last are used first again; the pass before an update runs
// backward, so the update (which must start with panel i) begins with the
// most recently used panel.
//
// Eviction: LLS_OOC_FARTHEST evicts the resident panel whose next use is
// latest (the paper's "latest in the future to be used" policy, i.e.
// Belady's MIN, possible because the whole access list is known before the
// solve starts); LLS_OOC_LRU evicts the least recently used one.  A modified
// panel is written back when it is evicted and at the end.
#include <algorithm>
#include <cstdint>
#include <limits>
#include <set>
#include <vector>

#include "lls.h"

namespace lls {
namespace {

struct Access {
  int64_t panel;
  bool write;
  int32_t kind = -1;  // LLS_OOC_K_*
  int64_t step = -1;  // step of Fig. 2, row block of Nullify, or -1
  int64_t pass = -1;  // index of the pass the access belongs to
};

struct PassList {
  std::vector<Access> acc;
  int64_t passes = 0;
  bool forward = true;  // direction of the last pass added
  // An access of the pass being built (its index is the number of passes
  // completed so far).
  void one(int64_t j, bool write, int32_t kind, int64_t step) {
    acc.push_back({j, write, kind, step, passes});
  }
  // Visits panels [lo, hi] in the given direction as one pass.
  void pass(int64_t lo, int64_t hi, bool fwd, bool write, int32_t kind, int64_t step) {
    if (lo > hi) return;
    if (fwd) {
      for (int64_t j = lo; j <= hi; ++j) one(j, write, kind, step);
    } else {
      for (int64_t j = hi; j >= lo; --j) one(j, write, kind, step);
    }
    forward = fwd;
    ++passes;
  }
};

// The factorization: the step loop and the block-SVD pass.
void add_factor_accesses(PassList& pl, int64_t m, int64_t n, int64_t nb, int q) {
  const int64_t P = (n + nb - 1) / nb;
  const int64_t steps = (std::min(m, n) + nb - 1) / nb;
  for (int64_t i = 0; i < steps; ++i) {
    const int64_t hi = P - 1;
    // Passes before the update, in order; directions alternate backward from
    // the P pass, which runs backward.
    std::vector<int32_t> kinds;
    if (i == 0) kinds.push_back(LLS_OOC_K_SAMPLE_ATG);
    if (q >= 1) {
      kinds.push_back(LLS_OOC_K_SAMPLE_AY);
      for (int t = 1; t < q; ++t) kinds.push_back(LLS_OOC_K_SAMPLE_ATW_AY);
      kinds.push_back(LLS_OOC_K_SAMPLE_ATW);
    }
    kinds.push_back(LLS_OOC_K_PRODUCT_TWV);
    const int64_t before = (int64_t)kinds.size();
    for (int64_t t = 0; t < before; ++t) {
      const bool fwd = ((before - 1 - t) % 2) == 1;  // the last one (the P pass) backward
      pl.pass(i, hi, fwd, false, kinds[(size_t)t], i);
    }
    pl.pass(i, hi, true, true, LLS_OOC_K_UPDATE, i);  // panel i first
  }
  if (steps == 0) return;  // m = 0 or n = 0: nothing is read
  pl.pass(0, P - 1, !pl.forward, true, LLS_OOC_K_SVD, -1);
}

// Nullify (with rank r) and the solve's reads.
void add_finish_accesses(PassList& pl, int64_t m, int64_t n, int64_t nb, int64_t r,
                         bool nullify) {
  const int64_t P = (n + nb - 1) / nb;
  const int64_t steps = (std::min(m, n) + nb - 1) / nb;
  if (steps == 0) return;
  if (nullify && r > 0 && r < n) {
    const int64_t pr = r / nb;         // first panel holding columns of D
    const int64_t top = (r - 1) / nb;  // panel of the last row block of C
    pl.pass(pr, P - 1, !pl.forward, false, LLS_OOC_K_NULL_GATHER, top);
    for (int64_t p = top; p >= 0; --p) {
      // read pass: panel p first, then the D panels other than p
      const bool fwd = !pl.forward;
      pl.one(p, false, LLS_OOC_K_NULL_READ, p);
      const int64_t lo = std::max(pr, p + 1);
      if (fwd) {
        for (int64_t j = lo; j <= P - 1; ++j) pl.one(j, false, LLS_OOC_K_NULL_READ, p);
      } else {
        for (int64_t j = P - 1; j >= lo; --j) pl.one(j, false, LLS_OOC_K_NULL_READ, p);
      }
      ++pl.passes;
      // write pass: the D panels other than p in the opposite order, then p
      if (fwd) {
        for (int64_t j = P - 1; j >= lo; --j) pl.one(j, true, LLS_OOC_K_NULL_WRITE, p);
      } else {
        for (int64_t j = lo; j <= P - 1; ++j) pl.one(j, true, LLS_OOC_K_NULL_WRITE, p);
      }
      pl.one(p, true, LLS_OOC_K_NULL_WRITE, p);
      ++pl.passes;
      pl.forward = !fwd;
    }
  }
  if (r > 0) {
    pl.pass(0, steps - 1, true, false, LLS_OOC_K_SOLVE_UTB, -1);
    pl.pass(0, (r - 1) / nb, false, false, LLS_OOC_K_SOLVE_TRSM, -1);
  }
}

PassList build_accesses(int64_t m, int64_t n, int64_t nb, int q, int64_t r, bool nullify) {
  PassList pl;
  add_factor_accesses(pl, m, n, nb, q);
  add_finish_accesses(pl, m, n, nb, r, nullify);
  return pl;
}

}  // namespace
}  // namespace lls

namespace lls {
namespace {

// Runs the cache over an access list (panel j is width(j) columns of m
// rows), counting traffic into *out and, if actions is not NULL, recording
// one action per access plus one FLUSH per modified panel left at the end.
template <class Width>
void simulate(const std::vector<Access>& acc, int64_t P, int64_t m, int64_t cache_panels,
              int32_t policy, Width width, lls_ooc_stats* out,
              std::vector<lls_ooc_action>* actions) {
  const int64_t N = (int64_t)acc.size();
  const int64_t INF = std::numeric_limits<int64_t>::max();
  // next use of the panel of each access
  std::vector<int64_t> next(N, INF), seen(P, INF);
  for (int64_t t = N - 1; t >= 0; --t) {
    next[t] = seen[acc[t].panel];
    seen[acc[t].panel] = t;
  }
  std::vector<int64_t> key(P, -1);   // resident panel: next use (FARTHEST) or last use (LRU)
  std::vector<int64_t> slot(P, -1);  // cache slot of a resident panel
  std::vector<char> dirty(P, 0);
  std::vector<int64_t> free_slots;
  for (int64_t s = std::min<int64_t>(cache_panels, P) - 1; s >= 0; --s) free_slots.push_back(s);
  std::set<std::pair<int64_t, int64_t>> order;  // (key, panel) of the resident panels
  int64_t loads = 0, stores = 0, hits = 0;
  double load_bytes = 0.0, store_bytes = 0.0;
  for (int64_t t = 0; t < N; ++t) {
    const int64_t j = acc[t].panel;
    lls_ooc_action a{acc[t].kind, acc[t].write ? 1 : 0, acc[t].step, acc[t].pass, j, -1, -1, 0, 0};
    if (slot[j] >= 0) {
      ++hits;
      order.erase({key[j], j});
    } else {
      if (free_slots.empty()) {
        // FARTHEST: largest next use; LRU: smallest last use
        auto victim = policy == LLS_OOC_FARTHEST ? std::prev(order.end()) : order.begin();
        const int64_t v = victim->second;
        order.erase(victim);
        a.evict = v;
        if (dirty[v]) {
          ++stores;
          store_bytes += 8.0 * (double)m * (double)width(v);
          dirty[v] = 0;
          a.store = 1;
        }
        free_slots.push_back(slot[v]);
        slot[v] = -1;
      }
      slot[j] = free_slots.back();
      free_slots.pop_back();
      ++loads;
      load_bytes += 8.0 * (double)m * (double)width(j);
      a.load = 1;
    }
    a.slot = slot[j];
    if (acc[t].write) dirty[j] = 1;
    key[j] = policy == LLS_OOC_FARTHEST ? next[t] : t;
    order.insert({key[j], j});
    if (actions) actions->push_back(a);
  }
  for (int64_t j = 0; j < P; ++j) {
    if (slot[j] >= 0 && dirty[j]) {
      ++stores;
      store_bytes += 8.0 * (double)m * (double)width(j);
      if (actions) actions->push_back({LLS_OOC_K_FLUSH, 0, -1, -1, j, slot[j], j, 1, 0});
    }
  }
  out->panels = P;
  out->accesses = N;
  out->hits = hits;
  out->loads = loads;
  out->stores = stores;
  out->load_bytes = load_bytes;
  out->store_bytes = store_bytes;
}

int check_plan_args(int64_t m, int64_t n, int32_t nb, int32_t q, int64_t rank, int32_t nullify,
                    int64_t cache_panels, int32_t policy) {
  if (m < 0 || n < 0 || nb < 1 || q < 0 || q > 4 || rank < 0 || rank > std::min(m, n) ||
      (nullify != 0 && nullify != 1) || cache_panels < 1 ||
      (policy != LLS_OOC_FARTHEST && policy != LLS_OOC_LRU))
    return LLS_ERR_ARG;
  if ((n + nb - 1) / nb > (int64_t)1 << 24) return LLS_ERR_ARG;  // the access list stays in memory
  return LLS_OK;
}

// Side traffic outside the panel cache, each written to host memory once
// and read back once by the solve: every step's W_V (n' x b), and with
// Nullify every row block's reflector panel ((bsz + n - r) x bsz).
double side_bytes(int64_t m, int64_t n, int64_t nb, int64_t rank, bool nullify) {
  double side = 0.0;
  const int64_t steps = (std::min(m, n) + nb - 1) / nb;
  for (int64_t i = 0; i < steps; ++i) {
    const int64_t k = i * nb, b = std::min<int64_t>(nb, std::min(m - k, n - k));
    side += 2.0 * 8.0 * (double)(n - k) * b;
  }
  if (nullify && rank > 0 && rank < n) {
    for (int64_t p = (rank - 1) / nb; p >= 0; --p) {
      const int64_t bsz = std::min<int64_t>(rank, (p + 1) * nb) - p * nb;
      side += 2.0 * 8.0 * (double)(bsz + n - rank) * bsz;
    }
  }
  return side;
}

}  // namespace
}  // namespace lls

namespace lls {

std::vector<lls_ooc_action> ooc_schedule_phase(int64_t m, int64_t n, int64_t nb, int q,
                                               int64_t r, bool nullify, int64_t cache_panels,
                                               int32_t policy, int phase) {
  PassList pl;
  if (phase != 2) add_factor_accesses(pl, m, n, nb, q);
  if (phase != 1) add_finish_accesses(pl, m, n, nb, r, nullify);
  std::vector<lls_ooc_action> acts;
  lls_ooc_stats st{};
  const int64_t P = (n + nb - 1) / nb;
  simulate(pl.acc, P, m, cache_panels, policy,
           [&](int64_t j) { return std::min<int64_t>(nb, n - j * nb); }, &st, &acts);
  return acts;
}

}  // namespace lls

extern "C" int lls_ooc_plan(int64_t m, int64_t n, int32_t nb, int32_t q, int64_t rank,
                            int32_t nullify, int64_t cache_panels, int32_t policy,
                            lls_ooc_stats* out) {
  if (!out) return LLS_ERR_ARG;
  int e = lls::check_plan_args(m, n, nb, q, rank, nullify, cache_panels, policy);
  if (e != LLS_OK) return e;
  const int64_t P = (n + nb - 1) / nb;
  lls::PassList pl = lls::build_accesses(m, n, nb, q, rank, nullify != 0);
  lls::simulate(pl.acc, P, m, cache_panels, policy,
                [&](int64_t j) { return std::min<int64_t>(nb, n - j * nb); }, out, nullptr);
  out->passes = pl.passes;
  out->side_bytes = lls::side_bytes(m, n, nb, rank, nullify != 0);
  return LLS_OK;
}

extern "C" int lls_ooc_schedule(int64_t m, int64_t n, int32_t nb, int32_t q, int64_t rank,
                                int32_t nullify, int64_t cache_panels, int32_t policy,
                                int32_t phase, lls_ooc_action* actions, int64_t max_actions,
                                int64_t* count) {
  if (!count || max_actions < 0 || (max_actions > 0 && !actions) || phase < 0 || phase > 2)
    return LLS_ERR_ARG;
  int e = lls::check_plan_args(m, n, nb, q, rank, nullify, cache_panels, policy);
  if (e != LLS_OK) return e;
  std::vector<lls_ooc_action> acts =
      lls::ooc_schedule_phase(m, n, nb, q, rank, nullify != 0, cache_panels, policy, phase);
  *count = (int64_t)acts.size();
  if (!actions) return LLS_OK;
  if (max_actions < (int64_t)acts.size()) return LLS_ERR_CAPACITY;
  std::copy(acts.begin(), acts.end(), actions);
  return LLS_OK;
}

extern "C" int lls_ooc_simulate(const int64_t* panels, const int8_t* writes, int64_t count,
                                int64_t num_panels, int64_t rows, int64_t cols,
                                int64_t cache_panels, int32_t policy, lls_ooc_stats* out) {
  if (!out || count < 0 || (count > 0 && !panels) || num_panels < 1 || rows < 0 || cols < 0 ||
      cache_panels < 1 || (policy != LLS_OOC_FARTHEST && policy != LLS_OOC_LRU))
    return LLS_ERR_ARG;
  std::vector<lls::Access> acc((size_t)count);
  for (int64_t t = 0; t < count; ++t) {
    if (panels[t] < 0 || panels[t] >= num_panels) return LLS_ERR_ARG;
    acc[(size_t)t] = {panels[t], writes ? writes[t] != 0 : false, -1, -1, -1};
  }
  lls::simulate(acc, num_panels, rows, cache_panels, policy, [&](int64_t) { return cols; }, out,
                nullptr);
  out->passes = 0;
  out->side_bytes = 0.0;
  return LLS_OK;
}
