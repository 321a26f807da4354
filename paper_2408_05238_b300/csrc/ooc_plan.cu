// Out-of-core planning: the host<->device panel traffic of a randUTV solve
// whose matrix lives in host memory and passes through a device cache of
// whole column panels (the paper's block cache, Sec. 3.4 variants v23c-v23e,
// with the GPU's memory in the role of main memory and host memory in the
// role of the disk).  Host code only: no CUDA call.
//
// The matrix T (m x n, column-major) is split into P = ceil(n / nb) column
// panels of nb columns (the last one narrower), each moved whole (all m
// rows).  The planned solve visits the panels in passes:
//
//   step i (k = i nb), trailing panels i..P-1:
//     sampling   Y = (A^T A)^q A^T G over A_BR: the first product A_j^T G
//                is taken during the previous step's update pass (for step 0
//                in a pass of its own); for q >= 1, q + 1 further passes
//                (W += A_j Y_j fused with the next Y_j = A_j^T W)
//     P pass     P = T(:, k:n) W_V, read
//     update     panel i first (right update, panel QR), then every j > i:
//                right and left update, and the next step's A_j^T G; the
//                panels are modified
//   after the loop, one pass over all panels (the block SVDs' V_s and U_s^T
//   updates, modified); with Nullify and 0 < r < n, per row block of C
//   (panel-aligned, bottom up): its own panel, then two passes over the
//   panels holding D = T(0:r, r:n) (read, then modified); the solve reads
//   panels 0..s-1 forward (U^T b) and the panels of T_11 backward (T_11^{-1}).
//
// Consecutive passes alternate direction so that the panels used last are
// used first again; the pass before an update runs backward, so the update
// (which must start with panel i) begins with the most recently used panel.
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
};

struct PassList {
  std::vector<Access> acc;
  int64_t passes = 0;
  bool forward = true;  // direction of the last pass added
  // Visits panels [lo, hi] in the given direction.
  void pass(int64_t lo, int64_t hi, bool fwd, bool write) {
    if (lo > hi) return;
    if (fwd) {
      for (int64_t j = lo; j <= hi; ++j) acc.push_back({j, write});
    } else {
      for (int64_t j = hi; j >= lo; --j) acc.push_back({j, write});
    }
    forward = fwd;
    ++passes;
  }
};

PassList build_accesses(int64_t m, int64_t n, int64_t nb, int q, int64_t r, bool nullify) {
  PassList pl;
  const int64_t P = (n + nb - 1) / nb;
  const int64_t steps = (std::min(m, n) + nb - 1) / nb;
  for (int64_t i = 0; i < steps; ++i) {
    const int64_t hi = P - 1;
    // Passes before the update: sampling (pass A_j^T G at step 0, then q + 1
    // for q >= 1) and the P pass; directions alternate backward from the P
    // pass, which runs backward.
    int64_t before = (i == 0 ? 1 : 0) + (q >= 1 ? q + 1 : 0) + 1;
    for (int64_t t = 0; t < before; ++t) {
      const bool fwd = ((before - 1 - t) % 2) == 1;  // last one (the P pass) backward
      pl.pass(i, hi, fwd, false);
    }
    pl.pass(i, hi, true, true);  // update: panel i first
  }
  if (steps == 0) return pl;  // m = 0 or n = 0: nothing is read
  pl.pass(0, P - 1, !pl.forward, true);  // block-SVD updates
  if (nullify && r > 0 && r < n) {
    const int64_t pr = r / nb;  // first panel holding columns of D
    const int64_t top = (r - 1) / nb;  // panel of C's last row block
    for (int64_t p = top; p >= 0; --p) {
      pl.acc.push_back({p, true});  // C_11 (and C_01 above it) of this row block
      ++pl.passes;
      pl.pass(pr, P - 1, !pl.forward, false);  // P = [C_01 | D_0] W
      pl.pass(pr, P - 1, !pl.forward, true);   // D_0 -= P_2 W^T
    }
  }
  if (r > 0) {
    pl.pass(0, steps - 1, true, false);        // U^T b
    pl.pass(0, (r - 1) / nb, false, false);    // T_11^{-1}
  }
  return pl;
}

}  // namespace
}  // namespace lls

namespace lls {
namespace {

// Runs the cache over an access list; panel j is `width(j)` columns of m rows.
template <class Width>
void simulate(const std::vector<Access>& acc, int64_t P, int64_t m, int64_t cache_panels,
              int32_t policy, Width width, lls_ooc_stats* out) {
  const int64_t N = (int64_t)acc.size();
  const int64_t INF = std::numeric_limits<int64_t>::max();
  // next use of the panel of each access
  std::vector<int64_t> next(N, INF), seen(P, INF);
  for (int64_t t = N - 1; t >= 0; --t) {
    next[t] = seen[acc[t].panel];
    seen[acc[t].panel] = t;
  }
  std::vector<int64_t> key(P, -1);  // resident panel: next use (FARTHEST) or last use (LRU)
  std::vector<char> resident(P, 0), dirty(P, 0);
  std::set<std::pair<int64_t, int64_t>> order;  // (key, panel) of the resident panels
  int64_t loads = 0, stores = 0, hits = 0, nres = 0;
  double load_bytes = 0.0, store_bytes = 0.0;
  for (int64_t t = 0; t < N; ++t) {
    const int64_t j = acc[t].panel;
    if (resident[j]) {
      ++hits;
      order.erase({key[j], j});
    } else {
      if (nres == cache_panels) {
        // FARTHEST: largest next use; LRU: smallest last use
        auto victim = policy == LLS_OOC_FARTHEST ? std::prev(order.end()) : order.begin();
        const int64_t v = victim->second;
        order.erase(victim);
        resident[v] = 0;
        --nres;
        if (dirty[v]) {
          ++stores;
          store_bytes += 8.0 * (double)m * (double)width(v);
          dirty[v] = 0;
        }
      }
      resident[j] = 1;
      ++nres;
      ++loads;
      load_bytes += 8.0 * (double)m * (double)width(j);
    }
    if (acc[t].write) dirty[j] = 1;
    key[j] = policy == LLS_OOC_FARTHEST ? next[t] : t;
    order.insert({key[j], j});
  }
  for (int64_t j = 0; j < P; ++j) {
    if (resident[j] && dirty[j]) {
      ++stores;
      store_bytes += 8.0 * (double)m * (double)width(j);
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

}  // namespace
}  // namespace lls

extern "C" int lls_ooc_plan(int64_t m, int64_t n, int32_t nb, int32_t q, int64_t rank,
                            int32_t nullify, int64_t cache_panels, int32_t policy,
                            lls_ooc_stats* out) {
  if (!out) return LLS_ERR_ARG;
  if (m < 0 || n < 0 || nb < 1 || q < 0 || q > 4 || rank < 0 || rank > std::min(m, n) ||
      (nullify != 0 && nullify != 1) || cache_panels < 1 ||
      (policy != LLS_OOC_FARTHEST && policy != LLS_OOC_LRU))
    return LLS_ERR_ARG;
  const int64_t P = (n + nb - 1) / nb;
  if (P > (int64_t)1 << 24) return LLS_ERR_ARG;  // the access list stays in memory
  lls::PassList pl = lls::build_accesses(m, n, nb, q, rank, nullify != 0);
  lls::simulate(pl.acc, P, m, cache_panels, policy,
                [&](int64_t j) { return std::min<int64_t>(nb, n - j * nb); }, out);
  out->passes = pl.passes;
  // Side traffic outside the panel cache, each written to host memory once
  // and read back once by the solve: every step's W_V (n' x b), and with
  // Nullify every row block's reflector panel ((bsz + n - r) x bsz).
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
  out->side_bytes = side;
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
    acc[(size_t)t] = {panels[t], writes ? writes[t] != 0 : false};
  }
  lls::simulate(acc, num_panels, rows, cache_panels, policy, [&](int64_t) { return cols; }, out);
  out->passes = 0;
  out->side_bytes = 0.0;
  return LLS_OK;
}
