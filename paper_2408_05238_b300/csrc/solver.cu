// Host driver: randUTV (Fig. 2), Compute_rank and Nullify (Fig. 3), and the
// solve x = V (T_tl^{-1} (U^T b)) of Fig. 4, chained from the launchers of
// the other translation units on the handle's stream.
//
// Differences from the paper's formulation (same mathematics):
//  * U is never formed, V only on request (explicit_v).  Each step keeps its
//    reflectors (W_U below the diagonal of T, W_V in a side buffer), their
//    compact-WY factors and the diagonal block's singular vectors; U^T b and,
//    without an explicit V, V y are applied from them (the paper's v23t
//    variant applies U to B on the fly, Sec. 3.5).
//  * The right update of step i runs over all m rows of columns k..n-1
//    (Fig. 2 prints only the A_BR block; the rows above must change too for
//    A V = U T to hold).
//  * The diagonal-block SVD and its two updates A_01 <- A_01 V_SVD and
//    A_12 <- U_SVD^T A_12 are taken off the step loop.  Later steps never
//    read those blocks (the next sample only reads A_22), and the row update
//    commutes with the later right updates of the same rows, so all SVDs run
//    as one batched launch after the loop, then all column updates, then all
//    row updates.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <optional>
#include <vector>

#include "lls_kernels.h"
#include "oz_gemm.h"
#include "solver.h"
#include "tf32_gemm.h"

namespace lls {

namespace {

Scratch scratch_of(DevBuf& b) { return Scratch{b.p, b.bytes}; }

// Largest split-K scratch any GEMM of the step loop asks for.
size_t loop_gemm_scratch(int64_t m, int64_t n, int nb, int64_t max_nrhs) {
  size_t need = 0;
  for (int64_t k = 0; k < std::min(m, n); k += nb) {
    int64_t b = std::min<int64_t>(nb, std::min(m - k, n - k));
    int64_t mp = m - k, np = n - k;
    need = std::max(need, gemm_scratch_bytes(np, b, mp));      // A^T G, A^T W
    need = std::max(need, gemm_scratch_bytes(mp, b, np));      // A Y
    need = std::max(need, gemm_scratch_bytes(b, b, std::max(mp, np)));  // Gram
    need = std::max(need, gemm_scratch_bytes(m, b, np));       // T W_V
    need = std::max(need, gemm_scratch_bytes(b, np - b, mp));  // W_U^T T
    need = std::max(need, gemm_scratch_bytes(b, max_nrhs, mp));
    need = std::max(need, gemm_scratch_bytes(b, max_nrhs, np));
    need = std::max(need, gemm_scratch_bytes(b, b + n, n));
    need = std::max(need, gemm_scratch_bytes(n, b, n));
  }
  return need;
}

// Waits for the handle's stream and reports B's finiteness check (read
// through the handle's pinned status mirror: a copy into pageable memory
// would go through the driver's shared staging buffer).
Status read_nonfinite_flag(Handle& h, const DevStatus* ds) {
  if (!h.hstat) LLS_CUDA(cudaMallocHost((void**)&h.hstat, sizeof(DevStatus)));
  LLS_CUDA(cudaMemcpyAsync(&h.hstat->nonfinite, &ds->nonfinite, 2 * sizeof(int),
                           cudaMemcpyDeviceToHost, h.stream));  // nonfinite, barrier_err
  LLS_CUDA(cudaStreamSynchronize(h.stream));
  if (h.hstat->nonfinite) return make_error(LLS_ERR_NONFINITE, "B has a NaN or Inf entry", 6);
  if (h.hstat->barrier_err) return make_error(LLS_ERR_TIMEOUT, "a replay's grid barrier timed out");
  return ok_status();
}

}  // namespace

size_t factor_bytes(int64_t m, int64_t n, int nb, bool explicit_v, bool keep_a) {
  int64_t steps = ceil_div(std::min(m, n), nb);
  size_t blk = (size_t)nb * nb * sizeof(double);
  size_t b = (size_t)m * n * sizeof(double) + (size_t)n * n * sizeof(double);
  b += 5 * steps * blk + 3 * steps * nb * sizeof(double);
  // Nullify panels at worst (r ~ n/2): n/2 x (nb + n/2)
  b += (size_t)(n / 2 + nb) * (size_t)(n / 2 + nb) * sizeof(double);
  if (explicit_v) b += (size_t)n * n * sizeof(double);
  if (keep_a) b += (size_t)m * n * sizeof(double);
  return b;
}

// The GEMMs of a factorization on the handle's stream: FP64 (fgemm), the
// update products per the precision mode (xgemm: FP64, exact-slice or split
// TF32 on the tensor cores) and the Gram products of the T factors (ggemm:
// FP64-accurate in every mode -- the T factor decides whether I - W T W^T is
// orthogonal, and a TF32 Gram's FP32 sums of squares would leave it off by
// about 1e-6, so the TF32 modes take the exact-slice GEMM there).  Scratch
// is grown to each shape's plan first: the plan depends on the shape alone,
// so a result never depends on which handle (or worker) computed it or on
// what that handle ran before.
struct FactorGemms {
  Handle& h;
  cudaStream_t st;
  int nb;
  DevStatus* ds;
  bool oz;
  int tf_terms;
  FactorGemms(Handle& h_, int nb_)
      : h(h_), st(h_.stream), nb(nb_), ds(h_.dstat.as<DevStatus>()),
        oz(h_.opt.precision == LLS_MIXED_BF16),
        tf_terms(h_.opt.precision == LLS_MIXED_BF16_3xTF32 ? 3
                 : h_.opt.precision == LLS_MIXED_BF16_TF32 ? 1 : 0) {}
  bool tc() const { return oz || tf_terms > 0; }
  size_t tc_ws_bytes(int64_t mm, int64_t nn, int64_t kk) const {
    return oz ? oz_gemm_workspace_bytes(mm, nn, kk) : tf32_gemm_workspace_bytes(mm, nn, kk, tf_terms);
  }
  Status fgemm(bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t mm, int64_t nn, int64_t kk,
               double alpha, const double* Aa, int64_t lda_, const double* Bb, int64_t ldb_,
               double beta, double* Cc, int64_t ldc_) {
    LLS_TRY(h.gemm_ws.reserve(gemm_scratch_bytes(mm, nn, kk)));
    return gemm(ta, tb, ma, mb, mm, nn, kk, alpha, Aa, lda_, Bb, ldb_, beta, Cc, ldc_,
                scratch_of(h.gemm_ws), st);
  }
  Status xgemm(bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t mm, int64_t nn, int64_t kk,
               double alpha, const double* Aa, int64_t lda_, const double* Bb, int64_t ldb_,
               double beta, double* Cc, int64_t ldc_) {
    if (oz)
      return oz_gemm(ta, tb, ma, mb, mm, nn, kk, alpha, Aa, lda_, Bb, ldb_, beta, Cc, ldc_, false,
                     scratch_of(h.oz_ws), &ds->barrier_err, st);
    if (tf_terms)
      return tf32_gemm(ta, tb, ma, mb, mm, nn, kk, alpha, Aa, lda_, Bb, ldb_, beta, Cc, ldc_,
                       tf_terms, scratch_of(h.oz_ws), &ds->barrier_err, st);
    return fgemm(ta, tb, ma, mb, mm, nn, kk, alpha, Aa, lda_, Bb, ldb_, beta, Cc, ldc_);
  }
  Status ggemm(int64_t kk, const double* W, int64_t ldw_, int64_t bb, double* S) {
    if (tf_terms) {
      LLS_TRY(h.oz_ws.reserve(oz_gemm_workspace_bytes(bb, bb, kk)));
      return oz_gemm(true, false, kUnitLower, kUnitLower, bb, bb, kk, 1.0, W, ldw_, W, ldw_, 0.0, S,
                     nb, false, scratch_of(h.oz_ws), &ds->barrier_err, st);
    }
    return xgemm(true, false, kUnitLower, kUnitLower, bb, bb, kk, 1.0, W, ldw_, W, ldw_, 0.0, S, nb);
  }
};

// ---------------------------------------------------------------------------
// randUTV + rank (+ Nullify when opt.nullify)
// ---------------------------------------------------------------------------
Status factorize(Handle& h, Factor& f, const double* A, int64_t m, int64_t n, int64_t lda,
                 double tol, bool keep_a) {
  cudaStream_t st = h.stream;
  int nb = 0, q = 0;
  effective_nb_q(h.opt, h.tune.get(), m, n, &nb, &q);
  f.m = m;
  f.n = n;
  f.ldt = std::max<int64_t>(m, 1);
  f.nb = nb;
  f.q = q;
  f.precision = h.opt.precision;
  f.nullified = false;
  f.has_v = h.opt.explicit_v != 0;
  f.has_a = keep_a && h.opt.max_refine > 0;
  if (!f.has_v) f.Vx.release();
  if (!f.has_a) f.A0.release();
  f.ks.clear();
  f.bs.clear();
  f.rz.clear();
  f.rank = f.rank_count = 0;
  const int64_t mn = std::min(m, n);
  for (int64_t k = 0; k < mn; k += nb) {
    f.ks.push_back(k);
    f.bs.push_back(std::min<int64_t>(nb, std::min(m - k, n - k)));
  }
  const int64_t steps = (int64_t)f.ks.size();
  const size_t blk = (size_t)nb * nb;
  const int64_t ldt = f.ldt, ldw = std::max<int64_t>(n, 1);

  LLS_TRY(f.T.reserve(sizeof(double) * (size_t)ldt * n));
  LLS_TRY(f.WV.reserve(sizeof(double) * (size_t)ldw * n));
  LLS_TRY(f.TV.reserve(sizeof(double) * blk * std::max<int64_t>(steps, 1)));
  LLS_TRY(f.TU.reserve(sizeof(double) * blk * std::max<int64_t>(steps, 1)));
  LLS_TRY(f.US.reserve(sizeof(double) * blk * std::max<int64_t>(steps, 1)));
  LLS_TRY(f.VS.reserve(sizeof(double) * blk * std::max<int64_t>(steps, 1)));
  LLS_TRY(f.Rblk.reserve(sizeof(double) * blk * std::max<int64_t>(steps, 1)));
  LLS_TRY(f.tauV.reserve(sizeof(double) * nb * std::max<int64_t>(steps, 1)));
  LLS_TRY(f.tauU.reserve(sizeof(double) * nb * std::max<int64_t>(steps, 1)));
  LLS_TRY(f.sigma.reserve(sizeof(double) * nb * std::max<int64_t>(steps, 1)));
  const int64_t ldv = std::max<int64_t>(n, 1);
  if (f.has_v) LLS_TRY(f.Vx.reserve(sizeof(double) * (size_t)ldv * n));
  if (f.has_a) LLS_TRY(f.A0.reserve(sizeof(double) * (size_t)ldt * n));

  // workspace
  const int64_t mx = std::max(m, n);
  LLS_TRY(h.G.reserve(sizeof(double) * (size_t)std::max<int64_t>(m, 1) * nb));
  LLS_TRY(h.Wt.reserve(sizeof(double) * (size_t)std::max<int64_t>(mx, 1) * nb));
  LLS_TRY(h.P.reserve(sizeof(double) * (size_t)std::max<int64_t>(mx, 1) * nb));
  LLS_TRY(h.P2.reserve(sizeof(double) * (size_t)std::max<int64_t>(mx, 1) * nb));
  LLS_TRY(h.Q.reserve(sizeof(double) * (size_t)nb * std::max<int64_t>(n, 1)));
  LLS_TRY(h.Q2.reserve(sizeof(double) * (size_t)nb * std::max<int64_t>(n, 1)));
  LLS_TRY(h.S.reserve(sizeof(double) * blk));
  LLS_TRY(h.gemm_ws.reserve(loop_gemm_scratch(m, n, nb, 64)));
  LLS_TRY(h.panel_ws.reserve(panel_qr_scratch_bytes(std::max<int64_t>(mx + nb, 1), nb) + 64));
  LLS_TRY(h.dstat.reserve(sizeof(DevStatus)));
  DevStatus* ds = h.dstat.as<DevStatus>();
  LLS_CUDA(cudaMemsetAsync(ds, 0, sizeof(DevStatus), st));
  Scratch pws = scratch_of(h.panel_ws);
  // Mixed precision: the trailing updates and Nullify's products run on the
  // tensor cores, as FP64-accurate GEMMs (exact BF16 slices, oz_gemm.cu) or
  // with TF32 split operands (tf32_gemm.cu: 3xTF32 or plain TF32).
  FactorGemms g(h, nb);
  if (g.tc()) {
    size_t need = 0;
    for (int64_t i = 0; i < steps; ++i) {
      const int64_t k = f.ks[i], b = f.bs[i], mp = m - k, np = n - k;
      need = std::max(need, g.tc_ws_bytes(m, b, np));
      need = std::max(need, g.tc_ws_bytes(m, np, b));
      need = std::max(need, g.tc_ws_bytes(b, np - b, mp));
      need = std::max(need, g.tc_ws_bytes(mp, np - b, b));
      need = std::max(need, g.tc_ws_bytes(b, b, std::max(np, mp)));  // Gram W^T W
      if (g.tf_terms) need = std::max(need, oz_gemm_workspace_bytes(b, b, std::max(np, mp)));
      need = std::max(need, g.tc_ws_bytes(k, b, b));                 // A01 V_SVD
      if (f.has_v) {  // V's right update and V_SVD
        need = std::max(need, g.tc_ws_bytes(n, b, np));
        need = std::max(need, g.tc_ws_bytes(n, np, b));
        need = std::max(need, g.tc_ws_bytes(n, b, b));
      }
    }
    LLS_TRY(h.oz_ws.reserve(need));
  }
  // T <- A, with the finiteness check; V <- I; the refinement copy of A.
  LLS_TRY(copy_check(m, n, A, lda, f.T.d(), ldt, &ds->nonfinite, st));
  if (f.has_v) LLS_TRY(set_identity(n, f.Vx.d(), ldv, st));
  if (f.has_a) LLS_TRY(copy_matrix(m, n, f.T.d(), ldt, f.A0.d(), ldt, st));

  double* T = f.T.d();
  double* WV = f.WV.d();
  for (int64_t i = 0; i < steps; ++i) {
    const int64_t k = f.ks[i], b = f.bs[i];
    const int64_t mp = m - k, np = n - k;
    double* ABR = T + k + k * ldt;
    double* Y = WV + k + k * ldw;
    double* TVi = f.TV.d() + i * blk;
    double* TUi = f.TU.d() + i * blk;
    double* tauVi = f.tauV.d() + i * nb;
    double* tauUi = f.tauU.d() + i * nb;

    // ---- a1/a2: sketch and sample Y = (A_BR^T A_BR)^q A_BR^T G
    std::optional<TraceScope> phase;
    phase.emplace(kTrPhaseSample, st);
    if (h.opt.precision != LLS_FP64) {
      LLS_TRY(sample_bf16(h, ABR, ldt, mp, np, b, q, h.opt.seed, i, Y, ldw));
    } else {
      LLS_TRY(launch_sketch(h.opt.seed, i, mp, b, h.G.d(), std::max<int64_t>(m, 1), st));
      LLS_TRY(g.fgemm(true, false, kDense, kDense, np, b, mp, 1.0, ABR, ldt, h.G.d(),
                   std::max<int64_t>(m, 1), 0.0, Y, ldw));
      for (int it = 0; it < q; ++it) {
        LLS_TRY(g.fgemm(false, false, kDense, kDense, mp, b, np, 1.0, ABR, ldt, Y, ldw, 0.0, h.Wt.d(),
                     std::max<int64_t>(mp, 1)));
        LLS_TRY(g.fgemm(true, false, kDense, kDense, np, b, mp, 1.0, ABR, ldt, h.Wt.d(),
                     std::max<int64_t>(mp, 1), 0.0, Y, ldw));
      }
    }
    // ---- a3: [Y, T_V, W_V] = unpivoted_QR(Y)
    phase.reset();
    phase.emplace(kTrPhaseQrY, st);
    LLS_TRY(panel_qr(np, b, Y, ldw, tauVi, pws, &ds->barrier_err, st, h.shares_device));
    LLS_TRY(g.ggemm(np, Y, ldw, b, h.S.d()));
    LLS_TRY(wy_tfactor(b, h.S.d(), nb, tauVi, TVi, nb, st));
    // ---- a4: T(:, k:n) <- T(:, k:n) - (T(:, k:n) W_V) T_V W_V^T, all m rows
    phase.reset();
    phase.emplace(kTrPhaseRight, st);
    double* Tk = T + k * ldt;
    LLS_TRY(g.xgemm(false, false, kDense, kUnitLower, m, b, np, 1.0, Tk, ldt, Y, ldw, 0.0, h.P.d(),
                  m));
    LLS_TRY(g.xgemm(false, false, kDense, kDense, m, b, b, 1.0, h.P.d(), m, TVi, nb, 0.0, h.P2.d(),
                  m));
    LLS_TRY(g.xgemm(false, true, kDense, kUnitLower, m, np, b, -1.0, h.P2.d(), m, Y, ldw, 1.0, Tk,
                  ldt));
    if (f.has_v) {  // V(:, k:n) <- V(:, k:n) (I - W_V T_V W_V^T), all n rows
      double* Vk = f.Vx.d() + k * ldv;
      LLS_TRY(g.xgemm(false, false, kDense, kUnitLower, n, b, np, 1.0, Vk, ldv, Y, ldw, 0.0, h.P.d(),
                    ldv));
      LLS_TRY(g.xgemm(false, false, kDense, kDense, n, b, b, 1.0, h.P.d(), ldv, TVi, nb, 0.0,
                    h.P2.d(), ldv));
      LLS_TRY(g.xgemm(false, true, kDense, kUnitLower, n, np, b, -1.0, h.P2.d(), ldv, Y, ldw, 1.0, Vk,
                    ldv));
    }
    // ---- a5: [[A11; A21], T_U, W_U] = unpivoted_QR([A11; A21])
    phase.reset();
    phase.emplace(kTrPhasePanel, st);
    LLS_TRY(panel_qr(mp, b, ABR, ldt, tauUi, pws, &ds->barrier_err, st, h.shares_device));
    LLS_TRY(copy_upper(b, ABR, ldt, f.Rblk.d() + i * blk, nb, st));
    LLS_TRY(g.ggemm(mp, ABR, ldt, b, h.S.d()));
    LLS_TRY(wy_tfactor(b, h.S.d(), nb, tauUi, TUi, nb, st));
    // ---- a6: [A12; A22] <- (I - W_U T_U W_U^T)^T [A12; A22]
    phase.reset();
    phase.emplace(kTrPhaseLeft, st);
    if (np > b) {
      double* A12 = ABR + b * ldt;
      LLS_TRY(g.xgemm(true, false, kUnitLower, kDense, b, np - b, mp, 1.0, ABR, ldt, A12, ldt, 0.0,
                    h.Q.d(), nb));
      LLS_TRY(g.xgemm(true, false, kDense, kDense, b, np - b, b, 1.0, TUi, nb, h.Q.d(), nb, 0.0,
                    h.Q2.d(), nb));
      LLS_TRY(g.xgemm(false, false, kUnitLower, kDense, mp, np - b, b, -1.0, ABR, ldt, h.Q2.d(), nb,
                    1.0, A12, ldt));
    }
  }

  // ---- a7: all diagonal-block SVDs in one launch, then their updates
  std::optional<TraceScope> phase;
  phase.emplace(kTrPhaseSvd, st);
  if (steps > 0) {
    LLS_TRY(jacobi_svd_batched((int)steps, nb, (int)f.bs.back(), f.Rblk.d(), nb, (int64_t)blk,
                               f.sigma.d(), nb, f.US.d(), nb, (int64_t)blk, f.VS.d(), nb,
                               (int64_t)blk, &ds->svd_status, st));
  }
  for (int64_t i = 0; i < steps; ++i) {
    const int64_t k = f.ks[i], b = f.bs[i];
    LLS_TRY(set_diag_block(b, f.sigma.d() + i * nb, T + k + k * ldt, ldt, st));
    if (k > 0) {  // A01 <- A01 V_SVD
      LLS_TRY(g.xgemm(false, false, kDense, kDense, k, b, b, 1.0, T + k * ldt, ldt,
                    f.VS.d() + i * blk, nb, 0.0, h.P.d(), k));
      LLS_TRY(copy_matrix(k, b, h.P.d(), k, T + k * ldt, ldt, st));
    }
    if (f.has_v) {  // V(:, k:k+b) <- V(:, k:k+b) V_SVD (later steps never touch these columns)
      LLS_TRY(g.xgemm(false, false, kDense, kDense, n, b, b, 1.0, f.Vx.d() + k * ldv, ldv,
                    f.VS.d() + i * blk, nb, 0.0, h.P.d(), ldv));
      LLS_TRY(copy_matrix(n, b, h.P.d(), ldv, f.Vx.d() + k * ldv, ldv, st));
    }
  }
  for (int64_t i = 0; i < steps; ++i) {
    const int64_t k = f.ks[i], b = f.bs[i], np = n - k;
    if (np > b) {  // A12 <- U_SVD^T A12
      double* A12 = T + k + (k + b) * ldt;
      LLS_TRY(g.xgemm(true, false, kDense, kDense, b, np - b, b, 1.0, f.US.d() + i * blk, nb, A12,
                    ldt, 0.0, h.Q.d(), nb));
      LLS_TRY(copy_matrix(b, np - b, h.Q.d(), nb, A12, ldt, st));
    }
  }

  phase.reset();
  return finish_factorization(h, f, tol);
}

// ---------------------------------------------------------------------------
// a8 Compute_rank and a9 Nullify on a factor whose step loop is done
// ---------------------------------------------------------------------------
Status finish_factorization(Handle& h, Factor& f, double tol) {
  cudaStream_t st = h.stream;
  const int64_t m = f.m, n = f.n, ldt = f.ldt, mn = std::min(m, n);
  const int nb = f.nb;
  const int64_t ldv = std::max<int64_t>(n, 1);
  double* T = f.T.d();
  LLS_TRY(h.dstat.reserve(sizeof(DevStatus)));
  LLS_TRY(h.S.reserve(sizeof(double) * (size_t)nb * nb));
  FactorGemms g(h, nb);
  DevStatus* ds = g.ds;
  Scratch pws = scratch_of(h.panel_ws);
  std::optional<TraceScope> phase;
  // ---- a8: Compute_rank
  phase.emplace(kTrPhaseRank, st);
  if (mn > 0) {
    LLS_TRY(resolve_tol(tol, std::max(m, n), T, &ds->tol, st));
    LLS_TRY(rank_scan_dev(mn, T, ldt, &ds->tol, ds->rank, st));
  }
  phase.reset();
  if (!h.hstat) LLS_CUDA(cudaMallocHost((void**)&h.hstat, sizeof(DevStatus)));
  LLS_CUDA(cudaMemcpyAsync(h.hstat, ds, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  LLS_CUDA(cudaStreamSynchronize(st));
  DevStatus hs = *h.hstat;
  if (hs.nonfinite) return make_error(LLS_ERR_NONFINITE, "A has a NaN or Inf entry", 2);
  if (hs.barrier_err) return make_error(LLS_ERR_TIMEOUT, "a device-side wait timed out");
  if (hs.rank[2]) return make_error(LLS_ERR_NONFINITE, "NaN on the diagonal of T");
  if (hs.svd_status) return make_error(LLS_ERR_SVD_NOCONV, "block SVD did not converge");
  f.tol = mn > 0 ? hs.tol : tol;
  f.rank = mn > 0 ? hs.rank[0] : 0;
  f.rank_count = mn > 0 ? hs.rank[1] : 0;

  // ---- a9: Nullify_top_right_part_of_T (Fig. 3)
  //
  // Row block [C11 D1] (rows j0..j1-1 of T, C11 = T(j0:j1, j0:j1), D1 =
  // T(j0:j1, r:n)) is annihilated by one reflector per row, bottom row first,
  // each acting on column i and columns r..n-1.  Written as a QR: with rows
  // and columns of the block reversed and transposed,
  //   M = [ C11 reversed^T ; D1 reversed^T ]   ((bsz + L) x bsz, L = n - r),
  // M(p', j) = T(j1-1-j, j1-1-p') for p' < bsz, M(bsz+p, j) = T(j1-1-j, r+p);
  // the top block of M is upper triangular, so the Householder QR M = Q R
  // produces exactly the RZ reflectors (their top part is the identity).
  // [C11 D1] Q = R^T gives the new C11 (reversed back) and D1 = 0; the rows
  // above (C01 | D0 in the same coordinates) are multiplied by
  // Q = I - W T W^T from the right, and x gets Q from the left.
  const int64_t r = f.rank;
  if (h.opt.nullify && r > 0 && r < n) {
    TraceScope nullify_phase(kTrPhaseNullify, st);
    const int64_t L = n - r;
    int64_t j1 = r;
    size_t off_m = 0, off_t = 0, off_tau = 0;
    while (j1 > 0) {
      int64_t j0 = std::max<int64_t>(0, j1 - nb);
      Factor::RzBlock bl{j0, j1 - j0, off_m, off_t, off_tau};
      off_m += (size_t)(bl.bsz + L) * bl.bsz;
      off_t += (size_t)bl.bsz * bl.bsz;
      off_tau += (size_t)bl.bsz;
      f.rz.push_back(bl);
      j1 = j0;
    }
    LLS_TRY(f.RzM.reserve(sizeof(double) * off_m));
    LLS_TRY(f.RzT.reserve(sizeof(double) * off_t));
    LLS_TRY(f.RzTau.reserve(sizeof(double) * off_tau));
    const int64_t xrows = f.has_v ? std::max(r, n) : r;  // rows updated per block: T's, V's
    LLS_TRY(h.xc.reserve(sizeof(double) * (size_t)std::max<int64_t>(xrows, 1) * nb));
    LLS_TRY(h.gemm_ws.reserve(std::max(h.gemm_ws.bytes,
                                       std::max(gemm_scratch_bytes(nb, nb, L + nb),
                                                gemm_scratch_bytes(xrows, nb, L)))));
    LLS_TRY(h.panel_ws.reserve(panel_qr_scratch_bytes(L + nb, nb) + 64));
    pws = scratch_of(h.panel_ws);
    LLS_TRY(h.P.reserve(sizeof(double) * (size_t)std::max<int64_t>(xrows, 1) * nb));
    LLS_TRY(h.P2.reserve(sizeof(double) * (size_t)std::max<int64_t>(xrows, 1) * nb));
    // [X_rev | X_tail] <- [X_rev | X_tail] (I - W T_z W^T) with W = [I; W_bot]:
    // the block's reflectors applied from the right to `rows` rows of a
    // matrix X (ld ldx) whose columns j0..j0+bsz-1 are taken reversed and
    // whose columns r..n-1 form the tail (Update of Fig. 3).
    auto apply_rz_right = [&](int64_t rows, double* Xm, int64_t ldx, int64_t j0, int64_t bsz,
                              const double* Wbot, int64_t ldm, const double* Tz) -> Status {
      double* Xc = h.xc.d();
      double* D0 = Xm + r * ldx;
      LLS_TRY(copy_cols_reversed(rows, bsz, Xm + j0 * ldx, ldx, Xc, rows, st));
      LLS_TRY(copy_matrix(rows, bsz, Xc, rows, h.P.d(), rows, st));
      if (g.tc()) LLS_TRY(h.oz_ws.reserve(std::max(g.tc_ws_bytes(rows, bsz, L), g.tc_ws_bytes(rows, L, bsz))));
      if (g.tc()) LLS_TRY(h.oz_ws.reserve(g.tc_ws_bytes(rows, bsz, bsz)));
      LLS_TRY(g.xgemm(false, false, kDense, kDense, rows, bsz, L, 1.0, D0, ldx, Wbot, ldm, 1.0,
                    h.P.d(), rows));
      LLS_TRY(g.xgemm(false, false, kDense, kDense, rows, bsz, bsz, 1.0, h.P.d(), rows, Tz, bsz, 0.0,
                    h.P2.d(), rows));
      LLS_TRY(g.xgemm(false, true, kDense, kDense, rows, L, bsz, -1.0, h.P2.d(), rows, Wbot, ldm, 1.0,
                    D0, ldx));
      // X_rev -= P2 W_top^T with W_top = I, then reversed back into X
      LLS_TRY(axpy_matrix(rows, bsz, -1.0, h.P2.d(), rows, Xc, rows, st));
      LLS_TRY(copy_cols_reversed(rows, bsz, Xc, rows, Xm + j0 * ldx, ldx, st));
      return ok_status();
    };
    for (const auto& bl : f.rz) {
      const int64_t j0 = bl.j0, bsz = bl.bsz, ldm = bsz + L;
      double* M = f.RzM.d() + bl.off_m;
      double* Tz = f.RzT.d() + bl.off_t;
      double* tz = f.RzTau.d() + bl.off_tau;
      LLS_TRY(rz_gather(bsz, L, T, ldt, j0, r, M, ldm, st));
      LLS_TRY(panel_qr(ldm, bsz, M, ldm, tz, pws, &ds->barrier_err, st, h.shares_device));
      if (g.tc()) LLS_TRY(h.oz_ws.reserve(g.tc_ws_bytes(bsz, bsz, ldm)));
      LLS_TRY(g.ggemm(ldm, M, ldm, bsz, h.S.d()));
      LLS_TRY(wy_tfactor(bsz, h.S.d(), nb, tz, Tz, bsz, st));
      LLS_TRY(rz_scatter(bsz, M, ldm, T, ldt, j0, r, L, st));
      // Update(C_01, D_0): the rows of T above the block
      if (j0 > 0) LLS_TRY(apply_rz_right(j0, T, ldt, j0, bsz, M + bsz, ldm, Tz));
      // Update(E_1, F): all n rows of an explicit V
      if (f.has_v) LLS_TRY(apply_rz_right(n, f.Vx.d(), ldv, j0, bsz, M + bsz, ldm, Tz));
    }
    f.nullified = true;
    LLS_CUDA(cudaMemcpyAsync(&h.hstat->barrier_err, &ds->barrier_err, sizeof(int),
                             cudaMemcpyDeviceToHost, st));
    LLS_CUDA(cudaStreamSynchronize(st));
    if (h.hstat->barrier_err) return make_error(LLS_ERR_TIMEOUT, "Nullify grid barrier timed out");
  }
  if (f.rank != f.rank_count) return make_error(LLS_WARN_RANK_NONPREFIX, "rank is not a prefix");
  return ok_status();
}

// ---------------------------------------------------------------------------
// a10: x = V (T_tl^{-1} (U^T b)), from four replays of the stored factors
// (U^T, U, V^T, V), which the refinement of the TF32 modes uses as well.
// ---------------------------------------------------------------------------
namespace {

// FP64 GEMM on the handle's stream with its split-K scratch grown to the
// shape's plan first.
Status hgemm(Handle& h, bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t mm, int64_t nn,
             int64_t kk, double alpha, const double* Aa, int64_t lda_, const double* Bb,
             int64_t ldb_, double beta, double* Cc, int64_t ldc_) {
  LLS_TRY(h.gemm_ws.reserve(gemm_scratch_bytes(mm, nn, kk)));
  return gemm(ta, tb, ma, mb, mm, nn, kk, alpha, Aa, lda_, Bb, ldb_, beta, Cc, ldc_,
              scratch_of(h.gemm_ws), h.stream);
}

// y = beta y + alpha op(A) x (op(A) mm x kk, x kk x nrhs): the thin products
// for nrhs <= kThinMaxRhs, else the FP64 GEMM.
Status hgemv(Handle& h, bool ta, int64_t mm, int64_t nrhs, int64_t kk, double alpha,
             const double* Aa, int64_t lda_, const double* x, int64_t ldx, double beta, double* y,
             int64_t ldy) {
  if (nrhs <= kThinMaxRhs) {
    LLS_TRY(h.gemm_ws.reserve(thin_gemv_scratch_bytes(ta, mm, kk, nrhs)));
    return thin_gemv(ta, false, mm, kk, nrhs, alpha, Aa, lda_, x, ldx, beta, y, ldy,
                     scratch_of(h.gemm_ws), h.stream);
  }
  return hgemm(h, ta, false, kDense, kDense, mm, nrhs, kk, alpha, Aa, lda_, x, ldx, beta, y, ldy);
}

// With at most four right-hand sides, a factor whose larger side has at
// least kPersistentMinRows rows replays its reflectors as one cooperative
// launch each (replay_persistent) and the refinement's triangular solves
// likewise (trsm_upper_inv_persistent).  The choice depends on the shape
// alone, never on the handle, so a solve gives the same bits on any handle or
// worker; smaller factors -- the batched and most served problems -- keep the
// per-step kernels, which need no cooperative launch and let worker streams
// overlap.
constexpr int64_t kPersistentMinRows = 4096;
bool persistent_solve(const Factor& f, int64_t nrhs) {
  return nrhs <= 4 && f.nb <= 128 && !f.ks.empty() && std::max(f.m, f.n) >= kPersistentMinRows;
}
// The reflectors also need a TMA map: an even leading dimension and a 16-byte
// aligned base, which every factor buffer of the library has (its arenas
// align each buffer to 256 bytes).
bool persistent_replay(const Factor& f, int64_t nrhs, const double* W, int64_t ldw_, int64_t M) {
  return persistent_solve(f, nrhs) &&
         replay_persistent_fits(f.nb, nrhs, W, ldw_, M, f.ks.back() + f.bs.back());
}

// Buffers of one replay: two nb x nrhs panels and the thin path's scratch.
Status reserve_replay(Handle& h, Factor& f, int64_t nrhs) {
  LLS_TRY(h.sp.reserve(sizeof(double) * (size_t)f.nb * nrhs));
  LLS_TRY(h.sp2.reserve(sizeof(double) * (size_t)f.nb * nrhs));
  LLS_TRY(h.xc.reserve(sizeof(double) * (size_t)f.nb * nrhs));
  if (nrhs <= kThinMaxRhs) {
    size_t need = thin_scratch_bytes(std::max(f.m, f.n), f.nb, nrhs);
    if (persistent_solve(f, nrhs)) need = std::max(need, replay_persistent_scratch_bytes(f.nb, nrhs));
    LLS_TRY(h.gemm_ws.reserve(need));
  }
  return ok_status();
}

// Every reflector step of one replay (forward: U^T / V^T order) in a single
// cooperative launch; W, ldw and Tf are the factor's reflectors and T factors.
Status replay_steps(Handle& h, Factor& f, bool forward, int64_t M, const double* W, int64_t ldw_,
                    const double* Tf, double* x, int64_t ldx, int64_t nrhs) {
  const int64_t kmax = f.ks.back() + f.bs.back();
  return replay_persistent(forward, M, f.nb, (int64_t)f.ks.size(), kmax, W, ldw_, Tf, x, ldx, nrhs,
                           scratch_of(h.gemm_ws), &h.dstat.as<DevStatus>()->barrier_err, h.stream);
}

// One step's reflector block applied to x (M x nrhs): x <- (I - W op(T) W^T) x.
Status step_reflect(Handle& h, int64_t M, int64_t b, int64_t nrhs, const double* W, int64_t ldw_,
                    const double* T, int nb, bool transT, double* x, int64_t ldx) {
  if (nrhs <= kThinMaxRhs)
    return apply_reflectors_thin(M, b, nrhs, W, ldw_, T, nb, transT, x, ldx, scratch_of(h.gemm_ws),
                                 h.stream);
  double* p = h.sp.d();
  double* p2 = h.sp2.d();
  LLS_TRY(hgemm(h, true, false, kUnitLower, kDense, b, nrhs, M, 1.0, W, ldw_, x, ldx, 0.0, p, nb));
  LLS_TRY(hgemm(h, transT, false, kDense, kDense, b, nrhs, b, 1.0, T, nb, p, nb, 0.0, p2, nb));
  return hgemm(h, false, false, kUnitLower, kDense, M, nrhs, b, -1.0, W, ldw_, p2, nb, 1.0, x, ldx);
}

// x(0:b) <- op(S) x(0:b) for one step's b x b singular-vector block.
Status step_small(Handle& h, int64_t b, int64_t nrhs, const double* S, int nb, bool transS, double* x,
                  int64_t ldx) {
  if (nrhs <= kThinMaxRhs) return small_block_mul(b, nrhs, S, nb, transS, x, ldx, h.stream);
  LLS_TRY(hgemm(h, transS, false, kDense, kDense, b, nrhs, b, 1.0, S, nb, x, ldx, 0.0, h.sp.d(), nb));
  return copy_matrix(b, nrhs, h.sp.d(), nb, x, ldx, h.stream);
}

// One Nullify row block's reflectors applied to z (n x nrhs) in its
// coordinates [rows j0..j0+bsz reversed; rows r..n]: z <- (I - W op(T_z) W^T) z
// with W = [I; W_bot] (Fig. 3's Update, written as a QR of the reversed block).
Status nullify_block(Handle& h, Factor& f, const Factor::RzBlock& bl, int64_t nrhs, bool transT,
                     double* Z, int64_t ldz) {
  cudaStream_t st = h.stream;
  const int64_t r = f.rank, L = f.n - r, j0 = bl.j0, bsz = bl.bsz, ldm = bsz + L;
  const double* M = f.RzM.d() + bl.off_m;
  const double* Tz = f.RzT.d() + bl.off_t;
  double* zc = h.xc.d();
  double* p = h.sp.d();
  double* p2 = h.sp2.d();
  if (nrhs <= kThinMaxRhs) {
    // p = reversed rows of the block + W_bot^T Z_tail; p2 = op(T_z) p; the
    // block's rows (W_top = I, reversed) and the tail take -p2 and -W_bot p2
    LLS_TRY(copy_rows_reversed(bsz, nrhs, Z + j0, ldz, p, bsz, st));
    LLS_TRY(hgemv(h, true, bsz, nrhs, L, 1.0, M + bsz, ldm, Z + r, ldz, 1.0, p, bsz));
    LLS_TRY(small_blocks_batched(1, bsz, bsz, nrhs, Tz, transT, p, bsz, p2, bsz, st));
    LLS_TRY(axpy_rows_reversed(bsz, nrhs, -1.0, p2, bsz, Z + j0, ldz, st));
    return hgemv(h, false, L, nrhs, bsz, -1.0, M + bsz, ldm, p2, bsz, 1.0, Z + r, ldz);
  }
  LLS_TRY(copy_rows_reversed(bsz, nrhs, Z + j0, ldz, zc, bsz, st));
  LLS_TRY(copy_matrix(bsz, nrhs, zc, bsz, p, bsz, st));
  LLS_TRY(hgemm(h, true, false, kDense, kDense, bsz, nrhs, L, 1.0, M + bsz, ldm, Z + r, ldz, 1.0, p,
                bsz));
  LLS_TRY(hgemm(h, transT, false, kDense, kDense, bsz, nrhs, bsz, 1.0, Tz, bsz, p, bsz, 0.0, p2, bsz));
  LLS_TRY(axpy_matrix(bsz, nrhs, -1.0, p2, bsz, zc, bsz, st));  // W_top = I
  LLS_TRY(hgemm(h, false, false, kDense, kDense, L, nrhs, bsz, -1.0, M + bsz, ldm, p2, bsz, 1.0,
                Z + r, ldz));
  return copy_rows_reversed(bsz, nrhs, zc, bsz, Z + j0, ldz, st);
}

// With few right-hand sides every step's b x b block of a replay in one
// launch: x(0:kmax) <- blockdiag(op(S_i)) x(0:kmax).  In U^T / V^T order each
// block multiplies rows k_i..k_i+b_i after that step's reflector, and no later
// step touches those rows; in U / V order each multiplies them before its
// reflector, and no earlier step has touched them: either way all of them can
// run together, after (or before) the reflector loop.
Status batched_small(Handle& h, Factor& f, const double* S, bool transS, double* x, int64_t ldx,
                     int64_t nrhs) {
  const int64_t nblk = (int64_t)f.ks.size();
  if (nblk == 0) return ok_status();
  const int64_t kmax = f.ks.back() + f.bs.back();
  LLS_TRY(h.sbat.reserve(sizeof(double) * (size_t)kmax * nrhs));
  LLS_TRY(small_blocks_batched(nblk, f.nb, kmax, nrhs, S, transS, x, ldx, h.sbat.d(), kmax,
                               h.stream));
  return copy_matrix(kmax, nrhs, h.sbat.d(), kmax, x, ldx, h.stream);
}

}  // namespace

// c (m x nrhs) <- U^T c = U_SVD,s^T H_s^T ... U_SVD,0^T H_0^T c (first step first).
Status apply_ut(Handle& h, Factor& f, double* c, int64_t ldc, int64_t nrhs) {
  const size_t blk = (size_t)f.nb * f.nb;
  LLS_TRY(reserve_replay(h, f, nrhs));
  const bool thin = nrhs <= kThinMaxRhs;
  if (persistent_replay(f, nrhs, f.T.d(), f.ldt, f.m))
    LLS_TRY(replay_steps(h, f, true, f.m, f.T.d(), f.ldt, f.TU.d(), c, ldc, nrhs));
  else
    for (size_t i = 0; i < f.ks.size(); ++i) {
      const int64_t k = f.ks[i], b = f.bs[i];
      LLS_TRY(step_reflect(h, f.m - k, b, nrhs, f.T.d() + k + k * f.ldt, f.ldt, f.TU.d() + i * blk,
                           f.nb, true, c + k, ldc));
      if (!thin) LLS_TRY(step_small(h, b, nrhs, f.US.d() + i * blk, f.nb, true, c + k, ldc));
    }
  if (thin) LLS_TRY(batched_small(h, f, f.US.d(), true, c, ldc, nrhs));
  return ok_status();
}

// w (m x nrhs) <- U w = H_0 U_SVD,0 ... H_s U_SVD,s w (last step first).
Status apply_u(Handle& h, Factor& f, double* w, int64_t ldw_, int64_t nrhs) {
  const size_t blk = (size_t)f.nb * f.nb;
  LLS_TRY(reserve_replay(h, f, nrhs));
  const bool thin = nrhs <= kThinMaxRhs;
  if (thin) LLS_TRY(batched_small(h, f, f.US.d(), false, w, ldw_, nrhs));
  if (persistent_replay(f, nrhs, f.T.d(), f.ldt, f.m))
    return replay_steps(h, f, false, f.m, f.T.d(), f.ldt, f.TU.d(), w, ldw_, nrhs);
  for (size_t ii = f.ks.size(); ii-- > 0;) {
    const int64_t k = f.ks[ii], b = f.bs[ii];
    if (!thin) LLS_TRY(step_small(h, b, nrhs, f.US.d() + ii * blk, f.nb, false, w + k, ldw_));
    LLS_TRY(step_reflect(h, f.m - k, b, nrhs, f.T.d() + k + k * f.ldt, f.ldt, f.TU.d() + ii * blk, f.nb,
                         false, w + k, ldw_));
  }
  return ok_status();
}

// z (n x nrhs) <- V z; rows kz..n of z are zero (kz = r for [y; 0]), which an
// explicit V uses.  V = H_0 V_SVD,0 ... H_s V_SVD,s Z_0 ... Z_last with the
// Nullify blocks Z in processing order: the last block first, then the steps
// last first.
Status apply_v(Handle& h, Factor& f, double* z, int64_t ldz, int64_t nrhs, int64_t kz) {
  const int64_t n = f.n, ldv = std::max<int64_t>(n, 1);
  const size_t blk = (size_t)f.nb * f.nb;
  LLS_TRY(reserve_replay(h, f, nrhs));
  if (f.has_v) {  // V with Nullify's reflectors included
    LLS_TRY(h.z2.reserve(sizeof(double) * (size_t)n * nrhs));
    LLS_TRY(hgemm(h, false, false, kDense, kDense, n, nrhs, kz, 1.0, f.Vx.d(), ldv, z, ldz, 0.0,
                  h.z2.d(), ldv));
    return copy_matrix(n, nrhs, h.z2.d(), ldv, z, ldz, h.stream);
  }
  if (f.nullified)
    for (auto it = f.rz.rbegin(); it != f.rz.rend(); ++it)
      LLS_TRY(nullify_block(h, f, *it, nrhs, false, z, ldz));
  const bool thin = nrhs <= kThinMaxRhs;
  if (thin) LLS_TRY(batched_small(h, f, f.VS.d(), false, z, ldz, nrhs));
  if (persistent_replay(f, nrhs, f.WV.d(), ldv, n))
    return replay_steps(h, f, false, n, f.WV.d(), ldv, f.TV.d(), z, ldz, nrhs);
  for (size_t ii = f.ks.size(); ii-- > 0;) {
    const int64_t k = f.ks[ii], b = f.bs[ii];
    if (!thin) LLS_TRY(step_small(h, b, nrhs, f.VS.d() + ii * blk, f.nb, false, z + k, ldz));
    LLS_TRY(step_reflect(h, n - k, b, nrhs, f.WV.d() + k + k * ldv, ldv, f.TV.d() + ii * blk, f.nb,
                         false, z + k, ldz));
  }
  return ok_status();
}

// z (n x nrhs) <- V^T z (the steps first step first, then the Nullify blocks
// in processing order, each transposed).
Status apply_vt(Handle& h, Factor& f, double* z, int64_t ldz, int64_t nrhs) {
  const int64_t n = f.n, ldv = std::max<int64_t>(n, 1);
  const size_t blk = (size_t)f.nb * f.nb;
  LLS_TRY(reserve_replay(h, f, nrhs));
  if (f.has_v) {
    LLS_TRY(h.z2.reserve(sizeof(double) * (size_t)n * nrhs));
    LLS_TRY(hgemm(h, true, false, kDense, kDense, n, nrhs, n, 1.0, f.Vx.d(), ldv, z, ldz, 0.0,
                  h.z2.d(), ldv));
    return copy_matrix(n, nrhs, h.z2.d(), ldv, z, ldz, h.stream);
  }
  const bool thin = nrhs <= kThinMaxRhs;
  if (persistent_replay(f, nrhs, f.WV.d(), ldv, n))
    LLS_TRY(replay_steps(h, f, true, n, f.WV.d(), ldv, f.TV.d(), z, ldz, nrhs));
  else
    for (size_t i = 0; i < f.ks.size(); ++i) {
      const int64_t k = f.ks[i], b = f.bs[i];
      LLS_TRY(step_reflect(h, n - k, b, nrhs, f.WV.d() + k + k * ldv, ldv, f.TV.d() + i * blk, f.nb,
                           true, z + k, ldz));
      if (!thin) LLS_TRY(step_small(h, b, nrhs, f.VS.d() + i * blk, f.nb, true, z + k, ldz));
    }
  if (thin) LLS_TRY(batched_small(h, f, f.VS.d(), true, z, ldz, nrhs));
  if (f.nullified)
    for (const auto& bl : f.rz) LLS_TRY(nullify_block(h, f, bl, nrhs, true, z, ldz));
  return ok_status();
}

Status solve_factored(Handle& h, Factor& f, const double* B, int64_t nrhs, int64_t ldb, double* X,
                      int64_t ldx) {
  cudaStream_t st = h.stream;
  const int64_t m = f.m, n = f.n, ldt = f.ldt, ldw = std::max<int64_t>(n, 1);
  const int64_t r = f.rank;
  if (n == 0 || nrhs == 0) return ok_status();
  if (r == 0 || m == 0) return fill_zero(n, nrhs, X, ldx, st);
  std::optional<TraceScope> solve_phase;
  if (!h.in_refine) solve_phase.emplace(kTrPhaseSolve, st);
  LLS_TRY(h.bw.reserve(sizeof(double) * (size_t)m * nrhs));
  LLS_TRY(h.z.reserve(sizeof(double) * (size_t)n * nrhs));
  LLS_TRY(h.dstat.reserve(sizeof(DevStatus)));
  DevStatus* ds = h.dstat.as<DevStatus>();
  double* Bw = h.bw.d();
  double* Z = h.z.d();
  LLS_CUDA(cudaMemsetAsync(&ds->nonfinite, 0, 2 * sizeof(int), st));  // nonfinite, barrier_err
  LLS_TRY(copy_check(m, nrhs, B, ldb, Bw, m, &ds->nonfinite, st));
  LLS_TRY(apply_ut(h, f, Bw, m, nrhs));  // c = U^T b
  LLS_TRY(h.gemm_ws.reserve(trsm_upper_scratch_bytes(r, nrhs)));
  LLS_TRY(trsm_upper(r, nrhs, f.T.d(), ldt, Bw, m, scratch_of(h.gemm_ws), st));  // y = T_tl^{-1} c
  LLS_TRY(copy_matrix(r, nrhs, Bw, m, Z, ldw, st));                              // z = [y; 0]
  if (r < n) LLS_TRY(fill_zero(n - r, nrhs, Z + r, ldw, st));
  LLS_TRY(apply_v(h, f, Z, ldw, nrhs, r));                                        // x = V z
  LLS_TRY(copy_matrix(n, nrhs, Z, ldw, X, ldx, st));
  return read_nonfinite_flag(h, ds);
}

namespace {

// Per-column ||dx|| / ||x|| of the last correction (max over columns) from
// the norms refine_update wrote.
double max_correction(const std::vector<double>& norms, int64_t nrhs) {
  double corr = 0.0;
  for (int64_t j = 0; j < nrhs; ++j) {
    const double dn = std::sqrt(norms[2 * j]), xn = std::sqrt(norms[2 * j + 1]);
    const double c = xn > 0.0 ? dn / xn : (dn > 0.0 ? INFINITY : 0.0);
    corr = std::max(corr, c);
  }
  return corr;
}

// Ratio of the largest dropped to the smallest kept singular value of the
// diagonal blocks above which the minimum-norm refinement is not applied.
constexpr double kMinNormGap = 1e-2;

// x += D (n x nrhs), then the last correction's size: returns -1 when it
// grew over `prev` (the correction is undone: the iteration does not
// contract for these factors), else the correction.
Status add_correction(Handle& h, int64_t n, int64_t nrhs, const double* D, double* X, int64_t ldx,
                      double prev, bool first, double* corr) {
  cudaStream_t st = h.stream;
  std::vector<double> norms(2 * (size_t)nrhs);
  LLS_TRY(refine_update(n, nrhs, D, n, X, ldx, h.nrm.d(), st));
  LLS_CUDA(cudaMemcpyAsync(norms.data(), h.nrm.d(), sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost,
                           st));
  LLS_CUDA(cudaStreamSynchronize(st));
  *corr = max_correction(norms, nrhs);
  if (!first && *corr > prev) {
    LLS_TRY(axpy_matrix(n, nrhs, -1.0, D, n, X, ldx, st));
    *corr = -1.0;
  }
  return ok_status();
}

// The refinement of the TF32 modes.  Their factors carry the TF32 split's
// errors, so range(V_1) is off the row space by about that error times the
// condition number kappa of T_11: x <- x + P r then converges to a solution
// in the tilted range(V_1), and a one-stage x <- x + A^T P^T P P^T A^T r
// carries P P^T ~ (A^T A)^+ and contracts only when kappa^2 eps < 1.  Two
// stages that need only kappa eps < 1:
//  1. least squares: x <- x + N N^T A^T (b - A x), N = V_1 T_11^{-1}, from
//     x = P b.  In z (x = N z) it is z <- z + K^T (b - K z) with K = A N
//     = U_1 up to kappa eps; its fixed point has r orthogonal to
//     range(A V_1) = range(A).
//  2. minimum norm: x <- x + L L^T (x_ls - x), L = A^T U_1 T_11^{-T}, from
//     x = 0: the fixed point is x_ls projected onto range(L) = range(A^T).
// For a matrix of numerical rank r that is the minimum-norm least-squares
// solution.  Without a gap at the rank (singular values beyond it
// comparable to the kept ones) A itself is not of rank r and the fixed
// points leave the truncated solution P b: the diagonal blocks' singular
// values are checked first and, without a gap of kMinNormGap, x = P b is
// kept (warning).
Status refine_min_norm(Handle& h, Factor& f, const double* A, int64_t lda, const double* B,
                       int64_t nrhs, int64_t ldb, double* X, int64_t ldx) {
  cudaStream_t st = h.stream;
  const int64_t m = f.m, n = f.n, r = f.rank, ldt = f.ldt;
  LLS_TRY(h.nrm.reserve(sizeof(double) * std::max<int64_t>(2 * nrhs, 2)));
  LLS_TRY(diag_gap(std::min(m, n), f.sigma.d(), r, h.nrm.d(), st));
  double gap[2];
  LLS_CUDA(cudaMemcpyAsync(gap, h.nrm.d(), sizeof(gap), cudaMemcpyDeviceToHost, st));
  LLS_CUDA(cudaStreamSynchronize(st));
  if (gap[1] > kMinNormGap * gap[0])
    return make_error(LLS_WARN_REFINE_NOCONV,
                      "no gap at the rank (largest dropped / smallest kept singular value " +
                          std::to_string(gap[1] / gap[0]) + "): refinement not applied");
  LLS_TRY(h.rr.reserve(sizeof(double) * (size_t)m * nrhs));
  LLS_TRY(h.rs.reserve(sizeof(double) * (size_t)n * nrhs));
  LLS_TRY(h.dd.reserve(sizeof(double) * (size_t)n * nrhs));
  LLS_TRY(h.z2.reserve(sizeof(double) * (size_t)n * nrhs));
  LLS_TRY(h.gemm_ws.reserve(std::max(trsm_upper_scratch_bytes(r, nrhs),
                                     trsm_upper_trans_scratch_bytes(r, nrhs))));
  double* rr = h.rr.d();
  double* rs = h.rs.d();
  double* dd = h.dd.d();
  double* xls = h.z2.d();
  // With few right-hand sides the 64 x 64 diagonal blocks of T_11 are
  // inverted once and each triangular solve multiplies by them.
  const bool thin = nrhs <= kThinMaxRhs;
  if (thin) {
    LLS_TRY(h.dinv.reserve(trsm_inverse_bytes(r)));
    LLS_TRY(trsm_block_inverses(r, f.T.d(), ldt, h.dinv.d(), st));
  }
  // With at most four on a large factor (persistent_solve), each solve is one
  // cooperative launch with a grid barrier per block.
  const bool coop_trsm = persistent_solve(f, nrhs);
  if (coop_trsm) LLS_TRY(h.sp2.reserve(64));
  auto trsm_both = [&](double* y, int64_t ldy, bool trans_first) -> Status {
    if (coop_trsm) {
      int* err = &h.dstat.as<DevStatus>()->barrier_err;
      const Scratch sc = scratch_of(h.sp2);
      LLS_TRY(trsm_upper_inv_persistent(r, nrhs, f.T.d(), ldt, h.dinv.d(), y, ldy, trans_first, sc,
                                        err, st));
      return trsm_upper_inv_persistent(r, nrhs, f.T.d(), ldt, h.dinv.d(), y, ldy, !trans_first, sc,
                                       err, st);
    }
    if (thin) {
      LLS_TRY(trsm_upper_inv(r, nrhs, f.T.d(), ldt, h.dinv.d(), y, ldy, trans_first, st));
      return trsm_upper_inv(r, nrhs, f.T.d(), ldt, h.dinv.d(), y, ldy, !trans_first, st);
    }
    LLS_TRY(h.gemm_ws.reserve(std::max(trsm_upper_scratch_bytes(r, nrhs),
                                       trsm_upper_trans_scratch_bytes(r, nrhs))));
    if (trans_first) LLS_TRY(trsm_upper_trans(r, nrhs, f.T.d(), ldt, y, ldy, scratch_of(h.gemm_ws), st));
    LLS_TRY(trsm_upper(r, nrhs, f.T.d(), ldt, y, ldy, scratch_of(h.gemm_ws), st));
    if (!trans_first) LLS_TRY(trsm_upper_trans(r, nrhs, f.T.d(), ldt, y, ldy, scratch_of(h.gemm_ws), st));
    return ok_status();
  };
  int steps = 0;
  double corr = 0.0;
  bool converged[2] = {false, false};
  for (int stage = 0; stage < 2; ++stage) {
    if (stage == 1) {  // x_ls = x; x = 0
      LLS_TRY(copy_matrix(n, nrhs, X, ldx, xls, n, st));
      LLS_TRY(fill_zero(n, nrhs, X, ldx, st));
    }
    double prev = 0.0;
    for (int it = 1; it <= h.opt.max_refine; ++it) {
      double* D;
      if (stage == 0) {  // dx = V [T_11^{-1} T_11^{-T} (V^T A^T (b - A x))(0:r); 0]
        LLS_TRY(copy_matrix(m, nrhs, B, ldb, rr, m, st));
        LLS_TRY(hgemv(h, false, m, nrhs, n, -1.0, A, lda, X, ldx, 1.0, rr, m));
        LLS_TRY(hgemv(h, true, n, nrhs, m, 1.0, A, lda, rr, m, 0.0, rs, n));
        LLS_TRY(apply_vt(h, f, rs, n, nrhs));
        LLS_TRY(trsm_both(rs, n, true));
        if (r < n) LLS_TRY(fill_zero(n - r, nrhs, rs + r, n, st));
        LLS_TRY(apply_v(h, f, rs, n, nrhs, r));
        D = rs;
      } else {  // dx = A^T U [T_11^{-T} T_11^{-1} (U^T A (x_ls - x))(0:r); 0]
        LLS_TRY(copy_matrix(n, nrhs, xls, n, rs, n, st));
        LLS_TRY(axpy_matrix(n, nrhs, -1.0, X, ldx, rs, n, st));
        LLS_TRY(hgemv(h, false, m, nrhs, n, 1.0, A, lda, rs, n, 0.0, rr, m));
        LLS_TRY(apply_ut(h, f, rr, m, nrhs));
        LLS_TRY(trsm_both(rr, m, false));
        if (r < m) LLS_TRY(fill_zero(m - r, nrhs, rr + r, m, st));
        LLS_TRY(apply_u(h, f, rr, m, nrhs));
        LLS_TRY(hgemv(h, true, n, nrhs, m, 1.0, A, lda, rr, m, 0.0, dd, n));
        D = dd;
      }
      double c = 0.0;
      LLS_TRY(add_correction(h, n, nrhs, D, X, ldx, prev, it == 1, &c));
      if (c < 0.0) break;  // grew: undone
      ++steps;
      corr = c;
      if (c <= h.opt.refine_tol) {
        converged[stage] = true;
        break;
      }
      if (it > 1 && c > 0.5 * prev) break;  // no longer contracting: rounding floor
      prev = c;
    }
  }
  h.refine_steps = steps;
  h.refine_corr = corr;
  LLS_TRY(read_nonfinite_flag(h, h.dstat.as<DevStatus>()));  // the replays' barrier flag
  if (converged[0] && converged[1]) return ok_status();
  return make_error(LLS_WARN_REFINE_NOCONV, "refinement correction " + std::to_string(corr) +
                                                " above refine_tol");
}

}  // namespace

// ---------------------------------------------------------------------------
// Iterative refinement: x <- x + P (b - A x), P = V_1 T_11^{-1} U_1^T applied
// by solve_factored, the residual in FP64 with the original A; for factors
// made in a TF32 mode, refine_min_norm above.
// ---------------------------------------------------------------------------
Status solve_refined(Handle& h, Factor& f, const double* A, int64_t lda, const double* B,
                     int64_t nrhs, int64_t ldb, double* X, int64_t ldx) {
  h.refine_steps = 0;
  h.refine_corr = 0.0;
  LLS_TRY(solve_factored(h, f, B, nrhs, ldb, X, ldx));
  const int64_t m = f.m, n = f.n;
  if (!A && f.has_a) {
    A = f.A0.d();
    lda = f.ldt;
  }
  if (h.opt.max_refine <= 0 || !A || m == 0 || n == 0 || nrhs == 0 || f.rank == 0)
    return ok_status();
  TraceScope refine_phase(kTrPhaseRefine, h.stream);
  struct InRefine {
    Handle& h;
    explicit InRefine(Handle& hh) : h(hh) { h.in_refine = true; }
    ~InRefine() { h.in_refine = false; }
  } in_refine(h);
  if (f.precision == LLS_MIXED_BF16_3xTF32 || f.precision == LLS_MIXED_BF16_TF32)
    return refine_min_norm(h, f, A, lda, B, nrhs, ldb, X, ldx);
  cudaStream_t st = h.stream;
  LLS_TRY(h.rr.reserve(sizeof(double) * (size_t)m * nrhs));
  LLS_TRY(h.dd.reserve(sizeof(double) * (size_t)n * nrhs));
  LLS_TRY(h.nrm.reserve(sizeof(double) * 2 * (size_t)nrhs));
  LLS_TRY(h.gemm_ws.reserve(gemm_scratch_bytes(m, nrhs, n)));
  std::vector<double> norms(2 * (size_t)nrhs);
  double prev = 0.0;
  for (int it = 1; it <= h.opt.max_refine; ++it) {
    // r = b - A x
    LLS_TRY(copy_matrix(m, nrhs, B, ldb, h.rr.d(), m, st));
    LLS_TRY(hgemv(h, false, m, nrhs, n, -1.0, A, lda, X, ldx, 1.0, h.rr.d(), m));
    // d = P r; x += d
    LLS_TRY(solve_factored(h, f, h.rr.d(), nrhs, m, h.dd.d(), n));
    LLS_TRY(refine_update(n, nrhs, h.dd.d(), n, X, ldx, h.nrm.d(), st));
    LLS_CUDA(cudaMemcpyAsync(norms.data(), h.nrm.d(), sizeof(double) * 2 * nrhs,
                             cudaMemcpyDeviceToHost, st));
    LLS_CUDA(cudaStreamSynchronize(st));
    const double corr = max_correction(norms, nrhs);
    if (it > 1 && corr > prev) {
      // growing corrections: the factors are too inaccurate for this matrix
      // (the iteration does not contract); keep the previous iterate
      LLS_TRY(axpy_matrix(n, nrhs, -1.0, h.dd.d(), n, X, ldx, st));
      break;
    }
    h.refine_steps = it;
    h.refine_corr = corr;
    if (corr <= h.opt.refine_tol) return ok_status();
    if (it > 1 && corr > 0.5 * prev) break;  // no longer contracting: rounding floor
    prev = corr;
  }
  return make_error(LLS_WARN_REFINE_NOCONV, "refinement correction " + std::to_string(h.refine_corr) +
                                                " above refine_tol");
}

}  // namespace lls
