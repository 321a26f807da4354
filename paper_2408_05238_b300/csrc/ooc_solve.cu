// Out-of-core solve (lls_solve_ooc): the randUTV least-squares solve with
// the matrix in pinned host memory and at most `cache_panels` column panels
// of it on the device at a time (the paper's block cache of Sec. 3.5, with
// device memory as the cache and host memory as the disk).
//
// The executor follows the schedule of ooc_plan.cu action by action: before
// an access it writes back the panel the action evicts (if modified) and
// loads the accessed panel into its slot, then runs the step of the method
// the access stands for on that slot, with the same launchers and the same
// arithmetic as the in-core solver (solver.cu).  Phase 1 (the step loop and
// the block-SVD pass) ends with every modified panel written back; the rank
// is then read, and phase 2 (Nullify and the solve's panel reads) runs from
// an empty cache.  Side data stays on the device (the sketch, Y, W, the WY
// products, per-step T_V, T_U, U_s, V_s) except each step's W_V and each
// Nullify block's reflector panel, which go to pinned host memory and come
// back for x = V z.  Copies run in stream order on the handle's stream (no
// overlap of copies and compute in this version).
//
// Every operand handed to a launcher is first checked, on the host, to lie
// inside the buffer it belongs to; a failed check returns LLS_ERR_ARG
// before anything is launched.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lls_kernels.h"
#include "solver.h"

namespace lls {

std::vector<lls_ooc_action> ooc_schedule_phase(int64_t m, int64_t n, int64_t nb, int q,
                                               int64_t r, bool nullify, int64_t cache_panels,
                                               int32_t policy, int phase);

namespace {

// A buffer of doubles (device or pinned host) and its length.
struct Span {
  double* p = nullptr;
  int64_t n = 0;
};

Span span_of(DevBuf& b) { return Span{b.d(), (int64_t)(b.bytes / sizeof(double))}; }

// rows x cols at ptr with leading dimension ld must lie inside b.
Status inside(const Span& b, const double* ptr, int64_t rows, int64_t cols, int64_t ld,
              const char* what) {
  if (rows <= 0 || cols <= 0) return ok_status();
  if (!b.p || ptr < b.p || ld < rows)
    return make_error(LLS_ERR_ARG, std::string("out-of-core extent check failed: ") + what);
  const int64_t off = ptr - b.p;
  const int64_t last = off + (cols - 1) * ld + rows - 1;
  if (last >= b.n)
    return make_error(LLS_ERR_ARG, std::string("out-of-core extent check failed: ") + what);
  return ok_status();
}

}  // namespace
}  // namespace lls

namespace lls {
namespace {

// Pinned host buffer of doubles.
struct HostBuf {
  double* p = nullptr;
  int64_t n = 0;
  HostBuf() = default;
  HostBuf(const HostBuf&) = delete;
  HostBuf& operator=(const HostBuf&) = delete;
  ~HostBuf() {
    if (p) cudaFreeHost(p);
  }
  Status alloc(int64_t count) {
    if (count <= 0) count = 1;
    if (cudaMallocHost((void**)&p, sizeof(double) * (size_t)count) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return make_error(LLS_ERR_NOMEM, "pinned host allocation failed");
    }
    n = count;
    return ok_status();
  }
  Span span() const { return Span{p, n}; }
};

struct OocSolve {
  Handle& h;
  cudaStream_t st;
  int64_t m, n, nb, P, steps, C, nrhs;
  int q;
  uint64_t seed;
  bool nullify;
  int64_t r = 0, rcount = 0;
  int64_t L = 0;
  HostBuf Hs, WVh, RZh;  // the matrix (m x n, ld m), each step's W_V, Nullify's panels
  std::vector<int64_t> rz_off;  // offset of block p's panel in RZh
  DevBuf slots, G, Ya, Yb, Wa, Wb, Pm, P2, Qb, Q2, S, WU, TV, TU, US, VS, R11, tauV, tauU,
      sigma, Tb, M, D1a, D1b, Xc, TZ, tz, c, sp, sp2, Z, zc;
  // Y (W_V after its QR) and the next step's Y; W and the previous W; D_1
  // and the next block's rows: pairs whose roles swap
  DevBuf *Y = &Ya, *Yn = &Yb, *W = &Wa, *Wp = &Wb, *D1 = &D1a, *D1n = &D1b;
  DevStatus* ds = nullptr;

  explicit OocSolve(Handle& hh) : h(hh), st(hh.stream) {}
  // Nothing queued may still use the pinned buffers when they are freed.
  ~OocSolve() { cudaStreamSynchronize(st); }

  int64_t c0(int64_t j) const { return j * nb; }
  int64_t w(int64_t j) const { return std::min(nb, n - j * nb); }
  int64_t kk(int64_t i) const { return i * nb; }
  int64_t bb(int64_t i) const { return std::min(nb, std::min(m - i * nb, n - i * nb)); }
  double* slot(int64_t s) { return slots.d() + s * m * nb; }
  Span slot_span(int64_t s) { return Span{slot(s), m * nb}; }
  double* blk(DevBuf& b, int64_t i) { return b.d() + i * nb * nb; }

  Status gm(bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t M_, int64_t N_, int64_t K_,
            double alpha, const double* A, int64_t lda, const Span& sa, const double* B,
            int64_t ldb, const Span& sb, double beta, double* Cc, int64_t ldc, const Span& sc) {
    if (M_ <= 0 || N_ <= 0) return ok_status();
    if (K_ > 0) {
      LLS_TRY(inside(sa, A, ta ? K_ : M_, ta ? M_ : K_, lda, "gemm A"));
      LLS_TRY(inside(sb, B, tb ? N_ : K_, tb ? K_ : N_, ldb, "gemm B"));
    }
    LLS_TRY(inside(sc, Cc, M_, N_, ldc, "gemm C"));
    LLS_TRY(h.gemm_ws.reserve(gemm_scratch_bytes(M_, N_, K_)));
    return gemm(ta, tb, ma, mb, M_, N_, K_, alpha, A, lda, B, ldb, beta, Cc, ldc,
                Scratch{h.gemm_ws.p, h.gemm_ws.bytes}, st);
  }
  Status cp(int64_t rows, int64_t cols, const double* src, int64_t lds, const Span& ss,
            double* dst, int64_t ldd, const Span& sd) {
    LLS_TRY(inside(ss, src, rows, cols, lds, "copy source"));
    LLS_TRY(inside(sd, dst, rows, cols, ldd, "copy destination"));
    return copy_matrix(rows, cols, src, lds, dst, ldd, st);
  }
  Status qr(int64_t rows, int64_t cols, double* A, int64_t lda, const Span& sa, double* tau,
            const Span& stau) {
    LLS_TRY(inside(sa, A, rows, cols, lda, "panel"));
    LLS_TRY(inside(stau, tau, std::min(rows, cols), 1, std::max<int64_t>(std::min(rows, cols), 1),
                   "tau"));
    return panel_qr(rows, cols, A, lda, tau, Scratch{h.panel_ws.p, h.panel_ws.bytes},
                    &ds->barrier_err, st);
  }
  // T factor of the unit-lower reflectors stored at A (rows x b) into T (ld ldt).
  Status tfactor(int64_t rows, int64_t b, const double* A, int64_t lda, const Span& sa,
                 const double* tau, double* T, int64_t ldt, const Span& stt) {
    LLS_TRY(gm(true, false, kUnitLower, kUnitLower, b, b, rows, 1.0, A, lda, sa, A, lda, sa, 0.0,
               S.d(), nb, span_of(S)));
    LLS_TRY(inside(stt, T, b, b, ldt, "T factor"));
    return wy_tfactor(b, S.d(), nb, tau, T, ldt, st);
  }
  Status load(int64_t panel, int64_t s) {
    LLS_TRY(inside(Hs.span(), Hs.p + c0(panel) * m, m, w(panel), m, "host panel"));
    return cuda_status(cudaMemcpyAsync(slot(s), Hs.p + c0(panel) * m,
                                       sizeof(double) * (size_t)(m * w(panel)),
                                       cudaMemcpyHostToDevice, st),
                       "load a panel");
  }
  Status store(int64_t panel, int64_t s) {
    LLS_TRY(inside(Hs.span(), Hs.p + c0(panel) * m, m, w(panel), m, "host panel"));
    return cuda_status(cudaMemcpyAsync(Hs.p + c0(panel) * m, slot(s),
                                       sizeof(double) * (size_t)(m * w(panel)),
                                       cudaMemcpyDeviceToHost, st),
                       "write back a panel");
  }

  // ---- workspace ---------------------------------------------------------
  Status setup() {
    const int64_t blk = nb * nb, mb = m * nb, nbn = n * nb;
    for (DevBuf* b : {&slots, &G, &Ya, &Yb, &Wa, &Wb, &Pm, &P2, &Qb, &Q2, &S, &WU, &TV, &TU, &US,
                      &VS, &R11, &tauV, &tauU, &sigma, &Tb, &M, &D1a, &D1b, &Xc, &TZ, &tz, &c, &sp,
                      &sp2, &Z, &zc})
      b->bind(st);
    auto res = [](DevBuf& b, int64_t doubles) {
      return b.reserve(sizeof(double) * (size_t)std::max<int64_t>(doubles, 1));
    };
    LLS_TRY(res(slots, C * mb));
    LLS_TRY(res(G, mb));
    LLS_TRY(res(Ya, nbn));
    LLS_TRY(res(Yb, nbn));
    LLS_TRY(res(Wa, mb));
    LLS_TRY(res(Wb, mb));
    LLS_TRY(res(Pm, mb));
    LLS_TRY(res(P2, mb));
    LLS_TRY(res(Qb, blk));
    LLS_TRY(res(Q2, blk));
    LLS_TRY(res(S, blk));
    LLS_TRY(res(WU, mb));
    for (DevBuf* b : {&TV, &TU, &US, &VS, &R11}) LLS_TRY(res(*b, steps * blk));
    for (DevBuf* b : {&tauV, &tauU, &sigma}) LLS_TRY(res(*b, steps * nb));
    LLS_TRY(res(c, m * nrhs));
    LLS_TRY(res(sp, nb * nrhs));
    LLS_TRY(res(sp2, nb * nrhs));
    LLS_TRY(res(Z, n * nrhs));
    LLS_TRY(res(zc, nb * nrhs));
    LLS_TRY(h.panel_ws.reserve(panel_qr_scratch_bytes(std::max(m, n) + nb, nb) + 64));
    LLS_TRY(h.dstat.reserve(sizeof(DevStatus)));
    ds = h.dstat.as<DevStatus>();
    LLS_CUDA(cudaMemsetAsync(ds, 0, sizeof(DevStatus), st));
    LLS_TRY(WVh.alloc(n * n));
    return ok_status();
  }

  // ---- phase 1: sampling, the P pass, the update pass, the block SVDs ----
  Status op_sample_atg(int64_t i, int64_t j, double* X, const Span& xs, bool first) {
    const int64_t k = kk(i), b = bb(i), yo = c0(j) - k;
    if (first) {
      LLS_TRY(inside(span_of(G), G.d(), m - k, b, m, "sketch"));
      LLS_TRY(launch_sketch(seed, i, m - k, b, G.d(), m, st));
    }
    return gm(true, false, kDense, kDense, w(j), b, m - k, 1.0, X + k, m, xs, G.d(), m,
              span_of(G), 0.0, Y->d() + yo, n, span_of(*Y));
  }
  Status op_sample_ay(int64_t i, int64_t j, double* X, const Span& xs, bool first) {
    const int64_t k = kk(i), b = bb(i), yo = c0(j) - k;
    return gm(false, false, kDense, kDense, m - k, b, w(j), 1.0, X + k, m, xs, Y->d() + yo, n,
              span_of(*Y), first ? 0.0 : 1.0, W->d(), m, span_of(*W));
  }
  Status op_sample_atw_ay(int64_t i, int64_t j, double* X, const Span& xs, bool first) {
    const int64_t k = kk(i), b = bb(i), yo = c0(j) - k;
    if (first) std::swap(W, Wp);
    LLS_TRY(gm(true, false, kDense, kDense, w(j), b, m - k, 1.0, X + k, m, xs, Wp->d(), m,
               span_of(*Wp), 0.0, Y->d() + yo, n, span_of(*Y)));
    return gm(false, false, kDense, kDense, m - k, b, w(j), 1.0, X + k, m, xs, Y->d() + yo, n,
              span_of(*Y), first ? 0.0 : 1.0, W->d(), m, span_of(*W));
  }
  Status op_sample_atw(int64_t i, int64_t j, double* X, const Span& xs, bool) {
    const int64_t k = kk(i), b = bb(i), yo = c0(j) - k;
    return gm(true, false, kDense, kDense, w(j), b, m - k, 1.0, X + k, m, xs, W->d(), m,
              span_of(*W), 0.0, Y->d() + yo, n, span_of(*Y));
  }
  // P += T(:, panel j) W_V(rows of panel j); first: QR of Y -> (W_V, T_V), W_V to host
  Status op_product_twv(int64_t i, int64_t j, double* X, const Span& xs, bool first) {
    const int64_t k = kk(i), b = bb(i), yo = c0(j) - k;
    const Span ys = span_of(*Y);
    if (first) {
      LLS_TRY(qr(n - k, b, Y->d(), n, ys, tauV.d() + i * nb, span_of(tauV)));
      LLS_TRY(tfactor(n - k, b, Y->d(), n, ys, tauV.d() + i * nb, blk(TV, i), nb, span_of(TV)));
      LLS_TRY(inside(WVh.span(), WVh.p + k + k * n, n - k, b, n, "host W_V"));
      LLS_CUDA(cudaMemcpy2DAsync(WVh.p + k + k * n, sizeof(double) * n, Y->d(), sizeof(double) * n,
                                 sizeof(double) * (n - k), b, cudaMemcpyDeviceToHost, st));
    }
    const OperandMode mode = j == i ? kUnitLower : kDense;
    return gm(false, false, kDense, mode, m, b, w(j), 1.0, X, m, xs, Y->d() + yo, n, ys,
              first ? 0.0 : 1.0, Pm.d(), m, span_of(Pm));
  }
  // rows k..m of `cols` columns at Xk (ld m) <- (I - W_U T_U W_U^T)^T (...)
  Status left_update(int64_t i, double* Xk, int64_t cols, const Span& xs) {
    const int64_t k = kk(i), b = bb(i);
    LLS_TRY(gm(true, false, kUnitLower, kDense, b, cols, m - k, 1.0, WU.d(), m, span_of(WU), Xk, m,
               xs, 0.0, Qb.d(), nb, span_of(Qb)));
    LLS_TRY(gm(true, false, kDense, kDense, b, cols, b, 1.0, blk(TU, i), nb, span_of(TU), Qb.d(),
               nb, span_of(Qb), 0.0, Q2.d(), nb, span_of(Q2)));
    return gm(false, false, kUnitLower, kDense, m - k, cols, b, -1.0, WU.d(), m, span_of(WU),
              Q2.d(), nb, span_of(Q2), 1.0, Xk, m, xs);
  }
  Status op_update(int64_t i, int64_t j, double* X, const Span& xs, bool first) {
    const int64_t k = kk(i), b = bb(i), yo = c0(j) - k, wj = w(j);
    const bool nxt = i + 1 < steps;
    if (first) {
      LLS_TRY(gm(false, false, kDense, kDense, m, b, b, 1.0, Pm.d(), m, span_of(Pm), blk(TV, i), nb,
                 span_of(TV), 0.0, P2.d(), m, span_of(P2)));
      if (nxt) {
        LLS_TRY(inside(span_of(G), G.d(), m - kk(i + 1), bb(i + 1), m, "sketch"));
        LLS_TRY(launch_sketch(seed, i + 1, m - kk(i + 1), bb(i + 1), G.d(), m, st));
      }
    }
    // right update, all m rows
    const OperandMode mode = j == i ? kUnitLower : kDense;
    LLS_TRY(gm(false, true, kDense, mode, m, wj, b, -1.0, P2.d(), m, span_of(P2), Y->d() + yo, n,
               span_of(*Y), 1.0, X, m, xs));
    if (j == i) {
      LLS_TRY(qr(m - k, b, X + k, m, xs, tauU.d() + i * nb, span_of(tauU)));
      LLS_TRY(inside(span_of(R11), blk(R11, i), b, b, nb, "R11"));
      LLS_TRY(inside(xs, X + k, b, b, m, "R11 source"));
      LLS_TRY(copy_upper(b, X + k, m, blk(R11, i), nb, st));
      LLS_TRY(tfactor(m - k, b, X + k, m, xs, tauU.d() + i * nb, blk(TU, i), nb, span_of(TU)));
      LLS_TRY(cp(m - k, b, X + k, m, xs, WU.d(), m, span_of(WU)));
      if (wj > b) LLS_TRY(left_update(i, X + k + b * m, wj - b, xs));  // narrow last step
    } else {
      LLS_TRY(left_update(i, X + k, wj, xs));
    }
    if (nxt && j >= i + 1) {
      const int64_t k2 = kk(i + 1), b2 = bb(i + 1), yo2 = c0(j) - k2;
      LLS_TRY(gm(true, false, kDense, kDense, wj, b2, m - k2, 1.0, X + k2, m, xs, G.d(), m,
                 span_of(G), 0.0, Yn->d() + yo2, n, span_of(*Yn)));
    }
    if (nxt && j == P - 1) std::swap(Y, Yn);
    return ok_status();
  }
  Status op_svd(int64_t j, double* X, const Span& xs, bool first) {
    if (first) {
      LLS_TRY(jacobi_svd_batched((int)steps, (int)nb, (int)bb(steps - 1), R11.d(), nb, nb * nb,
                                 sigma.d(), nb, US.d(), nb, nb * nb, VS.d(), nb, nb * nb,
                                 &ds->svd_status, st));
    }
    const int64_t wj = w(j);
    if (j < steps) {
      const int64_t k = kk(j), b = bb(j);
      if (k > 0) {
        LLS_TRY(gm(false, false, kDense, kDense, k, b, b, 1.0, X, m, xs, blk(VS, j), nb,
                   span_of(VS), 0.0, Pm.d(), m, span_of(Pm)));
        LLS_TRY(cp(k, b, Pm.d(), m, span_of(Pm), X, m, xs));
      }
      LLS_TRY(inside(xs, X + k, b, b, m, "diagonal block"));
      LLS_TRY(set_diag_block(b, sigma.d() + j * nb, X + k, m, st));
      if (wj > b) {
        LLS_TRY(gm(true, false, kDense, kDense, b, wj - b, b, 1.0, blk(US, j), nb, span_of(US),
                   X + k + b * m, m, xs, 0.0, Qb.d(), nb, span_of(Qb)));
        LLS_TRY(cp(b, wj - b, Qb.d(), nb, span_of(Qb), X + k + b * m, m, xs));
      }
    }
    for (int64_t i = 0; i < std::min(j, steps); ++i) {
      const int64_t k = kk(i), b = bb(i);
      LLS_TRY(gm(true, false, kDense, kDense, b, wj, b, 1.0, blk(US, i), nb, span_of(US), X + k, m,
                 xs, 0.0, Qb.d(), nb, span_of(Qb)));
      LLS_TRY(cp(b, wj, Qb.d(), nb, span_of(Qb), X + k, m, xs));
    }
    return ok_status();
  }

  // ---- phase 2: Nullify (panel-aligned row blocks) and the solve ----------
  int64_t blk_j0(int64_t p) const { return p * nb; }
  int64_t blk_size(int64_t p) const { return std::min(r, (p + 1) * nb) - p * nb; }
  // Columns of panel j in D = T(0:r, r:n): first local column, count, first D column.
  void dcols(int64_t j, int64_t* loc, int64_t* cnt, int64_t* dc) const {
    const int64_t lo = std::max(c0(j), r);
    *loc = lo - c0(j);
    *cnt = c0(j) + w(j) - lo;
    *dc = lo - r;
  }
  Status setup_nullify() {
    L = n - r;
    const int64_t blocks = (r - 1) / nb + 1;
    for (DevBuf* b : {&Tb, &M, &D1a, &D1b, &Xc, &TZ, &tz}) b->bind(st);
    auto res = [](DevBuf& b, int64_t doubles) {
      return b.reserve(sizeof(double) * (size_t)std::max<int64_t>(doubles, 1));
    };
    LLS_TRY(res(Tb, nb * (nb + L)));
    LLS_TRY(res(M, (nb + L) * nb));
    LLS_TRY(res(D1a, nb * L));
    LLS_TRY(res(D1b, nb * L));
    LLS_TRY(res(Xc, m * nb));
    LLS_TRY(res(TZ, blocks * nb * nb));
    LLS_TRY(res(tz, nb));
    rz_off.assign((size_t)blocks, 0);
    int64_t off = 0;
    for (int64_t p = 0; p < blocks; ++p) {
      rz_off[(size_t)p] = off;
      off += (blk_size(p) + L) * blk_size(p);
    }
    return RZh.alloc(off);
  }
  Status op_null_gather(int64_t p, int64_t j, double* X, const Span& xs) {
    int64_t loc, cnt, dc;
    dcols(j, &loc, &cnt, &dc);
    return cp(blk_size(p), cnt, X + blk_j0(p) + loc * m, m, xs, D1->d() + dc * nb, nb,
              span_of(*D1));
  }
  Status op_null_read(int64_t p, int64_t j, double* X, const Span& xs, bool first) {
    const int64_t j0 = blk_j0(p), bsz = blk_size(p), ldm = bsz + L;
    const Span ms = span_of(M);
    if (first && j != p) return make_error(LLS_ERR_ARG, "Nullify read pass must start at its block");
    if (first) {  // panel p: this block's reflectors from [C_11 | D_1], then C_01 reversed
      LLS_TRY(cp(bsz, bsz, X + j0, m, xs, Tb.d(), nb, span_of(Tb)));
      LLS_TRY(cp(bsz, L, D1->d(), nb, span_of(*D1), Tb.d() + bsz * nb, nb, span_of(Tb)));
      LLS_TRY(inside(ms, M.d(), ldm, bsz, ldm, "Nullify panel"));
      LLS_TRY(rz_gather(bsz, L, Tb.d(), nb, 0, bsz, M.d(), ldm, st));
      LLS_TRY(qr(ldm, bsz, M.d(), ldm, ms, tz.d(), span_of(tz)));
      LLS_TRY(tfactor(ldm, bsz, M.d(), ldm, ms, tz.d(), blk(TZ, p), bsz, span_of(TZ)));
      LLS_TRY(inside(RZh.span(), RZh.p + rz_off[(size_t)p], ldm, bsz, ldm, "host Nullify panel"));
      LLS_CUDA(cudaMemcpyAsync(RZh.p + rz_off[(size_t)p], M.d(), sizeof(double) * ldm * bsz,
                               cudaMemcpyDeviceToHost, st));
      if (j0 > 0) {
        LLS_TRY(inside(xs, X, j0, bsz, m, "C_01"));
        LLS_TRY(inside(span_of(Pm), Pm.d(), j0, bsz, m, "P"));
        LLS_TRY(copy_cols_reversed(j0, bsz, X, m, Pm.d(), m, st));
      }
    }
    if (j >= r / nb && j0 > 0) {  // D_0's part of P = [C_01 reversed | D_0] W
      int64_t loc, cnt, dc;
      dcols(j, &loc, &cnt, &dc);
      LLS_TRY(gm(false, false, kDense, kDense, j0, bsz, cnt, 1.0, X + loc * m, m, xs,
                 M.d() + bsz + dc, ldm, ms, 1.0, Pm.d(), m, span_of(Pm)));
    }
    return ok_status();
  }
  Status op_null_write(int64_t p, int64_t j, double* X, const Span& xs, bool first) {
    const int64_t j0 = blk_j0(p), bsz = blk_size(p), ldm = bsz + L;
    const Span ms = span_of(M);
    if (first && j0 > 0)
      LLS_TRY(gm(false, false, kDense, kDense, j0, bsz, bsz, 1.0, Pm.d(), m, span_of(Pm), blk(TZ, p),
                 bsz, span_of(TZ), 0.0, P2.d(), m, span_of(P2)));
    if (j >= r / nb) {  // D_0 -= P_2 W_bot^T, D_1 = 0, the next block's rows of D
      int64_t loc, cnt, dc;
      dcols(j, &loc, &cnt, &dc);
      if (j0 > 0)
        LLS_TRY(gm(false, true, kDense, kDense, j0, cnt, bsz, -1.0, P2.d(), m, span_of(P2),
                   M.d() + bsz + dc, ldm, ms, 1.0, X + loc * m, m, xs));
      LLS_TRY(inside(xs, X + j0 + loc * m, bsz, cnt, m, "D_1"));
      LLS_TRY(fill_zero(bsz, cnt, X + j0 + loc * m, m, st));
      if (p > 0)
        LLS_TRY(cp(nb, cnt, X + (j0 - nb) + loc * m, m, xs, D1n->d() + dc * nb, nb,
                   span_of(*D1n)));
    }
    if (j == p) {  // C_01 and C_11 of panel p
      if (j0 > 0) {
        LLS_TRY(inside(span_of(Xc), Xc.d(), j0, bsz, m, "C_01 copy"));
        LLS_TRY(inside(xs, X, j0, bsz, m, "C_01"));
        LLS_TRY(copy_cols_reversed(j0, bsz, X, m, Xc.d(), m, st));
        LLS_TRY(axpy_matrix(j0, bsz, -1.0, P2.d(), m, Xc.d(), m, st));
        LLS_TRY(copy_cols_reversed(j0, bsz, Xc.d(), m, X, m, st));
      }
      LLS_TRY(inside(span_of(Tb), Tb.d(), bsz, bsz + L, nb, "block scatter"));
      LLS_TRY(rz_scatter(bsz, M.d(), ldm, Tb.d(), nb, 0, bsz, L, st));
      LLS_TRY(inside(xs, X + j0, bsz, bsz, m, "C_11"));
      LLS_TRY(copy_upper_into(bsz, Tb.d(), nb, X + j0, m, st));
      if (p > 0) std::swap(D1, D1n);
    }
    return ok_status();
  }
  Status op_solve_utb(int64_t i, double* X, const Span& xs) {
    const int64_t k = kk(i), b = bb(i);
    LLS_TRY(gm(true, false, kUnitLower, kDense, b, nrhs, m - k, 1.0, X + k, m, xs, c.d() + k, m,
               span_of(c), 0.0, sp.d(), nb, span_of(sp)));
    LLS_TRY(gm(true, false, kDense, kDense, b, nrhs, b, 1.0, blk(TU, i), nb, span_of(TU), sp.d(), nb,
               span_of(sp), 0.0, sp2.d(), nb, span_of(sp2)));
    LLS_TRY(gm(false, false, kUnitLower, kDense, m - k, nrhs, b, -1.0, X + k, m, xs, sp2.d(), nb,
               span_of(sp2), 1.0, c.d() + k, m, span_of(c)));
    LLS_TRY(gm(true, false, kDense, kDense, b, nrhs, b, 1.0, blk(US, i), nb, span_of(US),
               c.d() + k, m, span_of(c), 0.0, sp.d(), nb, span_of(sp)));
    return cp(b, nrhs, sp.d(), nb, span_of(sp), c.d() + k, m, span_of(c));
  }
  Status op_solve_trsm(int64_t p, double* X, const Span& xs) {
    const int64_t a0 = c0(p), a1 = std::min(c0(p) + w(p), r), kb = a1 - a0;
    LLS_TRY(inside(xs, X + a0, kb, kb, m, "T_11 block"));
    LLS_TRY(inside(span_of(c), c.d() + a0, kb, nrhs, m, "solve block"));
    LLS_TRY(trsm_block(kb, nrhs, X + a0, m, c.d() + a0, m, st));
    return gm(false, false, kDense, kDense, a0, nrhs, kb, -1.0, X, m, xs, c.d() + a0, m,
              span_of(c), 1.0, c.d(), m, span_of(c));
  }

  // ---- the schedule --------------------------------------------------------
  Status run(const std::vector<lls_ooc_action>& acts) {
    int64_t last_pass = -2;
    for (const lls_ooc_action& a : acts) {
      if (a.panel < 0 || a.panel >= P || a.slot < 0 || a.slot >= C ||
          (a.evict >= 0 && a.evict >= P))
        return make_error(LLS_ERR_ARG, "out-of-core schedule entry out of range");
      if (a.kind == LLS_OOC_K_FLUSH) {
        LLS_TRY(store(a.panel, a.slot));
        continue;
      }
      if (a.evict >= 0 && a.store) LLS_TRY(store(a.evict, a.slot));
      if (a.load) LLS_TRY(load(a.panel, a.slot));
      const bool first = a.pass != last_pass;  // the first access of its pass
      last_pass = a.pass;
      double* X = slot(a.slot);
      const Span xs = slot_span(a.slot);
      const int64_t j = a.panel, s = a.step;
      switch (a.kind) {
        case LLS_OOC_K_SAMPLE_ATG: LLS_TRY(op_sample_atg(s, j, X, xs, first)); break;
        case LLS_OOC_K_SAMPLE_AY: LLS_TRY(op_sample_ay(s, j, X, xs, first)); break;
        case LLS_OOC_K_SAMPLE_ATW_AY: LLS_TRY(op_sample_atw_ay(s, j, X, xs, first)); break;
        case LLS_OOC_K_SAMPLE_ATW: LLS_TRY(op_sample_atw(s, j, X, xs, first)); break;
        case LLS_OOC_K_PRODUCT_TWV: LLS_TRY(op_product_twv(s, j, X, xs, first)); break;
        case LLS_OOC_K_UPDATE: LLS_TRY(op_update(s, j, X, xs, first)); break;
        case LLS_OOC_K_SVD: LLS_TRY(op_svd(j, X, xs, first)); break;
        case LLS_OOC_K_NULL_GATHER: LLS_TRY(op_null_gather(s, j, X, xs)); break;
        case LLS_OOC_K_NULL_READ: LLS_TRY(op_null_read(s, j, X, xs, first)); break;
        case LLS_OOC_K_NULL_WRITE: LLS_TRY(op_null_write(s, j, X, xs, first)); break;
        case LLS_OOC_K_SOLVE_UTB: LLS_TRY(op_solve_utb(j, X, xs)); break;
        case LLS_OOC_K_SOLVE_TRSM: LLS_TRY(op_solve_trsm(j, X, xs)); break;
        default: return make_error(LLS_ERR_ARG, "unknown out-of-core action");
      }
    }
    return ok_status();
  }

  // x = V Z [y; 0]: Nullify's reflectors (block 0 first), then each step's
  // V_s and W_V from the last step back.
  Status replay(double* Xh, int64_t ldx) {
    const Span zs = span_of(Z), cs = span_of(c);
    LLS_TRY(cp(r, nrhs, c.d(), m, cs, Z.d(), n, zs));
    if (r < n) {
      LLS_TRY(inside(zs, Z.d() + r, n - r, nrhs, n, "z tail"));
      LLS_TRY(fill_zero(n - r, nrhs, Z.d() + r, n, st));
    }
    if (nullify && r < n) {
      const int64_t blocks = (r - 1) / nb + 1;
      for (int64_t p = 0; p < blocks; ++p) {
        const int64_t j0 = blk_j0(p), bsz = blk_size(p), ldm = bsz + L;
        const Span ms = span_of(M);
        LLS_TRY(inside(ms, M.d(), ldm, bsz, ldm, "Nullify panel"));
        LLS_CUDA(cudaMemcpyAsync(M.d(), RZh.p + rz_off[(size_t)p], sizeof(double) * ldm * bsz,
                                 cudaMemcpyHostToDevice, st));
        LLS_TRY(inside(zs, Z.d() + j0, bsz, nrhs, n, "z block"));
        LLS_TRY(inside(span_of(zc), zc.d(), bsz, nrhs, bsz, "z copy"));
        LLS_TRY(copy_rows_reversed(bsz, nrhs, Z.d() + j0, n, zc.d(), bsz, st));
        LLS_TRY(cp(bsz, nrhs, zc.d(), bsz, span_of(zc), sp.d(), bsz, span_of(sp)));
        LLS_TRY(gm(true, false, kDense, kDense, bsz, nrhs, L, 1.0, M.d() + bsz, ldm, ms,
                   Z.d() + r, n, zs, 1.0, sp.d(), bsz, span_of(sp)));
        LLS_TRY(gm(false, false, kDense, kDense, bsz, nrhs, bsz, 1.0, blk(TZ, p), bsz, span_of(TZ),
                   sp.d(), bsz, span_of(sp), 0.0, sp2.d(), bsz, span_of(sp2)));
        LLS_TRY(axpy_matrix(bsz, nrhs, -1.0, sp2.d(), bsz, zc.d(), bsz, st));
        LLS_TRY(gm(false, false, kDense, kDense, L, nrhs, bsz, -1.0, M.d() + bsz, ldm, ms,
                   sp2.d(), bsz, span_of(sp2), 1.0, Z.d() + r, n, zs));
        LLS_TRY(copy_rows_reversed(bsz, nrhs, zc.d(), bsz, Z.d() + j0, n, st));
      }
    }
    for (int64_t i = steps - 1; i >= 0; --i) {
      const int64_t k = kk(i), b = bb(i);
      const Span ys = span_of(*Y);
      LLS_TRY(inside(WVh.span(), WVh.p + k + k * n, n - k, b, n, "host W_V"));
      LLS_TRY(inside(ys, Y->d(), n - k, b, n, "W_V"));
      LLS_CUDA(cudaMemcpy2DAsync(Y->d(), sizeof(double) * n, WVh.p + k + k * n, sizeof(double) * n,
                                 sizeof(double) * (n - k), b, cudaMemcpyHostToDevice, st));
      LLS_TRY(gm(false, false, kDense, kDense, b, nrhs, b, 1.0, blk(VS, i), nb, span_of(VS),
                 Z.d() + k, n, zs, 0.0, sp.d(), nb, span_of(sp)));
      LLS_TRY(cp(b, nrhs, sp.d(), nb, span_of(sp), Z.d() + k, n, zs));
      LLS_TRY(gm(true, false, kUnitLower, kDense, b, nrhs, n - k, 1.0, Y->d(), n, ys, Z.d() + k, n,
                 zs, 0.0, sp.d(), nb, span_of(sp)));
      LLS_TRY(gm(false, false, kDense, kDense, b, nrhs, b, 1.0, blk(TV, i), nb, span_of(TV), sp.d(),
                 nb, span_of(sp), 0.0, sp2.d(), nb, span_of(sp2)));
      LLS_TRY(gm(false, false, kUnitLower, kDense, n - k, nrhs, b, -1.0, Y->d(), n, ys, sp2.d(), nb,
                 span_of(sp2), 1.0, Z.d() + k, n, zs));
    }
    LLS_CUDA(cudaMemcpy2DAsync(Xh, sizeof(double) * ldx, Z.d(), sizeof(double) * n,
                               sizeof(double) * n, nrhs, cudaMemcpyDeviceToHost, st));
    return cuda_status(cudaStreamSynchronize(st), "synchronize");
  }
};

bool all_finite(const double* A, int64_t rows, int64_t cols, int64_t ld) {
  for (int64_t j = 0; j < cols; ++j)
    for (int64_t i = 0; i < rows; ++i)
      if (!std::isfinite(A[i + j * ld])) return false;
  return true;
}

}  // namespace
}  // namespace lls

namespace lls {
namespace {

Status solve_ooc(Handle& h, const double* A, int64_t m, int64_t n, int64_t lda, const double* B,
                 int64_t nrhs, int64_t ldb, double tol, double* X, int64_t ldx, int64_t* rank,
                 int64_t cache_panels, int32_t policy) {
  auto bad = [](int idx, const char* what) { return make_error(LLS_ERR_ARG, what, idx); };
  if (m < 0) return bad(3, "m < 0");
  if (n < 0) return bad(4, "n < 0");
  if (lda < std::max<int64_t>(1, m)) return bad(5, "lda < max(1, m)");
  if (nrhs < 0) return bad(7, "nrhs < 0");
  if (ldb < std::max<int64_t>(1, m)) return bad(8, "ldb < max(1, m)");
  if (tol != tol) return bad(9, "tol is NaN");
  if (ldx < std::max<int64_t>(1, n)) return bad(11, "ldx < max(1, n)");
  if (cache_panels < 1) return bad(13, "cache_panels < 1");
  if (policy != LLS_OOC_FARTHEST && policy != LLS_OOC_LRU) return bad(14, "unknown policy");
  if (m > 0 && n > 0 && !A) return bad(2, "NULL A");
  if (m > 0 && nrhs > 0 && !B) return bad(6, "NULL B");
  if (n > 0 && nrhs > 0 && !X) return bad(10, "NULL X");
  if (h.opt.precision != LLS_FP64 || h.opt.explicit_v || h.opt.max_refine)
    return bad(1, "out-of-core solves run in FP64 without explicit_v or refinement");
  if (rank) *rank = 0;
  if (n == 0 || nrhs == 0) return ok_status();
  if (m == 0) {
    for (int64_t j = 0; j < nrhs; ++j) std::memset(X + j * ldx, 0, sizeof(double) * n);
    return ok_status();
  }
  if (!all_finite(A, m, n, lda)) return make_error(LLS_ERR_NONFINITE, "A has a NaN or Inf entry", 2);
  if (!all_finite(B, m, nrhs, ldb))
    return make_error(LLS_ERR_NONFINITE, "B has a NaN or Inf entry", 6);
  int nb = 0, q = 0;
  effective_nb_q(h.opt, h.tune.get(), m, n, &nb, &q);

  OocSolve o(h);
  o.m = m;
  o.n = n;
  o.nb = nb;
  o.q = q;
  o.seed = h.opt.seed;
  o.nullify = h.opt.nullify != 0;
  o.nrhs = nrhs;
  o.P = (n + nb - 1) / nb;
  o.steps = (std::min(m, n) + nb - 1) / nb;
  o.C = std::min(cache_panels, o.P);
  LLS_TRY(o.Hs.alloc(m * n));
  for (int64_t j = 0; j < n; ++j) std::memcpy(o.Hs.p + j * m, A + j * lda, sizeof(double) * m);
  LLS_TRY(o.setup());

  // phase 1: the step loop and the block SVDs, every modified panel written back
  LLS_TRY(o.run(ooc_schedule_phase(m, n, nb, q, 0, false, o.C, policy, 1)));
  std::vector<double> sig((size_t)(o.steps * nb));
  LLS_CUDA(cudaStreamSynchronize(o.st));
  DevStatus hs{};
  LLS_CUDA(cudaMemcpy(&hs, o.ds, sizeof(DevStatus), cudaMemcpyDeviceToHost));
  if (hs.barrier_err) return make_error(LLS_ERR_TIMEOUT, "a device-side wait timed out");
  if (hs.svd_status) return make_error(LLS_ERR_SVD_NOCONV, "block SVD did not converge");
  LLS_CUDA(cudaMemcpy(sig.data(), o.sigma.d(), sizeof(double) * sig.size(),
                      cudaMemcpyDeviceToHost));
  // Compute_rank on diag(T) = the blocks' singular values
  const double t = tol >= 0.0 ? tol
                              : (double)std::max(m, n) * 2.220446049250313e-16 * std::fabs(sig[0]);
  int64_t r = -1, cnt = 0, pos = 0;
  for (int64_t i = 0; i < o.steps; ++i) {
    for (int64_t e = 0; e < o.bb(i); ++e, ++pos) {
      const double d = std::fabs(sig[(size_t)(i * nb + e)]);
      if (d != d) return make_error(LLS_ERR_NONFINITE, "NaN on the diagonal of T");
      if (d > t) ++cnt;
      else if (r < 0) r = pos;
    }
  }
  if (r < 0) r = pos;
  o.r = r;
  o.rcount = cnt;
  if (rank) *rank = r;
  if (r == 0) {
    for (int64_t j = 0; j < nrhs; ++j) std::memset(X + j * ldx, 0, sizeof(double) * n);
  } else {
    // phase 2: Nullify and the solve's panel reads, from an empty cache
    if (o.nullify && r < n) LLS_TRY(o.setup_nullify());
    LLS_CUDA(cudaMemcpy2DAsync(o.c.d(), sizeof(double) * m, B, sizeof(double) * ldb,
                               sizeof(double) * m, nrhs, cudaMemcpyHostToDevice, o.st));
    LLS_TRY(o.run(ooc_schedule_phase(m, n, nb, q, r, o.nullify, o.C, policy, 2)));
    LLS_TRY(o.replay(X, ldx));
    LLS_CUDA(cudaMemcpy(&hs, o.ds, sizeof(DevStatus), cudaMemcpyDeviceToHost));
    if (hs.barrier_err) return make_error(LLS_ERR_TIMEOUT, "a device-side wait timed out");
  }
  LLS_CUDA(cudaStreamSynchronize(o.st));
  if (r != cnt) return make_error(LLS_WARN_RANK_NONPREFIX, "rank is not a prefix");
  return ok_status();
}

}  // namespace
}  // namespace lls

extern "C" int lls_solve_ooc(lls_handle hh, const double* A, int64_t m, int64_t n, int64_t lda,
                             const double* B, int64_t nrhs, int64_t ldb, double tol, double* X,
                             int64_t ldx, int64_t* rank, int64_t cache_panels, int32_t policy) {
  lls::Handle* h = reinterpret_cast<lls::Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  lls::TraceGuard tg(*h);
  lls::Status s = lls::solve_ooc(*h, A, m, n, lda, B, nrhs, ldb, tol, X, ldx, rank, cache_panels,
                                 policy);
  h->last_arg = s.code != LLS_OK ? s.arg : 0;
  h->last_msg = s.code != LLS_OK ? s.msg : std::string();
  return s.code;
}
