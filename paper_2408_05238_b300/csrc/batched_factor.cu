// Persistent batched factorization: randUTV (Fig. 2, steps a1-a7) of many
// small, uneven FP64 problems in ONE kernel launch, after the
// algorithm-by-blocks idea of the paper (Sec. 3.4): each problem's
// factorization is cut into tasks on blocks of its matrices, and any CTA may
// run any task whose inputs are ready.
//
// Per problem the phases are, in order: copy A into T (with the finiteness
// check); per step i (k = i nb, b = min(nb, m - k, n - k)) the sketch G, the
// sample Y = A_BR^T G and q power passes W = A_BR Y, Y = A_BR^T W, the QR of
// Y with its T factor, P = T(:, k:n) W_V and P2 = P T_V by row blocks, the
// right update T(:, k:n) -= P2 W_V^T, the QR of the block column with its T
// factor and R_11, Q2 = T_U^T (W_U^T A_12) by column blocks, the left update
// A_12 -= W_U Q2; then the block SVDs, A_01 V_SVD by row blocks and
// U_SVD^T A_12 by column blocks -- the same operations, in the same order,
// as the solver's step loop (solver.cu), so the factors feed the same rank,
// Nullify and solve.  A phase has one task per 64 x 64 output tile (or row
// or column block) of its product, or a single task for the panel QRs.
//
// Scheduling (device task queue with per-problem dependency counters): one
// 64-bit word per problem holds (phase, tasks claimed); a CTA claims task t
// of a problem's current phase by compare-and-swap, runs it, and counts it in
// the problem's done counter; the CTA that completes the phase's last task
// resets the counter and publishes the next phase with a release store.
// Claims scan the problems in order (the host sorts them by decreasing work,
// so the largest start first), 32 per warp-wide probe.  Tasks never wait for
// each other inside a task, so nothing can deadlock; a CTA that finds no
// claimable task polls with a bounded number of tries and, when they run
// out, raises the error word (LLS_ERR_TIMEOUT) and every CTA exits.
//
// B300's FP64 pipe retires 2 DFMA per clock per SM, so every task is bound by
// it and plain shared-memory tiling reaches it; the win over separate
// launches is that all SMs stay busy across problems whose own phases are
// small or serial (panels, T factors, SVDs).
#include <algorithm>
#include <cstring>

#include "batched_factor.h"
#include "jacobi_block.cuh"
#include "philox.cuh"

namespace lls {
namespace {

constexpr int PB_THREADS = 256;
constexpr int PB_TILE = 64;   // output tile edge (rows and columns)
constexpr int PB_KC = 16;     // K per shared-memory slice of a tile product
constexpr int PB_LDS = 68;    // padded row of a slice
constexpr size_t kPbSmem = 2 * (size_t)PB_TILE * PB_TILE * sizeof(double);  // 64 KB

enum Kind {
  kCopy,
  kSketch,
  kAtG,
  kAy,
  kAtW,
  kQrY,
  kRightP,
  kRightUpd,
  kPanel,
  kLeftQ,
  kLeftUpd,
  kSvd,
  kSvdCols,
  kSvdRows
};

__device__ __forceinline__ int tiles(int x) { return (x + PB_TILE - 1) / PB_TILE; }

struct PhaseInfo {
  int kind, step, k, b, mp, np, ntasks;
};

// Phase `ph` of problem p: what it does and how many tasks it has (a phase
// with nothing to do has one empty task).
__device__ PhaseInfo phase_info(const PBProblem& p, int ph) {
  PhaseInfo f{kCopy, 0, 0, 0, p.m, p.n, tiles(p.m) * tiles(p.n)};
  if (ph == 0) return f;
  const int per = 8 + 2 * p.q;
  int idx = ph - 1;
  if (idx < p.steps * per) {
    const int i = idx / per, r = idx % per;
    f.step = i;
    f.k = i * p.nb;
    f.mp = p.m - f.k;
    f.np = p.n - f.k;
    f.b = min(p.nb, min(f.mp, f.np));
    if (r == 0) f.kind = kSketch;
    else if (r == 1) f.kind = kAtG;
    else if (r < 2 + 2 * p.q) f.kind = ((r - 2) & 1) ? kAtW : kAy;
    else f.kind = kQrY + (r - 2 - 2 * p.q);
    switch (f.kind) {
      case kSketch: case kAy: f.ntasks = tiles(f.mp); break;
      case kAtG: case kAtW: f.ntasks = tiles(f.np); break;
      case kQrY: case kPanel: f.ntasks = 1; break;
      case kRightP: f.ntasks = tiles(p.m); break;
      case kRightUpd: f.ntasks = tiles(p.m) * tiles(f.np); break;
      case kLeftQ: f.ntasks = max(1, tiles(f.np - f.b)); break;
      default: f.ntasks = max(1, tiles(f.mp) * tiles(f.np - f.b)); break;  // kLeftUpd
    }
    return f;
  }
  idx -= p.steps * per;
  f.kind = kSvd + idx;
  if (f.kind == kSvd) {
    f.ntasks = p.steps;
  } else {
    int nt = 0;
    for (int i = 0; i < p.steps; ++i) {
      const int k = i * p.nb, b = min(p.nb, min(p.m - k, p.n - k));
      nt += f.kind == kSvdCols ? tiles(k) : tiles(p.n - k - b);
    }
    f.ntasks = max(1, nt);
  }
  return f;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < PB_THREADS / 32; ++w) s += red[w];  // fixed order
  return s;
}

__device__ __forceinline__ double ld_op(const double* X, int64_t ld, bool ul, int sp, int sc) {
  if (ul) {
    if (sp < sc) return 0.0;
    if (sp == sc) return 1.0;
  }
  return X[sp + (int64_t)sc * ld];
}

// C(r0:r0+64, c0:c0+64) of the M x N matrix C (ld ldc), clipped, =
// alpha op(A) op(B) + beta C with op(A) M x K and op(B) K x N; a stored
// operand flagged ul is read as unit lower trapezoidal.  Fixed summation
// order: K ascending.  All threads of the CTA.
__device__ void tile_gemm(int M, int N, int K, int r0, int c0, bool ta, bool ula, const double* A,
                          int64_t lda, bool tb, bool ulb, const double* B, int64_t ldb,
                          double alpha, double beta, double* C, int64_t ldc, double* sm) {
  double* As = sm;                  // [PB_KC][PB_LDS]: As[kk][ii]
  double* Bs = sm + PB_KC * PB_LDS; // [PB_KC][PB_LDS]: Bs[kk][jj]
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (int k0 = 0; k0 < K; k0 += PB_KC) {
    for (int e = t; e < PB_TILE * PB_KC; e += PB_THREADS) {
      int ii, kk;
      if (!ta) { ii = e % PB_TILE; kk = e / PB_TILE; }
      else { kk = e % PB_KC; ii = e / PB_KC; }
      const int i = r0 + ii, k = k0 + kk;
      As[kk * PB_LDS + ii] =
          (i < M && k < K) ? (ta ? ld_op(A, lda, ula, k, i) : ld_op(A, lda, ula, i, k)) : 0.0;
    }
    for (int e = t; e < PB_TILE * PB_KC; e += PB_THREADS) {
      int jj, kk;
      if (!tb) { kk = e % PB_KC; jj = e / PB_KC; }
      else { jj = e % PB_TILE; kk = e / PB_TILE; }
      const int j = c0 + jj, k = k0 + kk;
      Bs[kk * PB_LDS + jj] =
          (j < N && k < K) ? (tb ? ld_op(B, ldb, ulb, j, k) : ld_op(B, ldb, ulb, k, j)) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < PB_KC; ++kk) {
      double a[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk * PB_LDS + ty * 4 + u];
        bv[u] = Bs[kk * PB_LDS + tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = r0 + ty * 4 + u;
    if (i >= M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = c0 + tx * 4 + v;
      if (j >= N) continue;
      double* c = C + i + (int64_t)j * ldc;
      *c = beta == 0.0 ? alpha * acc[u][v] : fma(alpha, acc[u][v], beta * *c);
    }
  }
}

// Makes this CTA's global writes of one sub-step visible to its own threads
// before the next sub-step reads them.
__device__ __forceinline__ void cta_barrier() {
  __threadfence_block();
  __syncthreads();
}

// Householder QR of the m x b panel A (ld lda) in place, LAPACK xLARFG
// convention (beta = -sign(alpha) ||(alpha, x)||, tau = (beta - alpha) /
// beta, v = (1, x / (alpha - beta)), tau = 0 for x = 0); R in the upper
// triangle, v below the diagonal, tau[min(m, b)].  One CTA.
__device__ void cta_geqrf(int m, int b, double* A, int64_t lda, double* tau, double* red) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int kmax = min(m, b);
  for (int j = 0; j < kmax; ++j) {
    double* aj = A + (int64_t)j * lda;
    double ss = 0.0;
    for (int p = j + 1 + t; p < m; p += PB_THREADS) ss = fma(aj[p], aj[p], ss);
    ss = block_sum(ss, red);
    const double alpha = aj[j];
    double tj = 0.0, beta = alpha, scale = 0.0;
    if (ss != 0.0) {
      beta = -copysign(hypot(alpha, sqrt(ss)), alpha);
      tj = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    __syncthreads();
    for (int p = j + 1 + t; p < m; p += PB_THREADS) aj[p] *= scale;
    cta_barrier();
    for (int c = j + 1 + warp; c < b; c += PB_THREADS / 32) {
      double* ac = A + (int64_t)c * lda;
      double s = 0.0;
      for (int p = j + 1 + lane; p < m; p += 32) s = fma(aj[p], ac[p], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const double w = (ac[j] + s) * tj;
      __syncwarp();
      if (lane == 0) ac[j] -= w;
      for (int p = j + 1 + lane; p < m; p += 32) ac[p] = fma(-w, aj[p], ac[p]);
    }
    if (t == 0) {
      aj[j] = beta;
      tau[j] = tj;
    }
    cta_barrier();
  }
}

// Compact-WY T factor (k x k, ld ldt) of H_0 ... H_{k-1} = I - W T W^T from
// the Gram matrix S = W^T W (ld lds) and tau: T(j, j) = tau_j and
// T(0:j, j) = -tau_j T(0:j, 0:j) S(0:j, j), column by column (T kept in
// shared memory, Ts: k x k).
__device__ void cta_tfactor(int k, const double* S, int64_t lds, const double* tau, double* T,
                            int64_t ldt, double* Ts) {
  const int t = threadIdx.x;
  for (int e = t; e < k * k; e += PB_THREADS) Ts[e] = 0.0;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    const double tj = tau[j];
    if (t < j) {
      double s = 0.0;
      for (int l = t; l < j; ++l) s = fma(Ts[t + l * k], S[l + (int64_t)j * lds], s);
      Ts[t + j * k] = -tj * s;
    }
    if (t == 0) Ts[j + j * k] = tj;
    __syncthreads();
  }
  for (int e = t; e < k * k; e += PB_THREADS) T[(e % k) + (int64_t)(e / k) * ldt] = Ts[e];
}

// X (rows x b block at X, ld ldx) <- X V (V b x b, ld ldv), in place; rows <= 64.
__device__ void cta_right_small(int rows, int b, double* X, int64_t ldx, const double* V,
                                int64_t ldv, double* sm) {
  for (int e = threadIdx.x; e < rows * b; e += PB_THREADS)
    sm[(e % rows) + (e / rows) * PB_TILE] = X[(e % rows) + (int64_t)(e / rows) * ldx];
  __syncthreads();
  for (int e = threadIdx.x; e < rows * b; e += PB_THREADS) {
    const int i = e % rows, j = e / rows;
    double s = 0.0;
    for (int l = 0; l < b; ++l) s = fma(sm[i + l * PB_TILE], V[l + (int64_t)j * ldv], s);
    X[i + (int64_t)j * ldx] = s;
  }
}

// X (b x cols block at X, ld ldx) <- U^T X (U b x b, ld ldu), in place; cols <= 64.
__device__ void cta_left_small_t(int b, int cols, double* X, int64_t ldx, const double* U,
                                 int64_t ldu, double* sm) {
  for (int e = threadIdx.x; e < b * cols; e += PB_THREADS)
    sm[(e % b) + (e / b) * PB_TILE] = X[(e % b) + (int64_t)(e / b) * ldx];
  __syncthreads();
  for (int e = threadIdx.x; e < b * cols; e += PB_THREADS) {
    const int i = e % b, j = e / b;
    double s = 0.0;
    for (int l = 0; l < b; ++l) s = fma(U[l + (int64_t)i * ldu], sm[l + j * PB_TILE], s);
    X[i + (int64_t)j * ldx] = s;
  }
}

// Task `task` of phase `f` of problem `p`.
__device__ void run_task(const PBProblem& p, const PhaseInfo& f, int task, double* sm, double* red) {
  const int m = p.m, n = p.n, nb = p.nb;
  const int64_t ldt = p.ldt, ldw = p.ldw;
  const int k = f.k, b = f.b, mp = f.mp, np = f.np;
  double* ABR = p.T + k + (int64_t)k * ldt;
  double* Y = p.WV + k + (int64_t)k * ldw;
  const size_t blk = (size_t)nb * nb;
  switch (f.kind) {
    case kCopy: {
      const int tr = task % tiles(m), tc = task / tiles(m);
      bool bad = false;
      for (int e = threadIdx.x; e < PB_TILE * PB_TILE; e += PB_THREADS) {
        const int i = tr * PB_TILE + (e % PB_TILE), j = tc * PB_TILE + (e / PB_TILE);
        if (i < m && j < n) {
          const double v = p.A[i + (int64_t)j * p.lda];
          bad |= !isfinite(v);
          p.T[i + (int64_t)j * ldt] = v;
        }
      }
      if (bad) atomicExch(p.flags, 1);
      break;
    }
    case kSketch: {
      // rows 64 task .. +63 of the (m - k) x b sketch of step i: 16 Philox blocks per column
      const int g0 = task * (PB_TILE / 4);
      for (int e = threadIdx.x; e < (PB_TILE / 4) * b; e += PB_THREADS) {
        const int g = g0 + e % (PB_TILE / 4), j = e / (PB_TILE / 4);
        if (4 * g >= mp) continue;
        double z[4];
        rng::block_normals(p.seed, (uint64_t)f.step, (uint64_t)g, (uint64_t)j, z);
#pragma unroll
        for (int w = 0; w < 4; ++w)
          if (4 * g + w < mp) p.G[4 * g + w + (int64_t)j * m] = z[w];
      }
      break;
    }
    case kAtG:  // Y = A_BR^T G
      tile_gemm(np, b, mp, task * PB_TILE, 0, true, false, ABR, ldt, false, false, p.G, m, 1.0, 0.0,
                Y, ldw, sm);
      break;
    case kAy:  // W = A_BR Y
      tile_gemm(mp, b, np, task * PB_TILE, 0, false, false, ABR, ldt, false, false, Y, ldw, 1.0, 0.0,
                p.W, m, sm);
      break;
    case kAtW:  // Y = A_BR^T W
      tile_gemm(np, b, mp, task * PB_TILE, 0, true, false, ABR, ldt, false, false, p.W, m, 1.0, 0.0,
                Y, ldw, sm);
      break;
    case kQrY: {  // [Y, T_V, W_V] = unpivoted_QR(Y)
      double* tauV = p.tauV + (size_t)f.step * nb;
      cta_geqrf(np, b, Y, ldw, tauV, red);
      tile_gemm(b, b, np, 0, 0, true, true, Y, ldw, false, true, Y, ldw, 1.0, 0.0, p.S, nb, sm);
      cta_barrier();
      cta_tfactor(b, p.S, nb, tauV, p.TV + f.step * blk, nb, sm);
      break;
    }
    case kRightP: {  // P = T(:, k:n) W_V, then P2 = P T_V, for 64 rows
      const int r0 = task * PB_TILE;
      tile_gemm(m, b, np, r0, 0, false, false, p.T + (int64_t)k * ldt, ldt, false, true, Y, ldw, 1.0,
                0.0, p.P, m, sm);
      cta_barrier();
      tile_gemm(m, b, b, r0, 0, false, false, p.P, m, false, false, p.TV + f.step * blk, nb, 1.0,
                0.0, p.P2, m, sm);
      break;
    }
    case kRightUpd: {  // T(:, k:n) -= P2 W_V^T
      const int tr = task % tiles(m), tc = task / tiles(m);
      tile_gemm(m, np, b, tr * PB_TILE, tc * PB_TILE, false, false, p.P2, m, true, true, Y, ldw,
                -1.0, 1.0, p.T + (int64_t)k * ldt, ldt, sm);
      break;
    }
    case kPanel: {  // [[A11; A21], T_U, W_U] = unpivoted_QR([A11; A21]); R_11 kept
      double* tauU = p.tauU + (size_t)f.step * nb;
      cta_geqrf(mp, b, ABR, ldt, tauU, red);
      double* R = p.Rblk + f.step * blk;
      for (int e = threadIdx.x; e < b * b; e += PB_THREADS) {
        const int i = e % b, j = e / b;
        R[i + (size_t)j * nb] = i <= j ? ABR[i + (int64_t)j * ldt] : 0.0;
      }
      tile_gemm(b, b, mp, 0, 0, true, true, ABR, ldt, false, true, ABR, ldt, 1.0, 0.0, p.S, nb, sm);
      cta_barrier();
      cta_tfactor(b, p.S, nb, tauU, p.TU + f.step * blk, nb, sm);
      break;
    }
    case kLeftQ: {  // Q = W_U^T A12, Q2 = T_U^T Q, for 64 columns of A12
      if (np <= b) break;
      double* A12 = ABR + (int64_t)b * ldt;
      const int c0 = task * PB_TILE;
      tile_gemm(b, np - b, mp, 0, c0, true, true, ABR, ldt, false, false, A12, ldt, 1.0, 0.0, p.Q,
                nb, sm);
      cta_barrier();
      tile_gemm(b, np - b, b, 0, c0, true, false, p.TU + f.step * blk, nb, false, false, p.Q, nb, 1.0,
                0.0, p.Q2, nb, sm);
      break;
    }
    case kLeftUpd: {  // A12 -= W_U Q2
      if (np <= b) break;
      double* A12 = ABR + (int64_t)b * ldt;
      const int tr = task % tiles(mp), tc = task / tiles(mp);
      tile_gemm(mp, np - b, b, tr * PB_TILE, tc * PB_TILE, false, true, ABR, ldt, false, false, p.Q2,
                nb, -1.0, 1.0, A12, ldt, sm);
      break;
    }
    case kSvd: {  // block SVD of step `task`, then its diagonal block of T = diag(sigma)
      const int i = task, ki = i * nb, bi = min(nb, min(m - ki, n - ki));
      svd::SvdBatch sb;
      sb.R = p.Rblk;
      sb.ldr = nb;
      sb.strideR = blk;
      sb.sigma = p.sigma;
      sb.strideS = nb;
      sb.U = p.US;
      sb.ldu = nb;
      sb.strideU = blk;
      sb.V = p.VS;
      sb.ldv = nb;
      sb.strideV = blk;
      sb.status = p.flags + 1;
      sb.b = nb;
      sb.b_last = bi;
      sb.count = i + 1;  // block i is the last of this one-block view: its size is bi
      svd::jacobi_svd_one(sb, i, sm);
      cta_barrier();
      double* D = p.T + ki + (int64_t)ki * ldt;
      const double* sg = p.sigma + (size_t)i * nb;
      for (int e = threadIdx.x; e < bi * bi; e += PB_THREADS) {
        const int r = e % bi, c = e / bi;
        if (r == c) D[r + (int64_t)c * ldt] = sg[r];
        else if (r < c) D[r + (int64_t)c * ldt] = 0.0;
      }
      break;
    }
    case kSvdCols:
    case kSvdRows: {
      // locate (step, block) of this task
      int rem = task;
      for (int i = 0; i < p.steps; ++i) {
        const int ki = i * nb, bi = min(nb, min(m - ki, n - ki));
        const int nt = f.kind == kSvdCols ? tiles(ki) : tiles(n - ki - bi);
        if (rem < nt) {
          if (f.kind == kSvdCols) {  // A01 <- A01 V_SVD, rows 64 rem .. of columns ki..ki+bi
            const int r0 = rem * PB_TILE;
            cta_right_small(min(PB_TILE, ki - r0), bi, p.T + r0 + (int64_t)ki * ldt, ldt,
                            p.VS + i * blk, nb, sm);
          } else {  // A12 <- U_SVD^T A12, columns 64 rem .. right of the block
            const int c0 = ki + bi + rem * PB_TILE;
            cta_left_small_t(bi, min(PB_TILE, n - c0), p.T + ki + (int64_t)c0 * ldt, ldt,
                             p.US + i * blk, nb, sm);
          }
          break;
        }
        rem -= nt;
      }
      break;
    }
    default:
      break;
  }
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(PB_THREADS, 2) batched_factor_kernel(PBArgs a) {
  extern __shared__ double sm[];
  __shared__ double red[PB_THREADS / 32];
  __shared__ int s_prob, s_phase, s_task, s_exit;
  const int t = threadIdx.x, lane = t & 31;
  long long idle = 0;
  for (;;) {
    if (t < 32) {
      // ---- claim: the first problem (in the host's order) with an unclaimed task
      int prob = -1, phase = 0, task = 0;
      for (int base = 0; base < a.count && prob < 0; base += 32) {
        const int j = base + lane;
        bool can = false;
        unsigned long long w = 0;
        if (j < a.count) {
          w = ld_acquire_u64(a.state + j);
          const int ph = (int)(w >> 32);
          if (ph < a.probs[j].nphases) can = (int)(w & 0xffffffffu) < phase_info(a.probs[j], ph).ntasks;
        }
        unsigned ballot = __ballot_sync(0xffffffffu, can);
        while (ballot && prob < 0) {
          const int src = __ffs(ballot) - 1;
          ballot &= ballot - 1;
          int got = 0, gph = 0, gt = 0;
          if (lane == src) {
            // claim by compare-and-swap; a lost race re-reads the word
            for (int tries = 0; tries < 64; ++tries) {
              const int ph = (int)(w >> 32);
              if (ph >= a.probs[j].nphases) break;
              const int c = (int)(w & 0xffffffffu);
              if (c >= phase_info(a.probs[j], ph).ntasks) break;
              const unsigned long long old = atomicCAS(a.state + j, w, w + 1);
              if (old == w) {
                got = 1;
                gph = ph;
                gt = c;
                break;
              }
              w = old;
            }
            __threadfence();
          }
          got = __shfl_sync(0xffffffffu, got, src);
          if (got) {
            prob = base + src;
            phase = __shfl_sync(0xffffffffu, gph, src);
            task = __shfl_sync(0xffffffffu, gt, src);
          }
        }
      }
      if (lane == 0) {
        s_prob = prob;
        s_phase = phase;
        s_task = task;
        s_exit = 0;
        if (prob < 0) {
          if (ld_acquire_u32(a.finished) >= (unsigned)a.count ||
              *reinterpret_cast<volatile int*>(a.err) != 0) {
            s_exit = 1;
          } else if (++idle > a.poll_limit) {
            atomicExch(a.err, LLS_ERR_TIMEOUT);
            s_exit = 1;
          } else {
            __nanosleep(idle > 64 ? 1000 : 100);
          }
        } else {
          idle = 0;
        }
      }
    }
    __syncthreads();
    if (s_exit) break;
    const int prob = s_prob;
    if (prob < 0) {
      __syncthreads();
      continue;
    }
    const PBProblem& p = a.probs[prob];
    const PhaseInfo f = phase_info(p, s_phase);
    run_task(p, f, s_task, sm, red);
    __threadfence();
    __syncthreads();
    if (t == 0) {
      // the last task of the phase publishes the next phase
      const unsigned d = atomicAdd(a.done + prob, 1u);
      if ((int)d == f.ntasks - 1) {
        a.done[prob] = 0u;
        __threadfence();
        st_release_u64(a.state + prob, (unsigned long long)(s_phase + 1) << 32);
        if (s_phase + 1 == p.nphases) atomicAdd(a.finished, 1u);
      }
    }
    __syncthreads();
  }
}

int num_sms_pb() {
  int dev = 0, n = 148;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

}  // namespace

bool batched_factor_available() { return true; }

int pb_num_phases(int m, int n, int nb, int q) {
  const int steps = (int)ceil_div(std::min(m, n), nb);
  return 1 + steps * (8 + 2 * q) + 3;
}

size_t pb_workspace_doubles(int64_t m, int64_t n, int nb) {
  return 4 * (size_t)m * nb + 2 * (size_t)nb * n + (size_t)nb * nb;
}

Status batched_factor_launch(const PBArgs& args, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    LLS_CUDA(cudaFuncSetAttribute(batched_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kPbSmem));
    attr_set = true;
  }
  int per_sm = 0;
  LLS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_factor_kernel, PB_THREADS,
                                                         kPbSmem));
  const int grid = std::max(1, std::min(per_sm, 2)) * num_sms_pb();
  TraceScope ts(kTrBatchedFactor, st);
  batched_factor_kernel<<<grid, PB_THREADS, kPbSmem, st>>>(args);
  LLS_LAUNCHED("batched_factor_kernel");
  return ok_status();
}

}  // namespace lls
