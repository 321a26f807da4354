// Householder QR of a tall panel (unpivoted_QR of Fig. 2: steps a3 and a5)
// and the compact-WY T factor of its reflectors.
//
// The panel (m x n, n <= nb) is factored one column at a time, as in
// Golub & Van Loan Alg. 5.2.1, by G cooperating CTAs, each owning a
// contiguous slab of rows, with reflectors in the LAPACK xLARFG convention
// (beta = -sign(alpha) ||(alpha, x)||, tau = (beta - alpha) / beta,
// v = (1, x / (alpha - beta)); tau = 0 when x = 0).
//
// Main kernel (panel_qr_slab_kernel): each CTA keeps its slab in shared
// memory for the whole panel.  Per column j, before a first grid barrier
// every CTA sums, over its rows below j, x_p^2 and x_p A(p, c) for the
// columns c > j (x = the column below the diagonal, before scaling), and the
// owner of row j publishes that row.  Between the first and a second
// barrier, CTA c mod G adds up column j + c over all CTAs in a fixed order
// (FP64 instructions are scarce on this part, so no CTA repeats another's
// sums) and CTA 0 derives beta, tau and the scale of v.  After it every CTA
// forms w_c = A(j, c) + (x^T A(:, c)) / (alpha - beta) = v^T A(:, c) and
// updates its rows, A(p, c) -= tau w_c v_p.  Partial sums and rows are
// double-buffered by column parity, which the barriers make safe.
//
// Panels whose slabs do not fit in shared memory use panel_qr_kernel, which
// works on the panel in global memory with three barriers per column.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "lls_kernels.h"

namespace lls {
namespace {

constexpr int PQ_THREADS = 256;
constexpr int PQ_MAX_CTAS = kPanelMaxCtas;

struct PanelArgs {
  int64_t m, n, lda, rows_per;
  double* A;
  double* tau;
  GridBarrier bar;
  double* part_ss;    // [G]
  double* part_dot;   // [G * n]
  double* dot_final;  // [n]
};

// Sum of one value per thread (threads >= count contribute 0) in a fixed
// order; the result is returned to every thread.
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = (threadIdx.x < 32 && threadIdx.x < (int)(blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
  if (threadIdx.x < 32) s = warp_sum(s);
  if (threadIdx.x == 0) red[32] = s;
  __syncthreads();
  return red[32];
}

__global__ void __launch_bounds__(PQ_THREADS) panel_qr_kernel(PanelArgs a) {
  unsigned int epoch = 0;  // grid barriers passed by this CTA
  extern __shared__ double smem[];
  double* v_s = smem;               // rows_per
  double* d_s = smem + a.rows_per;  // n
  __shared__ double red[33];
  const int G = gridDim.x, cta = blockIdx.x, t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5, nwarps = PQ_THREADS / 32;
  const int64_t m = a.m, n = a.n, lda = a.lda;
  double* A = a.A;
  const int64_t r0 = (int64_t)cta * a.rows_per;
  const int64_t r1 = min(m, r0 + a.rows_per);
  const int64_t kmax = min(m, n);

  auto own_ss = [&](int64_t j) {
    double s = 0.0;
    for (int64_t p = max(r0, j + 1) + t; p < r1; p += PQ_THREADS) {
      double x = A[p + j * lda];
      s = fma(x, x, s);
    }
    s = block_sum(s, red);
    if (t == 0) a.part_ss[cta] = s;
  };

  if (kmax > 0) own_ss(0);
  if (!grid_sync(a.bar, epoch)) return;

  for (int64_t j = 0; j < kmax; ++j) {
    // ---- 2. reflector scalars (identical in every CTA) and local dots
    double ss = block_sum(t < G ? __ldcg(a.part_ss + t) : 0.0, red);
    const double alpha = __ldcg(A + j + j * lda);
    double tau = 0.0, beta = alpha, scale = 0.0;
    if (ss != 0.0) {
      double sigma = sqrt(ss);
      beta = -copysign(hypot(alpha, sigma), alpha);
      tau = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    const int64_t lo = max(r0, j);
    const int64_t nr = r1 > lo ? r1 - lo : 0;
    for (int64_t p = lo + t; p < r1; p += PQ_THREADS) {
      double v = 1.0;
      if (p > j) {
        v = A[p + j * lda] * scale;
        A[p + j * lda] = v;
      }
      v_s[p - r0] = v;
    }
    __syncthreads();
    for (int64_t c = j + 1 + warp; c < n; c += nwarps) {
      double s = 0.0;
      for (int64_t p = lo + lane; p < r1; p += 32) s = fma(v_s[p - r0], A[p + c * lda], s);
      s = warp_sum(s);
      if (lane == 0) a.part_dot[(int64_t)cta * n + c] = s;
    }
    if (!grid_sync(a.bar, epoch)) return;

    // ---- 3a. cross-CTA reduction of the dot products (column c by CTA c mod G)
    for (int64_t c = j + 1 + cta; c < n; c += G) {
      double s = block_sum(t < G ? __ldcg(a.part_dot + (int64_t)t * n + c) : 0.0, red);
      if (t == 0) a.dot_final[c] = s;
    }
    if (!grid_sync(a.bar, epoch)) return;

    // ---- 3b. rank-1 update of this CTA's rows, then the next column's norm
    for (int64_t c = j + 1 + t; c < n; c += PQ_THREADS) d_s[c] = tau * __ldcg(a.dot_final + c);
    __syncthreads();
    if (tau != 0.0 && nr > 0) {
      const int64_t ncols = n - j - 1;
      for (int64_t idx = t; idx < nr * ncols; idx += PQ_THREADS) {
        int64_t p = lo + idx % nr, c = j + 1 + idx / nr;
        A[p + c * lda] -= d_s[c] * v_s[p - r0];
      }
    }
    if (t == 0 && j >= r0 && j < r1) A[j + j * lda] = beta;
    if (t == 0 && cta == 0) a.tau[j] = tau;
    __syncthreads();
    if (j + 1 < kmax) own_ss(j + 1);
    if (!grid_sync(a.bar, epoch)) return;
  }
}

constexpr int PS_TPC = 4;                  // threads per column
constexpr int PS_THREADS = 128 * PS_TPC;   // columns per panel <= 128

struct SlabArgs {
  int64_t m, lda;
  int n, rows_per, ldsl;
  double* A;
  double* tau;
  GridBarrier bar;
  double* part;  // [2][n][G]: partial sums, column-major over CTAs
  double* rowj;  // [2][n]: row j of the panel when column j is eliminated
  double* totg;  // [2][n + 4]: reduced sums of column j, then tau, beta, scale
};

// Reflector scalars of xLARFG from alpha and ss = ||x||^2 (ss > 0):
// beta = -sign(alpha) sqrt(alpha^2 + ss), tau = (beta - alpha) / beta,
// scale = 1 / (alpha - beta).  One thread computes them on every column, so
// their dependent FP64 chain sits on the panel's critical path and FP64
// instructions are scarce on this part: sqrt and the divisions are replaced
// by Newton-Raphson iterations (reciprocal square root y <- y (3 - d y^2) / 2,
// reciprocal r <- r (2 - d r)), two each, from single-precision seeds, after
// scaling d by an even power of two into [1, 4) (exact, on the exponent bits).
// With beta^2 = alpha^2 + ss to a few ulps the reflector is orthogonal to the
// same order.  Subnormal or huge d takes the library functions instead.
__device__ __forceinline__ void reflector_scalars(double alpha, double ss, double& tau,
                                                  double& beta, double& scale) {
  const double d = fma(alpha, alpha, ss);
  const long long db = __double_as_longlong(d);
  const int ex = (int)((db >> 52) & 0x7FF);
  if (ex < 64 || ex > 1983) {  // outside the range the scaled seeds cover
    beta = -copysign(hypot(alpha, sqrt(ss)), alpha);
    tau = (beta - alpha) / beta;
    scale = 1.0 / (alpha - beta);
    return;
  }
  const int e2 = (ex - 1023) & ~1;                                   // even exponent
  const double dm = __longlong_as_double(db - ((long long)e2 << 52));  // d 2^-e2 in [1, 4)
  double y = (double)rsqrtf((float)dm);
  y = y * fma(-0.5 * dm, y * y, 1.5);
  y = y * fma(-0.5 * dm, y * y, 1.5);                                // 1/sqrt(dm)
  const long long half = (long long)(e2 / 2) << 52;
  const double rn = __longlong_as_double(__double_as_longlong(y) - half);       // 1/nrm
  const double nrm = __longlong_as_double(__double_as_longlong(dm * y) + half);  // sqrt(d)
  const double aa = fabs(alpha);
  beta = -copysign(nrm, alpha);
  tau = fma(aa, rn, 1.0);  // (beta - alpha) / beta = 1 + |alpha| / nrm
  // scale = sign(alpha) / (|alpha| + nrm), with d2 = |alpha| + nrm in [nrm, 2 nrm]
  const double d2 = aa + nrm;
  const long long d2b = __double_as_longlong(d2);
  const int e3 = (int)((d2b >> 52) & 0x7FF) - 1023;
  const double d2m = __longlong_as_double(d2b - ((long long)e3 << 52));  // in [1, 2)
  double r = (double)(1.0f / (float)d2m);
  r = r * fma(-d2m, r, 2.0);
  r = r * fma(-d2m, r, 2.0);
  scale = copysign(__longlong_as_double(__double_as_longlong(r) - ((long long)e3 << 52)), alpha);
}

// Sum of the PS_TPC threads of one column, in a fixed pairing; commutative
// adds make the result bit-identical in all of them.
__device__ __forceinline__ double column_group_sum(double s) {
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  return s;
}

// Range [b, e) of part q of [lo, hi) split in PS_TPC contiguous pieces.
__device__ __forceinline__ void quarter(int lo, int hi, int q, int& b, int& e) {
  const int len = hi > lo ? hi - lo : 0;
  const int step = (len + PS_TPC - 1) / PS_TPC;
  b = min(hi, lo + q * step);
  e = min(hi, b + step);
  if (b > e) b = e;
}

__global__ void __launch_bounds__(PS_THREADS) panel_qr_slab_kernel(SlabArgs a) {
  unsigned int epoch = 0;  // grid barriers passed by this CTA
  extern __shared__ double sm[];
  const int n = a.n, ldsl = a.ldsl;
  double* slab = sm;                          // ldsl x n, column-major
  double* tot = slab + (size_t)ldsl * n;      // [n] reduced sums of this column
  double* roww = tot + n;                     // [n] row j, then tau w_c
  __shared__ double sc[3];                    // tau, beta, scale of the current column
  const int G = gridDim.x, cta = blockIdx.x, t = threadIdx.x;
  const int ci = t / PS_TPC, q = t % PS_TPC;  // column offset and quarter of this thread
  const int64_t m = a.m;
  const int64_t r0 = (int64_t)cta * a.rows_per;
  const int64_t r1 = m < r0 + a.rows_per ? m : r0 + a.rows_per;
  const int nr = r1 > r0 ? (int)(r1 - r0) : 0;
  const int kmax = m < (int64_t)n ? (int)m : n;

  for (int idx = t; idx < nr * n; idx += PS_THREADS) {
    const int p = idx % nr, c = idx / nr;
    slab[p + c * ldsl] = a.A[r0 + p + (int64_t)c * a.lda];
  }
  __syncthreads();

  // Partial sums for column j over this CTA's rows p > j: x^T A(:, j + ci).
  auto publish = [&](int j) {
    const int plo = (int)(j + 1 - r0 <= 0 ? 0 : (j + 1 - r0 >= nr ? nr : j + 1 - r0));
    const int ncol = n - j;
    double s0 = 0.0, s1 = 0.0;
    if (ci < ncol) {
      const double* xc = slab + (size_t)j * ldsl;
      const double* ac = slab + (size_t)(j + ci) * ldsl;
      int pb, pe;
      quarter(plo, nr, q, pb, pe);
      int p = pb;
      for (; p + 1 < pe; p += 2) {
        s0 = fma(xc[p], ac[p], s0);
        s1 = fma(xc[p + 1], ac[p + 1], s1);
      }
      if (p < pe) s0 = fma(xc[p], ac[p], s0);
    }
    const double s = column_group_sum(s0 + s1);
    double* P = a.part + (size_t)(j & 1) * n * G;
    if (ci < ncol && q == 0) P[(size_t)(j + ci) * G + cta] = s;
    if (r0 <= j && j < r0 + nr && t < ncol)
      a.rowj[(size_t)(j & 1) * n + j + t] = slab[(j - r0) + (size_t)(j + t) * ldsl];
  };

  if (kmax > 0) publish(0);
  const int warp = t >> 5, lane = t & 31;
  for (int j = 0; j < kmax; ++j) {
    if (!grid_sync(a.bar, epoch)) return;  // partial sums of column j are in
    const int ncol = n - j;
    // ---- column j + c is reduced by CTA c mod G, one warp per column, over
    // the CTAs in a fixed order; CTA 0 also derives the reflector.
    {
      const double* P = a.part + (size_t)(j & 1) * n * G;
      double* TG = a.totg + (size_t)(j & 1) * (n + 4);
      for (int c = cta + warp * G; c < ncol; c += G * (PS_THREADS / 32)) {
        const double* src = P + (size_t)(j + c) * G;
        double v[5];
#pragma unroll
        for (int u = 0; u < 5; ++u) v[u] = (lane + 32 * u < G) ? __ldcg(src + lane + 32 * u) : 0.0;
        double s = v[0];
#pragma unroll
        for (int u = 1; u < 5; ++u)
          if (lane + 32 * u < G) s += v[u];
        for (int g = lane + 160; g < G; g += 32) s += __ldcg(src + g);
        s = warp_sum(s);
        if (lane == 0) {
          TG[j + c] = s;
          if (c == 0) {
            const double alpha = __ldcg(a.rowj + (size_t)(j & 1) * n + j);
            double tau = 0.0, beta = alpha, scale = 0.0;
            if (s != 0.0) reflector_scalars(alpha, s, tau, beta, scale);
            TG[n] = tau;
            TG[n + 1] = beta;
            TG[n + 2] = scale;
          }
        }
      }
    }
    if (!grid_sync(a.bar, epoch)) return;  // totals and the reflector are in
    {
      const double* TG = a.totg + (size_t)(j & 1) * (n + 4);
      if (t < ncol) {
        tot[j + t] = __ldcg(TG + j + t);
        roww[j + t] = __ldcg(a.rowj + (size_t)(j & 1) * n + j + t);
      }
      if (t < 3) sc[t] = __ldcg(TG + n + t);
    }
    __syncthreads();
    const double tau = sc[0], beta = sc[1], scale = sc[2];
    for (int c = j + 1 + t; c < n; c += PS_THREADS) roww[c] = tau * fma(scale, tot[c], roww[c]);
    const int lo = (int)(j - r0 <= 0 ? 0 : (j - r0 >= nr ? nr : j - r0));  // first own row >= j
    const bool own_j = r0 <= j && j < r0 + nr;
    for (int p = lo + (own_j ? 1 : 0) + t; p < nr; p += PS_THREADS) slab[p + (size_t)j * ldsl] *= scale;
    __syncthreads();

    // ---- update of this CTA's rows: A(p, c) -= tau w_c v_p (v_j = 1)
    if (tau != 0.0 && ci + 1 < ncol) {
      const int c = j + 1 + ci;
      const double tw = roww[c];
      double* ac = slab + (size_t)c * ldsl;
      const double* vc = slab + (size_t)j * ldsl;
      int pb, pe;
      quarter(lo, nr, q, pb, pe);
      if (own_j && pb == lo && pb < pe) {
        ac[pb] -= tw;  // row j: v_j = 1
        ++pb;
      }
      for (int p = pb; p < pe; ++p) ac[p] = fma(-tw, vc[p], ac[p]);
    }
    __syncthreads();
    if (own_j && t == 0) slab[lo + (size_t)j * ldsl] = beta;
    if (cta == 0 && t == 0) a.tau[j] = tau;
    __syncthreads();
    if (j + 1 < kmax) publish(j + 1);
  }

  for (int idx = t; idx < nr * n; idx += PS_THREADS) {
    const int p = idx % nr, c = idx / nr;
    a.A[r0 + p + (int64_t)c * a.lda] = slab[p + c * ldsl];
  }
}

// Cluster kernel (panels of up to a few thousand rows): the C CTAs of one
// thread-block cluster (C <= 16) hold the panel in their shared memory and
// exchange partial sums through distributed shared memory, with one hardware
// cluster barrier per column.  A cluster is co-scheduled by construction, so
// this kernel needs no cooperative launch and no grid barrier, and panels of
// different streams run side by side.  Same arithmetic and reduction order
// as the slab kernel (partials per CTA, then in CTA order).
constexpr int PC_MAX_CLUSTER = 8;

struct ClusterArgs {
  int64_t m, lda;
  int n, rows_per, ldsl;
  double* A;
  double* tau;
};

__global__ void __launch_bounds__(PS_THREADS) panel_qr_cluster_kernel(ClusterArgs a) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double sm[];
  const int n = a.n, ldsl = a.ldsl;
  double* slab = sm;                          // ldsl x n, column-major
  double* part = slab + (size_t)ldsl * n;     // [2][n] this CTA's partial sums
  double* rowb = part + 2 * n;                // [2][n] row j, when this CTA owns it
  double* tot = rowb + 2 * n;                 // [n]
  double* roww = tot + n;                     // [n]
  __shared__ double sc[3];
  const int C = (int)cluster.num_blocks(), cr = (int)cluster.block_rank(), t = threadIdx.x;
  const int ci = t / PS_TPC, q = t % PS_TPC;
  const int64_t m = a.m;
  const int64_t r0 = (int64_t)cr * a.rows_per;
  const int64_t r1 = m < r0 + a.rows_per ? m : r0 + a.rows_per;
  const int nr = r1 > r0 ? (int)(r1 - r0) : 0;
  const int kmax = m < (int64_t)n ? (int)m : n;

  for (int idx = t; idx < nr * n; idx += PS_THREADS) {
    const int p = idx % nr, c = idx / nr;
    slab[p + c * ldsl] = a.A[r0 + p + (int64_t)c * a.lda];
  }
  __syncthreads();

  auto publish = [&](int j) {
    const int plo = (int)(j + 1 - r0 <= 0 ? 0 : (j + 1 - r0 >= nr ? nr : j + 1 - r0));
    const int ncol = n - j;
    double s0 = 0.0, s1 = 0.0;
    if (ci < ncol) {
      const double* xc = slab + (size_t)j * ldsl;
      const double* ac = slab + (size_t)(j + ci) * ldsl;
      int pb, pe;
      quarter(plo, nr, q, pb, pe);
      int p = pb;
      for (; p + 1 < pe; p += 2) {
        s0 = fma(xc[p], ac[p], s0);
        s1 = fma(xc[p + 1], ac[p + 1], s1);
      }
      if (p < pe) s0 = fma(xc[p], ac[p], s0);
    }
    const double s = column_group_sum(s0 + s1);
    if (ci < ncol && q == 0) part[(j & 1) * n + j + ci] = s;
    if (r0 <= j && j < r0 + nr && t < ncol)
      rowb[(j & 1) * n + j + t] = slab[(j - r0) + (size_t)(j + t) * ldsl];
  };

  if (kmax > 0) publish(0);
  for (int j = 0; j < kmax; ++j) {
    cluster.sync();  // partial sums (and row j) of column j are in
    const int ncol = n - j;
    const int owner = (int)(j / a.rows_per);
    if (t < ncol) {
      double s = 0.0;
      for (int r = 0; r < C; ++r) s += cluster.map_shared_rank(part, r)[(j & 1) * n + j + t];
      tot[j + t] = s;
      roww[j + t] = cluster.map_shared_rank(rowb, owner)[(j & 1) * n + j + t];
    }
    __syncthreads();
    if (t == 0) {
      const double ss = tot[j], alpha = roww[j];
      double tau = 0.0, beta = alpha, scale = 0.0;
      if (ss != 0.0) reflector_scalars(alpha, ss, tau, beta, scale);
      sc[0] = tau;
      sc[1] = beta;
      sc[2] = scale;
    }
    __syncthreads();
    const double tau = sc[0], beta = sc[1], scale = sc[2];
    for (int c = j + 1 + t; c < n; c += PS_THREADS) roww[c] = tau * fma(scale, tot[c], roww[c]);
    const int lo = (int)(j - r0 <= 0 ? 0 : (j - r0 >= nr ? nr : j - r0));  // first own row >= j
    const bool own_j = r0 <= j && j < r0 + nr;
    for (int p = lo + (own_j ? 1 : 0) + t; p < nr; p += PS_THREADS) slab[p + (size_t)j * ldsl] *= scale;
    __syncthreads();
    if (tau != 0.0 && ci + 1 < ncol) {
      const int c = j + 1 + ci;
      const double tw = roww[c];
      double* ac = slab + (size_t)c * ldsl;
      const double* vc = slab + (size_t)j * ldsl;
      int pb, pe;
      quarter(lo, nr, q, pb, pe);
      if (own_j && pb == lo && pb < pe) {
        ac[pb] -= tw;  // row j: v_j = 1
        ++pb;
      }
      for (int p = pb; p < pe; ++p) ac[p] = fma(-tw, vc[p], ac[p]);
    }
    __syncthreads();
    if (own_j && t == 0) slab[lo + (size_t)j * ldsl] = beta;
    if (cr == 0 && t == 0) a.tau[j] = tau;
    __syncthreads();
    if (j + 1 < kmax) publish(j + 1);
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory

  for (int idx = t; idx < nr * n; idx += PS_THREADS) {
    const int p = idx % nr, c = idx / nr;
    a.A[r0 + p + (int64_t)c * a.lda] = slab[p + c * ldsl];
  }
}

// T factor of the compact WY form: T(j, j) = tau_j and
// T(0:j, j) = -tau_j T(0:j, 0:j) S(0:j, j), S = W^T W (Schreiber-Van Loan).
__global__ void wy_tfactor_kernel(int64_t k, const double* __restrict__ S, int64_t lds,
                                  const double* __restrict__ tau, double* T, int64_t ldt) {
  for (int64_t idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
    int64_t i = idx % k, j = idx / k;
    if (i > j) T[i + j * ldt] = 0.0;
  }
  __syncthreads();
  for (int64_t j = 0; j < k; ++j) {
    const double tj = tau[j];
    for (int64_t i = threadIdx.x; i < j; i += blockDim.x) {
      double s = 0.0;
      for (int64_t l = i; l < j; ++l) s = fma(T[i + l * ldt], S[l + j * lds], s);
      T[i + j * ldt] = -tj * s;
    }
    if (threadIdx.x == 0) T[j + j * ldt] = tj;
    __syncthreads();
  }
}

constexpr int TF_MAX = 128;  // largest k of the register-resident T-factor kernel

// The same recurrence by rows: T(i, j) = -tau_j sum_{l=i}^{j-1} T(i, l) S(l, j)
// needs only row i's own earlier entries, so the rows are independent.  One
// warp per row (rows spread over CTAs, so the FP64 work of k^3/6 multiply-adds
// uses many SMs): lane L keeps T(i, l) for l = L, L + 32, ... in registers,
// each step j sums its lanes' terms and reduces across the warp in a fixed
// order, and lane j mod 32 keeps the new entry.
constexpr int TF_WARPS = 4;

__global__ void __launch_bounds__(TF_WARPS * 32) wy_tfactor_rows_kernel(
    int k, const double* __restrict__ S, int64_t lds, const double* __restrict__ tau, double* T,
    int64_t ldt) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * TF_WARPS + (threadIdx.x >> 5);
  if (i >= k) return;  // whole warps only: k rows, TF_WARPS rows per CTA
  double t[TF_MAX / 32];  // indexed by compile-time u only, so it stays in registers
  const double ti = tau[i];
#pragma unroll
  for (int u = 0; u < TF_MAX / 32; ++u) t[u] = (lane + 32 * u == i) ? ti : 0.0;
  for (int j = i + 1; j < k; ++j) {
    const double* Sj = S + (int64_t)j * lds;
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < TF_MAX / 32; ++u) {
      const int l = lane + 32 * u;
      if (l >= i && l < j) s = fma(t[u], __ldg(Sj + l), s);
    }
    s = warp_sum(s);
    const double tj = -tau[j] * s;
#pragma unroll
    for (int u = 0; u < TF_MAX / 32; ++u)
      if (lane + 32 * u == j) t[u] = tj;
  }
#pragma unroll
  for (int u = 0; u < TF_MAX / 32; ++u) {
    const int l = lane + 32 * u;
    if (l < k) T[i + (int64_t)l * ldt] = l >= i ? t[u] : 0.0;
  }
}

int panel_ctas(int64_t m) {
  static int nsm = -1;
  if (nsm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) nsm = 148;
  }
  int64_t g = std::max<int64_t>(1, ceil_div(m, 32));
  return (int)std::min<int64_t>(g, std::min(nsm, PQ_MAX_CTAS));
}

// Cooperative grids from different streams must not be resident at the same
// time: two partly resident grids could each hold the SM slots the other
// still needs while their CTAs wait at a grid barrier.  Every cooperative
// launch of the library therefore waits (on the device) for the previous one,
// whatever stream issued it; ordinary kernels still overlap freely.
struct CoopGate {
  std::mutex mu;
  int device = -1;
  cudaEvent_t last = nullptr;
};

CoopGate& coop_gate() {
  static CoopGate g;
  return g;
}

int max_dyn_smem() {
  static int bytes = -1;
  if (bytes < 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      v = 48 * 1024;
    bytes = v - 1024;  // room for the kernels' static shared memory
  }
  return bytes;
}

// Slab layout for the shared-memory kernel: rows per CTA, leading dimension
// (odd, to spread columns over banks) and dynamic shared memory.
struct SlabPlan {
  int G, rows_per, ldsl;
  size_t smem;
  bool fits;
};

SlabPlan slab_plan(int64_t m, int64_t n) {
  SlabPlan p;
  p.G = panel_ctas(m);
  p.rows_per = (int)ceil_div(m, p.G);
  p.ldsl = p.rows_per | 1;
  p.smem = sizeof(double) * ((size_t)p.ldsl * n + 2 * (size_t)n);
  p.fits = n <= PS_THREADS / PS_TPC && p.smem <= (size_t)max_dyn_smem();
  return p;
}

}  // namespace

Status coop_launch_gated(const void* fn, int G, int threads, void** args, size_t smem,
                         cudaStream_t st);

// Launches a cooperative kernel behind the library-wide gate.
Status coop_launch(const void* fn, int G, int threads, void** args, size_t smem,
                   cudaStream_t st) {
  LLS_TRY(coop_launch_gated(fn, G, threads, args, smem, st));
  if (g_guard_mode.load(std::memory_order_relaxed)) guard_after_launch("cooperative panel kernel");
  return ok_status();
}

Status coop_launch_gated(const void* fn, int G, int threads, void** args, size_t smem,
                         cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  CoopGate& gate = coop_gate();
  std::lock_guard<std::mutex> lock(gate.mu);
  int dev = 0;
  LLS_CUDA(cudaGetDevice(&dev));
  if (gate.last && gate.device == dev) LLS_CUDA(cudaStreamWaitEvent(st, gate.last, 0));
  LLS_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(threads), args, smem, st));
  if (gate.last && gate.device != dev) {
    cudaEventDestroy(gate.last);
    gate.last = nullptr;
  }
  if (!gate.last) {
    LLS_CUDA(cudaEventCreateWithFlags(&gate.last, cudaEventDisableTiming));
    gate.device = dev;
  }
  LLS_CUDA(cudaEventRecord(gate.last, st));
  return ok_status();
}

namespace {

// Largest cluster the panel kernel may use on this device: 16 CTAs (a
// non-portable size) when the device can hold one such cluster at the
// kernel's maximum shared memory, else the portable 8.
int max_cluster_ctas() {
  static std::once_flag once;
  static int v = PC_MAX_CLUSTER;
  std::call_once(once, [] {
    if (!allow_max_dyn_smem((const void*)panel_qr_cluster_kernel).ok()) return;
    if (cudaFuncSetAttribute(panel_qr_cluster_kernel,
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(PS_THREADS);
    cfg.dynamicSmemBytes = (size_t)max_dyn_smem();
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, panel_qr_cluster_kernel, &cfg) == cudaSuccess &&
        clusters >= 1)
      v = 16;
    cudaGetLastError();
  });
  return v;
}

// Cluster plan: the fewest CTAs (at most max_cluster_ctas(), at least enough
// that each holds <= 64 rows when m allows) whose slabs fit in shared memory.
struct ClusterPlan {
  int C, rows_per, ldsl;
  size_t smem;
  bool fits;
};

ClusterPlan cluster_plan(int64_t m, int64_t n) {
  ClusterPlan p{0, 0, 0, 0, false};
  if (n > PS_THREADS / PS_TPC) return p;
  const int cmax = max_cluster_ctas();
  for (int C = 1; C <= cmax; C *= 2) {
    const int64_t rows = ceil_div(m, C);
    if (rows > 64 && C < cmax) continue;  // spread the FP64 work first
    const int ldsl = (int)(rows | 1);
    const size_t smem = sizeof(double) * ((size_t)ldsl * n + 6 * (size_t)n);
    if (smem <= (size_t)max_dyn_smem()) {
      p = ClusterPlan{C, (int)rows, ldsl, smem, true};
      return p;
    }
  }
  return p;
}

}  // namespace

size_t panel_qr_scratch_bytes(int64_t m, int64_t n) {
  return panel_qr_scratch_layout_bytes(panel_ctas(m), n);
}

Status panel_qr(int64_t m, int64_t n, double* A, int64_t lda, double* tau, Scratch scratch,
                int* err, cudaStream_t st, bool shared_device) {
  if (m <= 0 || n <= 0) return ok_status();
  if (shared_device || m <= kClusterPanelRows || !slab_plan(m, n).fits) {
    const ClusterPlan cp = cluster_plan(m, n);
    if (cp.fits) {
      const int64_t k = std::min(m, n);
      TraceScope ts(kTrPanelQR, st, 2.0 * m * n * k - 2.0 * k * k * k / 3.0, 16.0 * m * n);
      ClusterArgs a{m, lda, (int)n, cp.rows_per, cp.ldsl, A, tau};
      LLS_TRY(allow_max_dyn_smem((const void*)panel_qr_cluster_kernel));
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cp.C);
      cfg.blockDim = dim3(PS_THREADS);
      cfg.dynamicSmemBytes = cp.smem;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = cp.C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      LLS_CUDA(cudaLaunchKernelEx(&cfg, panel_qr_cluster_kernel, a));
      LLS_LAUNCHED("panel_qr_cluster_kernel");
      return ok_status();
    }
  }
  if (scratch.bytes < panel_qr_scratch_bytes(m, n))
    return make_error(LLS_ERR_NOMEM, "panel_qr: scratch too small");
  char* base = static_cast<char*>(scratch.ptr);
  GridBarrier bar;
  bar.count = reinterpret_cast<unsigned int*>(base);
  bar.err = err;
  bar.limit = g_barrier_spin_limit.load(std::memory_order_relaxed);
  double* work = reinterpret_cast<double*>(base + 64);
  const int64_t k = std::min(m, n);
  TraceScope ts(kTrPanelQR, st, 2.0 * m * n * k - 2.0 * k * k * k / 3.0, 16.0 * m * n);
  LLS_CUDA(cudaMemsetAsync(base, 0, 8, st));

  const SlabPlan sp = slab_plan(m, n);
  if (sp.fits) {
    SlabArgs a;
    a.m = m;
    a.lda = lda;
    a.n = (int)n;
    a.rows_per = sp.rows_per;
    a.ldsl = sp.ldsl;
    a.A = A;
    a.tau = tau;
    a.bar = bar;
    a.part = work;
    a.rowj = work + 2 * (size_t)sp.G * n;
    a.totg = a.rowj + 2 * (size_t)n;
    LLS_TRY(allow_max_dyn_smem((const void*)panel_qr_slab_kernel));
    void* args[] = {&a};
    return coop_launch((const void*)panel_qr_slab_kernel, sp.G, PS_THREADS, args, sp.smem, st);
  }

  const int G = panel_ctas(m);
  PanelArgs a;
  a.m = m;
  a.n = n;
  a.lda = lda;
  a.rows_per = ceil_div(m, G);
  a.A = A;
  a.tau = tau;
  a.bar = bar;
  a.part_ss = work;
  a.part_dot = a.part_ss + G;
  a.dot_final = a.part_dot + (size_t)G * n;
  size_t smem = sizeof(double) * (size_t)(a.rows_per + n);
  if (smem > 200 * 1024) return make_error(LLS_ERR_ARG, "panel_qr: panel too tall");
  LLS_TRY(allow_max_dyn_smem((const void*)panel_qr_kernel));
  void* args[] = {&a};
  return coop_launch((const void*)panel_qr_kernel, G, PQ_THREADS, args, smem, st);
}

Status wy_tfactor(int64_t k, const double* S, int64_t lds, const double* tau, double* T,
                  int64_t ldt, cudaStream_t st) {
  if (k <= 0) return ok_status();
  TraceScope ts(kTrTFactor, st, (double)k * k * k / 3.0, 16.0 * k * k);
  if (k <= TF_MAX) {
    wy_tfactor_rows_kernel<<<(unsigned)ceil_div(k, TF_WARPS), TF_WARPS * 32, 0, st>>>(
        (int)k, S, lds, tau, T, ldt);
    LLS_LAUNCHED("wy_tfactor_kernel");
    return ok_status();
  }
  wy_tfactor_kernel<<<1, 256, 0, st>>>(k, S, lds, tau, T, ldt);
  LLS_LAUNCHED("wy_tfactor_kernel");
  return ok_status();
}

}  // namespace lls

extern "C" int lls_k_geqrf(int64_t m, int64_t n, double* A, int64_t lda, double* tau, double* T,
                           int64_t ldt, void* stream) {
  if (m < 0 || n < 0 || lda < (m > 1 ? m : 1)) return LLS_ERR_ARG;
  int64_t k = m < n ? m : n;
  if (k > 0 && (!A || !tau || !T || ldt < k)) return LLS_ERR_ARG;
  if (k == 0) return LLS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  lls::Scratch pq, gs;
  pq.bytes = lls::panel_qr_scratch_bytes(m, n) + 64;
  gs.bytes = lls::gemm_scratch_bytes(k, k, m);
  double* S = nullptr;
  int* err = nullptr;
  int code = LLS_OK;
  if (cudaMallocAsync(&pq.ptr, pq.bytes, st) != cudaSuccess ||
      (gs.bytes && cudaMallocAsync(&gs.ptr, gs.bytes, st) != cudaSuccess) ||
      cudaMallocAsync((void**)&S, sizeof(double) * k * k, st) != cudaSuccess ||
      cudaMallocAsync((void**)&err, sizeof(int), st) != cudaSuccess) {
    code = LLS_ERR_NOMEM;
  } else {
    cudaMemsetAsync(err, 0, sizeof(int), st);
    lls::Status s = lls::panel_qr(m, n, A, lda, tau, pq, err, st);
    if (s.ok())
      s = lls::gemm(true, false, lls::kUnitLower, lls::kUnitLower, k, k, m, 1.0, A, lda, A, lda,
                    0.0, S, k, gs, st);
    if (s.ok()) s = lls::wy_tfactor(k, S, k, tau, T, ldt, st);
    int herr = 0;
    if (s.ok()) {
      cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) s = lls::make_error(LLS_ERR_CUDA, "sync");
    }
    code = s.code;
    if (code == LLS_OK && herr) code = LLS_ERR_TIMEOUT;
  }
  if (pq.ptr) cudaFreeAsync(pq.ptr, st);
  if (gs.ptr) cudaFreeAsync(gs.ptr, st);
  if (S) cudaFreeAsync(S, st);
  if (err) cudaFreeAsync(err, st);
  return code;
}
