// SVD of the small diagonal block (Fig. 2, [A_11, U_SVD, V_SVD] = SVD(A_11);
// step a7) by one-sided (Hestenes) Jacobi: one CTA per block, or, for
// launches with few blocks, one thread-block cluster per block.
//
// The block (b x b, b <= 128) lives in shared memory; column pairs are
// orthogonalized by plane rotations in the parallel round-robin order
// (circle method: b - 1 rounds of b / 2 disjoint pairs per sweep), the
// rotations are accumulated into V.  Rutishauser's formulas:
//   zeta = (||a_q||^2 - ||a_p||^2) / (2 a_p^T a_q),
//   t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = c t
//   (divisions and square roots by Newton iterations, jacobi_rotation),
//   (a_p, a_q) <- (c a_p - s a_q, s a_p + c a_q).
// A pair is rotated when |a_p^T a_q| > sqrt(b) eps ||a_p|| ||a_q||; a sweep
// without a rotation ends the iteration.  Then sigma_j = ||a_j||, U = A V /
// sigma, sorted by descending sigma; columns with sigma = 0 get an
// orthonormal completion (Gram-Schmidt on unit vectors), so U is always
// orthogonal.  Several blocks (one per randUTV step) run in one launch.
#include <cooperative_groups.h>

#include <algorithm>

#include "internal.h"
#include "jacobi_block.cuh"
#include "lls_kernels.h"

namespace lls {
namespace {

using namespace svd;


__global__ void __launch_bounds__(SVD_THREADS) jacobi_svd_kernel(SvdBatch a) {
  extern __shared__ double As[];  // b x b, leading dimension b
  jacobi_svd_one(a, blockIdx.x, As);
}

// The same Jacobi iteration on a thread-block cluster of C CTAs per block,
// for launches with few blocks (a single CTA would leave most SMs idle and
// the sweep is bound by one SM's FP64 pipe).  Column j of A and of V lives in
// the shared memory of CTA j mod C (slot j / C); in each round CTA c's warp w
// takes pair w C + c of the circle order and reads and writes its two columns
// through distributed shared memory; a cluster barrier separates rounds.
// Rotation formulas, threshold, sweep limit, ordering and completion as in
// jacobi_svd_kernel, so both kernels compute the same factorization (up to
// the order of the dot-product sums).
constexpr int SVDC_WARPS = 8;

__global__ void __launch_bounds__(SVDC_WARPS * 32) jacobi_svd_cluster_kernel(SvdBatch a, int ns) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double smc[];
  const int C = (int)cluster.num_blocks(), cr = (int)cluster.block_rank();
  const int prob = blockIdx.x / C;
  const int b = (prob == a.count - 1) ? a.b_last : a.b;
  double* Al = smc;                       // ns columns of A (b doubles each)
  double* Vl = smc + (size_t)ns * SVD_MAX_B;  // ns columns of V
  __shared__ int s_flag;
  __shared__ double s_sig[SVD_MAX_B];  // sigma of the owned columns, at their global index
  __shared__ double s_all[SVD_MAX_B];  // all sigma, gathered
  __shared__ int s_rank[SVD_MAX_B];    // rank of each owned slot
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (b <= 0) return;  // whole cluster: b is the same for all its CTAs
  const double* R = a.R + prob * a.strideR;
  double* Uo = a.U + prob * a.strideU;
  double* Vo = a.V + prob * a.strideV;
  double* So = a.sigma + prob * a.strideS;

  // owned columns j = cr + C s
  for (int idx = t; idx < ns * b; idx += blockDim.x) {
    const int sl = idx / b, i = idx % b, j = cr + C * sl;
    if (j < b) {
      Al[sl * SVD_MAX_B + i] = (i <= j) ? R[i + (int64_t)j * a.ldr] : 0.0;
      Vl[sl * SVD_MAX_B + i] = (i == j) ? 1.0 : 0.0;
    }
  }
  if (t == 0) s_flag = 0;
  cluster.sync();

  const int bp = b + (b & 1);
  const int npairs = bp / 2;
  const double tol = sqrt((double)b) * 1.1102230246251565e-16;
  auto colA = [&](int j) { return cluster.map_shared_rank(Al, j % C) + (j / C) * SVD_MAX_B; };
  auto colV = [&](int j) { return cluster.map_shared_rank(Vl, j % C) + (j / C) * SVD_MAX_B; };

  int sweep = 0;
  for (; sweep < SVD_MAX_SWEEPS; ++sweep) {
    for (int round = 0; round < bp - 1; ++round) {
      const int pi = warp * C + cr;
      if (pi < npairs) {
        int p, q;
        pair_of(round, pi, bp, p, q);
        if (p > q) {
          const int tmp = p;
          p = q;
          q = tmp;
        }
        if (q < b) {  // the padding column (index b) is never rotated
          double* ap = colA(p);
          double* aq = colA(q);
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int r = lane; r < b; r += 32) {
            const double x = ap[r], y = aq[r];
            al = fma(x, x, al);
            be = fma(y, y, be);
            ga = fma(x, y, ga);
          }
          al = warp_sum(al);
          be = warp_sum(be);
          ga = warp_sum(ga);
          if (al > 0.0 && be > 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
            double c = 0.0, sn = 0.0;
            if (lane == 0) jacobi_rotation(al, be, ga, c, sn);
            c = __shfl_sync(0xffffffffu, c, 0);
            sn = __shfl_sync(0xffffffffu, sn, 0);
            for (int r = lane; r < b; r += 32) {
              const double x = ap[r], y = aq[r];
              ap[r] = c * x - sn * y;
              aq[r] = sn * x + c * y;
            }
            double* vp = colV(p);
            double* vq = colV(q);
            for (int r = lane; r < b; r += 32) {
              const double x = vp[r], y = vq[r];
              vp[r] = c * x - sn * y;
              vq[r] = sn * x + c * y;
            }
            if (lane == 0) s_flag = 1;
          }
        }
      }
      cluster.sync();
    }
    // did any CTA rotate in this sweep?
    int any = 0;
    for (int r = 0; r < C; ++r) any |= *cluster.map_shared_rank(&s_flag, r);
    cluster.sync();  // everyone has read the flags before they are reset
    if (t == 0) s_flag = 0;
    __syncthreads();
    if (!any) break;
  }
  if (cr == 0 && t == 0 && a.status && sweep >= SVD_MAX_SWEEPS)
    atomicExch(a.status, LLS_ERR_SVD_NOCONV);

  // sigma of the owned columns, gathered by every CTA for the ordering
  for (int sl = warp; sl < ns; sl += SVDC_WARPS) {
    const int j = cr + C * sl;
    if (j >= b) continue;
    double sq = 0.0;
    for (int r = lane; r < b; r += 32) sq = fma(Al[sl * SVD_MAX_B + r], Al[sl * SVD_MAX_B + r], sq);
    sq = warp_sum(sq);
    if (lane == 0) s_sig[j] = sqrt(sq);  // local copy, owner's slot
  }
  cluster.sync();
  // full sigma vector: column j's value lives in CTA j mod C's s_sig[j]
  for (int j = t; j < b; j += blockDim.x) s_all[j] = *cluster.map_shared_rank(&s_sig[j], j % C);
  __syncthreads();
  for (int sl = t; sl < ns; sl += blockDim.x) {
    const int j = cr + C * sl;
    if (j >= b) continue;
    int rk = 0;
    for (int i = 0; i < b; ++i) rk += (s_all[i] > s_all[j]) || (s_all[i] == s_all[j] && i < j);
    s_rank[sl] = rk;
    So[rk] = s_all[j];
  }
  __syncthreads();
  for (int idx = t; idx < ns * b; idx += blockDim.x) {
    const int sl = idx / b, i = idx % b, j = cr + C * sl;
    if (j >= b) continue;
    const int rk = s_rank[sl];
    const double sg = s_all[j];
    Vo[i + (int64_t)rk * a.ldv] = Vl[sl * SVD_MAX_B + i];
    Uo[i + (int64_t)rk * a.ldu] = sg > 0.0 ? Al[sl * SVD_MAX_B + i] / sg : 0.0;
  }
  cluster.sync();  // U and V written (cluster-scope release/acquire covers global memory)
  if (cr != 0) return;

  // Orthonormal completion for zero singular values (they sort last), by CTA 0.
  int nz = 0;
  for (int j = 0; j < b; ++j) nz += (s_all[j] > 0.0);
  double* w = Al;  // reuse shared memory: candidate vector (b) + dots (b)
  double* dots = Al + SVD_MAX_B;
  int cand = 0;
  for (int col = nz; col < b; ++col) {
    for (; cand < b; ++cand) {
      for (int i = t; i < b; i += blockDim.x) w[i] = (i == cand) ? 1.0 : 0.0;
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int j = t; j < col; j += blockDim.x) {
          double d = 0.0;
          for (int i = 0; i < b; ++i) d = fma(Uo[i + j * a.ldu], w[i], d);
          dots[j] = d;
        }
        __syncthreads();
        for (int i = t; i < b; i += blockDim.x) {
          double x = w[i];
          for (int j = 0; j < col; ++j) x -= dots[j] * Uo[i + j * a.ldu];
          w[i] = x;
        }
        __syncthreads();
      }
      double nn = 0.0;
      for (int i = 0; i < b; ++i) nn = fma(w[i], w[i], nn);
      __syncthreads();
      if (nn > 0.25) {
        const double inv = 1.0 / sqrt(nn);
        for (int i = t; i < b; i += blockDim.x) Uo[i + col * a.ldu] = w[i] * inv;
        __syncthreads();
        ++cand;
        break;
      }
    }
  }
}

}  // namespace

Status jacobi_svd_batched(int count, int b, int b_last, const double* R, int64_t ldr,
                          int64_t strideR, double* sigma, int64_t strideS, double* U, int64_t ldu,
                          int64_t strideU, double* V, int64_t ldv, int64_t strideV, int* status,
                          cudaStream_t st) {
  if (count <= 0) return ok_status();
  if (b > SVD_MAX_B || b_last > SVD_MAX_B) return make_error(LLS_ERR_ARG, "svd: b > 128");
  SvdBatch a{R, ldr, strideR, sigma, strideS, U, ldu, strideU, V, ldv, strideV, status, b, b_last,
             count};
  int bmax = std::max(b, b_last);
  TraceScope ts(kTrSvd, st, 0.0, 8.0 * 3.0 * count * (double)bmax * bmax);
  // Few blocks: spread each over a cluster (C CTAs) so the launch uses more SMs.
  const int C = bmax > 64 ? 8 : 4;
  if (bmax >= 32 && (int64_t)count * C <= 2 * 148) {
    const int ns = (bmax + C - 1) / C;
    const size_t smem = 2 * sizeof(double) * (size_t)ns * SVD_MAX_B;
    LLS_TRY(allow_max_dyn_smem((const void*)jacobi_svd_cluster_kernel));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(count * C));
    cfg.blockDim = dim3(SVDC_WARPS * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    LLS_CUDA(cudaLaunchKernelEx(&cfg, jacobi_svd_cluster_kernel, a, ns));
    LLS_LAUNCHED("jacobi_svd_cluster_kernel");
    return ok_status();
  }
  size_t smem = sizeof(double) * (size_t)std::max(bmax * bmax, 2 * bmax);
  LLS_TRY(allow_max_dyn_smem((const void*)jacobi_svd_kernel));
  jacobi_svd_kernel<<<count, SVD_THREADS, smem, st>>>(a);
  LLS_LAUNCHED("jacobi_svd_kernel");
  return ok_status();
}

Status jacobi_svd(int64_t b, const double* R, int64_t ldr, double* sigma, double* Us, int64_t ldu,
                  double* Vs, int64_t ldv, int* status, cudaStream_t st) {
  return jacobi_svd_batched(1, (int)b, (int)b, R, ldr, 0, sigma, 0, Us, ldu, 0, Vs, ldv, 0,
                            status, st);
}

}  // namespace lls

extern "C" int lls_k_jacobi_svd(int64_t b, const double* R, int64_t ldr, double* sigma, double* Us,
                                int64_t ldu, double* Vs, int64_t ldv, int* status, void* stream) {
  if (b < 0 || b > 128 || ldr < (b > 1 ? b : 1) || ldu < (b > 1 ? b : 1) ||
      ldv < (b > 1 ? b : 1))
    return LLS_ERR_ARG;
  if (b == 0) return LLS_OK;
  if (!R || !sigma || !Us || !Vs) return LLS_ERR_ARG;
  return lls::jacobi_svd(b, R, ldr, sigma, Us, ldu, Vs, ldv, status, (cudaStream_t)stream).code;
}
