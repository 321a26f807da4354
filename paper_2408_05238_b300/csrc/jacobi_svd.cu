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
#include "lls_kernels.h"

namespace lls {
namespace {

constexpr int SVD_THREADS = 256;
constexpr int SVD_MAX_B = 128;
constexpr int SVD_MAX_SWEEPS = 40;

struct SvdBatch {
  const double* R;
  int64_t ldr, strideR;
  double* sigma;
  int64_t strideS;
  double* U;
  int64_t ldu, strideU;
  double* V;
  int64_t ldv, strideV;
  int* status;  // one int for the whole batch (max over blocks), may be null
  int b, b_last, count;
};

__device__ __forceinline__ void pair_of(int round, int i, int bp, int& p, int& q) {
  // circle method on bp players: player bp-1 is fixed, the rest rotate.
  const int mm = bp - 1;
  if (i == 0) {
    p = mm;
    q = round;
  } else {
    p = (round + i) % mm;
    q = (round - i + mm) % mm;
  }
}

// Rotation (c, s) of Rutishauser's formulas with the divisions and square
// roots replaced by Newton-Raphson iterations (reciprocal r <- r (2 - x r),
// reciprocal square root y <- y (3 - x y^2) / 2, two each from a
// single-precision seed after an exact power-of-two scaling): fewer FP64
// instructions on the SVD's serial path.  c^2 + s^2 = 1 to a few ulps, so the
// accumulated V stays orthogonal to FP64 accuracy.
__device__ __forceinline__ double rcp_newton(double x) {  // x > 0, normal
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  const double m = __longlong_as_double(b - ((long long)e << 52));  // [1, 2)
  double r = (double)(1.0f / (float)m);
  r = r * fma(-m, r, 2.0);
  r = r * fma(-m, r, 2.0);
  return __longlong_as_double(__double_as_longlong(r) - ((long long)e << 52));
}
__device__ __forceinline__ double rsqrt_newton(double x) {  // x >= 1, normal
  const long long b = __double_as_longlong(x);
  const int e2 = ((int)((b >> 52) & 0x7FF) - 1023) & ~1;
  const double m = __longlong_as_double(b - ((long long)e2 << 52));  // [1, 4)
  double y = (double)rsqrtf((float)m);
  y = y * fma(-0.5 * m, y * y, 1.5);
  y = y * fma(-0.5 * m, y * y, 1.5);
  return __longlong_as_double(__double_as_longlong(y) - ((long long)(e2 / 2) << 52));
}
__device__ __forceinline__ void jacobi_rotation(double al, double be, double ga, double& c,
                                                double& sn) {
  const double g2 = fabs(2.0 * ga);
  double t;
  if (g2 < 1e-290 || g2 > 1e290) {  // outside the scaled seeds' range: library path
    const double zeta = (be - al) / (2.0 * ga);
    if (fabs(zeta) > 1e150) t = 0.5 / zeta;
    else t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    c = 1.0 / sqrt(1.0 + t * t);
    sn = c * t;
    return;
  }
  // zeta = (be - al) / (2 ga): the magnitude from the reciprocal, the sign of ga applied
  const double zeta = (ga < 0.0 ? -1.0 : 1.0) * ((be - al) * rcp_newton(g2));
  if (fabs(zeta) > 1e150) {
    t = 0.5 / zeta;
  } else {
    const double d = fma(zeta, zeta, 1.0);
    const double w = d * rsqrt_newton(d);  // sqrt(1 + zeta^2)
    t = copysign(rcp_newton(fabs(zeta) + w), zeta);
  }
  c = rsqrt_newton(fma(t, t, 1.0));
  sn = c * t;
}

__global__ void __launch_bounds__(SVD_THREADS) jacobi_svd_kernel(SvdBatch a) {
  extern __shared__ double As[];  // b x b, leading dimension b
  __shared__ int s_rot;
  __shared__ double s_sig[SVD_MAX_B];
  __shared__ int s_rank[SVD_MAX_B];
  const int prob = blockIdx.x;
  const int b = (prob == a.count - 1) ? a.b_last : a.b;
  if (b <= 0) return;
  const double* R = a.R + prob * a.strideR;
  double* Uo = a.U + prob * a.strideU;
  double* Vo = a.V + prob * a.strideV;
  double* So = a.sigma + prob * a.strideS;
  double* Vw = Uo;  // U's buffer holds the working V until the end
  const int64_t ldw = a.ldu;
  const int t = threadIdx.x;

  for (int idx = t; idx < b * b; idx += SVD_THREADS) {
    int i = idx % b, j = idx / b;
    As[idx] = (i <= j) ? R[i + j * a.ldr] : 0.0;
    Vw[i + j * ldw] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();

  const int bp = b + (b & 1);
  const int npairs = bp / 2;
  int tpp = SVD_THREADS / npairs;  // threads per pair, power of two <= 32
  int pw = 1;
  while (pw * 2 <= tpp && pw * 2 <= 32) pw *= 2;
  tpp = pw;
  const int group = t / tpp, gl = t % tpp;
  const bool active = group < npairs;
  const double tol = sqrt((double)b) * 1.1102230246251565e-16;
  const unsigned mask = 0xffffffffu;

  int sweep = 0;
  for (; sweep < SVD_MAX_SWEEPS; ++sweep) {
    if (t == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < bp - 1; ++round) {
      int p = 0, q = 0;
      if (active) pair_of(round, group, bp, p, q);
      if (p > q) {
        int tmp = p;
        p = q;
        q = tmp;
      }
      const bool valid = active && q < b;  // the padding column (index b) is never rotated
      double al = 0.0, be = 0.0, ga = 0.0;
      if (valid) {
        const double* ap = As + p * b;
        const double* aq = As + q * b;
        for (int r = gl; r < b; r += tpp) {
          double x = ap[r], y = aq[r];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
      }
      for (int o = tpp / 2; o > 0; o >>= 1) {
        al += __shfl_xor_sync(mask, al, o);
        be += __shfl_xor_sync(mask, be, o);
        ga += __shfl_xor_sync(mask, ga, o);
      }
      if (valid && al > 0.0 && be > 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
        double c, s;
        jacobi_rotation(al, be, ga, c, s);
        double* ap = As + p * b;
        double* aq = As + q * b;
        for (int r = gl; r < b; r += tpp) {
          double x = ap[r], y = aq[r];
          ap[r] = c * x - s * y;
          aq[r] = s * x + c * y;
        }
        double* vp = Vw + p * ldw;
        double* vq = Vw + q * ldw;
        for (int r = gl; r < b; r += tpp) {
          double x = vp[r], y = vq[r];
          vp[r] = c * x - s * y;
          vq[r] = s * x + c * y;
        }
        if (gl == 0) s_rot = 1;
      }
      __syncthreads();
    }
    if (!s_rot) break;
    __syncthreads();
  }
  if (t == 0 && a.status && sweep >= SVD_MAX_SWEEPS) atomicExch(a.status, LLS_ERR_SVD_NOCONV);

  // singular values and their descending order (ties broken by index)
  for (int j = t; j < b; j += SVD_THREADS) {
    double s = 0.0;
    for (int r = 0; r < b; ++r) s = fma(As[r + j * b], As[r + j * b], s);
    s_sig[j] = sqrt(s);
  }
  __syncthreads();
  for (int j = t; j < b; j += SVD_THREADS) {
    int rk = 0;
    for (int i = 0; i < b; ++i)
      rk += (s_sig[i] > s_sig[j]) || (s_sig[i] == s_sig[j] && i < j);
    s_rank[j] = rk;
    So[rk] = s_sig[j];
  }
  __syncthreads();
  // V columns to their sorted place, then U = A / sigma (also sorted).
  for (int idx = t; idx < b * b; idx += SVD_THREADS) {
    int i = idx % b, j = idx / b;
    Vo[i + s_rank[j] * a.ldv] = Vw[i + j * ldw];
  }
  __syncthreads();
  for (int idx = t; idx < b * b; idx += SVD_THREADS) {
    int i = idx % b, j = idx / b;
    double s = s_sig[j];
    Uo[i + s_rank[j] * a.ldu] = s > 0.0 ? As[i + j * b] / s : 0.0;
  }
  __syncthreads();
  // Orthonormal completion for zero singular values (they sort last).
  int nz = 0;
  for (int j = 0; j < b; ++j) nz += (s_sig[j] > 0.0);
  double* w = As;  // reuse shared memory: candidate vector (b) + dots (b)
  double* dots = As + b;
  int cand = 0;
  for (int col = nz; col < b; ++col) {
    for (; cand < b; ++cand) {
      for (int i = t; i < b; i += SVD_THREADS) w[i] = (i == cand) ? 1.0 : 0.0;
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int j = t; j < col; j += SVD_THREADS) {
          double d = 0.0;
          for (int i = 0; i < b; ++i) d = fma(Uo[i + j * a.ldu], w[i], d);
          dots[j] = d;
        }
        __syncthreads();
        for (int i = t; i < b; i += SVD_THREADS) {
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
        double inv = 1.0 / sqrt(nn);
        for (int i = t; i < b; i += SVD_THREADS) Uo[i + col * a.ldu] = w[i] * inv;
        __syncthreads();
        ++cand;
        break;
      }
    }
  }
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
