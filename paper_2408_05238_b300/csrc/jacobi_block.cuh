// One-sided (Hestenes) Jacobi SVD of one small block on one CTA of
// SVD_THREADS threads: the step shared by the batched SVD launch
// (jacobi_svd.cu) and the persistent batched factorization
// (batched_factor.cu).  See jacobi_svd.cu for the method.
#pragma once

#include <stdint.h>

#include "lls.h"

namespace lls {
namespace svd {

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

// SVD of block `prob` of the batch: R = U diag(sigma) V^T, sigma descending.
// As: b x b doubles of shared memory; all SVD_THREADS threads of the CTA call
// it together.
inline __device__ void jacobi_svd_one(const SvdBatch& a, int prob, double* As) {
  __shared__ int s_rot;
  __shared__ double s_sig[SVD_MAX_B];
  __shared__ int s_rank[SVD_MAX_B];
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

}  // namespace svd
}  // namespace lls
