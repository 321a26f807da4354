// FP64 GEMM for the dense contractions of randUTV (steps a2, a4, a6 and the
// small products of the SVD, Nullify and solve steps).
//
// sm_103a has no FP64 tensor-core kind (tcgen05 has none, and mma.sync f64
// measured slower than DFMA on B300), so this is a register-blocked DFMA
// kernel: 64 x 64 output tile per CTA, 16-deep K slices staged in shared
// memory, 4 x 4 outputs per thread, the next slice prefetched into
// registers while the current one is consumed.  At ~2 DFMA/clk/SM the FP64
// pipe, not memory, bounds every shape the solver issues (arithmetic
// intensity >= 2 b / 8 flop/byte with b = nb), so the design goal is simply
// to keep that pipe busy: enough CTAs (split-K with a deterministic
// reduction when the output has few tiles) and no stalls on loads.
#include <algorithm>

#include "internal.h"
#include "lls_kernels.h"

namespace lls {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ double load_op(const double* X, int64_t ld, int64_t p, int64_t c,
                                          int mode) {
  // (p, c) index the STORED matrix.
  if (mode == kUnitLower) {
    if (p < c) return 0.0;
    if (p == c) return 1.0;
  }
  return X[p + c * ld];
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(NT) dgemm_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                                                   const double* __restrict__ A, int64_t lda,
                                                   int ma, const double* __restrict__ B,
                                                   int64_t ldb, int mb, double beta,
                                                   double* __restrict__ C, int64_t ldc,
                                                   int64_t kchunk, double* __restrict__ partial) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int t = threadIdx.x;
  const int tx = t % 16, ty = t / 16;
  const int64_t i0 = (int64_t)blockIdx.x * BM;
  const int64_t j0 = (int64_t)blockIdx.y * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = min(K, kbeg + kchunk);

  double ra[4], rb[4];
  auto load_tile = [&](int64_t k0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int i, k;
      if (!TA) {
        i = t % 64;
        k = t / 64 + 4 * e;
      } else {
        k = t % 16;
        i = t / 16 + 16 * e;
      }
      int64_t gi = i0 + i, gk = k0 + k;
      double v = 0.0;
      if (gi < M && gk < kend) v = TA ? load_op(A, lda, gk, gi, ma) : load_op(A, lda, gi, gk, ma);
      ra[e] = v;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int j, k;
      if (!TB) {
        k = t % 16;
        j = t / 16 + 16 * e;
      } else {
        j = t % 64;
        k = t / 64 + 4 * e;
      }
      int64_t gj = j0 + j, gk = k0 + k;
      double v = 0.0;
      if (gj < N && gk < kend) v = TB ? load_op(B, ldb, gj, gk, mb) : load_op(B, ldb, gk, gj, mb);
      rb[e] = v;
    }
  };
  auto store_tile = [&]() {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (!TA) As[t / 64 + 4 * e][t % 64] = ra[e];
      else As[t % 16][t / 16 + 16 * e] = ra[e];
      if (!TB) Bs[t % 16][t / 16 + 16 * e] = rb[e];
      else Bs[t / 64 + 4 * e][t % 64] = rb[e];
    }
  };

  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

  if (kbeg < kend) {
    load_tile(kbeg);
    store_tile();
    __syncthreads();
    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
      const bool more = k0 + BK < kend;
      if (more) load_tile(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
      }
      __syncthreads();
      if (more) {
        store_tile();
        __syncthreads();
      }
    }
  }

  if (partial) {
    double* P = partial + (int64_t)blockIdx.z * M * N;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int64_t gj = j0 + ty + 16 * b;
      if (gj >= N) continue;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        int64_t gi = i0 + tx + 16 * a;
        if (gi < M) P[gi + gj * M] = acc[a][b];
      }
    }
    return;
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    int64_t gj = j0 + ty + 16 * b;
    if (gj >= N) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int64_t gi = i0 + tx + 16 * a;
      if (gi >= M) continue;
      double* c = C + gi + gj * ldc;
      *c = (beta == 0.0) ? alpha * acc[a][b] : fma(alpha, acc[a][b], beta * *c);
    }
  }
}

// Narrow outputs (N <= 16: the right-hand sides of the solve, one block
// column of a factor): a 64 x 64 tile would leave 3/4 of every FMA idle, so
// these use a 128 x 16 tile, 8 outputs per thread (rows r + 32 a, columns
// c + 8 b), and split-K deep enough to put every SM to work.
constexpr int BM2 = 128, BN2 = 16, BK2 = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(NT) dgemm_narrow_kernel(
    int64_t M, int64_t N, int64_t K, double alpha, const double* __restrict__ A, int64_t lda,
    int ma, const double* __restrict__ B, int64_t ldb, int mb, double beta,
    double* __restrict__ C, int64_t ldc, int64_t kchunk, double* __restrict__ partial) {
  __shared__ double As[BK2][BM2 + 1];
  __shared__ double Bs[BK2][BN2 + 1];
  const int t = threadIdx.x;
  const int r = t & 31, c = t >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * BM2;
  const int64_t j0 = (int64_t)blockIdx.y * BN2;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = min(K, kbeg + kchunk);

  double ra[8], rb;
  auto load_tile = [&](int64_t k0) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int i = TA ? t / 16 + 16 * e : t % 128;
      const int k = TA ? t % 16 : t / 128 + 2 * e;
      const int64_t gi = i0 + i, gk = k0 + k;
      double v = 0.0;
      if (gi < M && gk < kend) v = TA ? load_op(A, lda, gk, gi, ma) : load_op(A, lda, gi, gk, ma);
      ra[e] = v;
    }
    const int j = TB ? t % 16 : t / 16;
    const int k = TB ? t / 16 : t % 16;
    const int64_t gj = j0 + j, gk = k0 + k;
    rb = 0.0;
    if (gj < N && gk < kend) rb = TB ? load_op(B, ldb, gj, gk, mb) : load_op(B, ldb, gk, gj, mb);
  };
  auto store_tile = [&]() {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (TA) As[t % 16][t / 16 + 16 * e] = ra[e];
      else As[t / 128 + 2 * e][t % 128] = ra[e];
    }
    if (TB) Bs[t / 16][t % 16] = rb;
    else Bs[t % 16][t / 16] = rb;
  };

  double acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = 0.0;

  if (kbeg < kend) {
    load_tile(kbeg);
    store_tile();
    __syncthreads();
    for (int64_t k0 = kbeg; k0 < kend; k0 += BK2) {
      const bool more = k0 + BK2 < kend;
      if (more) load_tile(k0 + BK2);
#pragma unroll
      for (int kk = 0; kk < BK2; ++kk) {
        const double b0 = Bs[kk][c], b1 = Bs[kk][c + 8];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const double av = As[kk][r + 32 * a];
          acc[a][0] = fma(av, b0, acc[a][0]);
          acc[a][1] = fma(av, b1, acc[a][1]);
        }
      }
      __syncthreads();
      if (more) {
        store_tile();
        __syncthreads();
      }
    }
  }

#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const int64_t gj = j0 + c + 8 * b;
    if (gj >= N) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t gi = i0 + r + 32 * a;
      if (gi >= M) continue;
      if (partial) {
        partial[(int64_t)blockIdx.z * M * N + gi + gj * M] = acc[a][b];
      } else {
        double* cp = C + gi + gj * ldc;
        *cp = (beta == 0.0) ? alpha * acc[a][b] : fma(alpha, acc[a][b], beta * *cp);
      }
    }
  }
}

// Split-K reduction: 32 outputs per CTA (one per lane), warp w summing
// splits w, w + 8, ... in order, then the 8 warp sums in order.  The order is
// fixed, so results do not depend on the launch.
__global__ void __launch_bounds__(256) splitk_reduce_kernel(int64_t M, int64_t N, int splits,
                                                            double alpha,
                                                            const double* __restrict__ partial,
                                                            double beta, double* __restrict__ C,
                                                            int64_t ldc) {
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t idx = (int64_t)blockIdx.x * 32 + lane;
  const int64_t MN = M * N;
  double s = 0.0;
  if (idx < MN)
    for (int z = w; z < splits; z += 8) s += partial[(int64_t)z * MN + idx];
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && idx < MN) {
    double tsum = red[0][lane];
#pragma unroll
    for (int u = 1; u < 8; ++u) tsum += red[u][lane];
    double* cp = C + (idx % M) + (idx / M) * ldc;
    *cp = (beta == 0.0) ? alpha * tsum : fma(alpha, tsum, beta * *cp);
  }
}

__global__ void scale_kernel(int64_t M, int64_t N, double beta, double* C, int64_t ldc) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  double* c = C + (idx % M) + (idx / M) * ldc;
  *c = (beta == 0.0) ? 0.0 : beta * *c;
}

// Enough CTAs to fill 148 SMs several times over: ~3 resident per SM.
constexpr int64_t kTargetCtas = 148 * 12;
constexpr int64_t kMinSplitDepth = 512;
// Narrow tiles: the FP64 pipe is the bound, so ~4 CTAs per SM suffice.
constexpr int64_t kNarrowTargetCtas = 148 * 4;
constexpr int64_t kNarrowMinSplitDepth = 2 * BK2;

struct GemmPlan {
  bool narrow;
  int splits;
};

GemmPlan plan_gemm(int64_t m, int64_t n, int64_t k) {
  GemmPlan p{n <= BN2, 1};
  if (m <= 0 || n <= 0 || k <= 0) return p;
  const int64_t bm = p.narrow ? BM2 : BM, bn = p.narrow ? BN2 : BN;
  const int64_t target = p.narrow ? kNarrowTargetCtas : kTargetCtas;
  const int64_t depth = p.narrow ? kNarrowMinSplitDepth : kMinSplitDepth;
  const int64_t cap = p.narrow ? 512 : 64;
  const int64_t tiles = ceil_div(m, bm) * ceil_div(n, bn);
  if (tiles >= (p.narrow ? 148 : target) || k < 2 * depth) return p;
  int64_t s = ceil_div(target, tiles);
  s = std::min<int64_t>(s, k / depth);
  s = std::min<int64_t>(s, cap);
  p.splits = (int)std::max<int64_t>(s, 1);
  return p;
}

}  // namespace

size_t gemm_scratch_bytes(int64_t m, int64_t n, int64_t k) {
  int s = plan_gemm(m, n, k).splits;
  return s > 1 ? (size_t)s * (size_t)m * (size_t)n * sizeof(double) : 0;
}

Status gemm(bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t m, int64_t n, int64_t k,
            double alpha, const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
            double* C, int64_t ldc, Scratch scratch, cudaStream_t st) {
  if (m <= 0 || n <= 0) return ok_status();
  if (k <= 0 || alpha == 0.0) {
    if (beta == 1.0) return ok_status();
    scale_kernel<<<(unsigned)ceil_div(m * n, 256), 256, 0, st>>>(m, n, beta, C, ldc);
    LLS_LAUNCHED("scale_kernel");
    return ok_status();
  }
  const GemmPlan plan = plan_gemm(m, n, k);
  int splits = plan.splits;
  // The split count is a function of the shape alone (never of the scratch
  // on hand), so the summation order, and with it every bit of the result,
  // is the same whoever calls: a caller must provide gemm_scratch_bytes().
  size_t need = splits > 1 ? (size_t)splits * m * n * sizeof(double) : 0;
  if (need > scratch.bytes)
    return make_error(LLS_ERR_NOMEM, "gemm: split-K scratch smaller than gemm_scratch_bytes()");
  int64_t kchunk = splits > 1 ? ceil_div(ceil_div(k, splits), BK) * BK : k;
  splits = (int)ceil_div(k, kchunk);
  double* partial = splits > 1 ? static_cast<double*>(scratch.ptr) : nullptr;
  dim3 grid((unsigned)ceil_div(m, plan.narrow ? BM2 : BM), (unsigned)ceil_div(n, plan.narrow ? BN2 : BN),
            (unsigned)splits);
  if (grid.y > 65535u) return make_error(LLS_ERR_ARG, "gemm: n too large for grid");
  {
    // algorithmic work: 2 m n k flops; bytes: op(A), op(B) once, C read + written
    TraceScope ts(kTrGemm, st, 2.0 * m * n * k,
                  8.0 * ((double)m * k + (double)k * n + (beta == 0.0 ? 1.0 : 2.0) * m * n));
#define LLS_GEMM_CASE(TA_, TB_)                                                              \
  if (plan.narrow)                                                                           \
    dgemm_narrow_kernel<TA_, TB_><<<grid, NT, 0, st>>>(m, n, k, alpha, A, lda, (int)ma, B,    \
                                                       ldb, (int)mb, beta, C, ldc, kchunk,    \
                                                       partial);                              \
  else                                                                                       \
    dgemm_kernel<TA_, TB_><<<grid, NT, 0, st>>>(m, n, k, alpha, A, lda, (int)ma, B, ldb,      \
                                                (int)mb, beta, C, ldc, kchunk, partial)
  if (!ta && !tb) LLS_GEMM_CASE(false, false);
  else if (!ta && tb) LLS_GEMM_CASE(false, true);
  else if (ta && !tb) LLS_GEMM_CASE(true, false);
  else LLS_GEMM_CASE(true, true);
#undef LLS_GEMM_CASE
    LLS_LAUNCHED("dgemm_kernel");
  }
  if (partial) {
    TraceScope ts(kTrSplitK, st, (double)splits * m * n, 8.0 * (splits + 2.0) * m * n);
    splitk_reduce_kernel<<<(unsigned)ceil_div(m * n, 32), 256, 0, st>>>(m, n, splits, alpha,
                                                                       partial, beta, C, ldc);
    LLS_LAUNCHED("splitk_reduce_kernel");
  }
  return ok_status();
}

}  // namespace lls

extern "C" int lls_k_gemm(int transa, int transb, int unit_lower_a, int unit_lower_b, int64_t m,
                          int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                          const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                          void* stream) {
  if (m < 0 || n < 0 || k < 0) return LLS_ERR_ARG;
  int64_t arows = transa ? k : m, brows = transb ? n : k;
  if (lda < (arows > 1 ? arows : 1) || ldb < (brows > 1 ? brows : 1) || ldc < (m > 1 ? m : 1))
    return LLS_ERR_ARG;
  if (m * n > 0 && (!C || (k > 0 && (!A || !B)))) return LLS_ERR_ARG;
  lls::Scratch s;
  size_t need = lls::gemm_scratch_bytes(m, n, k);
  if (need) {
    if (cudaMallocAsync(&s.ptr, need, (cudaStream_t)stream) != cudaSuccess) return LLS_ERR_NOMEM;
    s.bytes = need;
  }
  lls::Status st = lls::gemm(transa != 0, transb != 0,
                             unit_lower_a ? lls::kUnitLower : lls::kDense,
                             unit_lower_b ? lls::kUnitLower : lls::kDense, m, n, k, alpha, A, lda,
                             B, ldb, beta, C, ldc, s, (cudaStream_t)stream);
  if (s.ptr) cudaFreeAsync(s.ptr, (cudaStream_t)stream);
  return st.code;
}
