// Products with few right-hand sides (nrhs <= kThinMaxRhs): the replays of
// the solve of Fig. 4 (c = U^T b by steps, x = V z in reverse step order),
// their transposes (the refinement of the TF32 modes), the off-diagonal
// block updates of the triangular solves, and the FP64 residual products
// A x and A^T r of the refinement.
//
// The general FP64 GEMM tiles N by 16, so one right-hand side costs it the
// FP64 work of sixteen; on this part FP64 runs at 2 FMA per clock per SM,
// and that padding made every such product ALU-bound at 16 times its work.
// These kernels do nrhs columns of work and keep enough loads in flight to
// stream the matrix at HBM speed when nrhs is small:
//  * thin_n_kernel: y(i, c) = sum_k A(i, k) x(k, c).  A CTA owns 64 rows and
//    a K chunk; thread (i, g) of 256 loads A(i, k) for 16 k of each 64-wide
//    k tile (coalesced along i, 16 loads in flight), x staged in shared
//    memory, the four k groups added in a fixed order at the end.
//  * thin_t_kernel: y(j, c) = sum_i A(i, j) x(i, c).  A CTA owns 64 columns,
//    a row chunk and up to 4 right-hand sides; each lane walks rows, 8
//    columns per warp, the 32 lanes added by a fixed shuffle tree.
//  * K or row chunks (a split fixed by the shape alone, so results are
//    bit-identical run to run and handle to handle) write partial sums that
//    thin_reduce_kernel adds in a fixed order.
//  * A replay's b x b singular-vector blocks touch rows that no other step
//    of the replay reads afterwards (or before), so small_blocks_kernel
//    applies all of them in one launch.
// A unit lower trapezoidal operand (the reflector blocks W of a step) reads
// 0 above and 1 on its diagonal, without touching the stored upper part.
#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "warp_sum.cuh"

namespace lls {
namespace {

constexpr int TN_THREADS = 256;
constexpr int TN_ROWS = 64;       // rows per CTA of thin_n_kernel
constexpr int TN_KT = 64;         // k tile
constexpr int TT_COLS = 64;       // columns per CTA of thin_t_kernel
constexpr int TT_CG = 4;          // right-hand sides per CTA of thin_t_kernel (at most)
constexpr int kSplitTarget = 296; // CTAs a split aims for: 2 per SM of a 148-SM part
constexpr int kMinChunkT = 64;    // the shortest row chunk of thin_t_kernel (K <= 64: no split)
// FP64 multiply-adds issue at 2 per clock per SM here, so a product of a few
// hundred thousand of them takes microseconds even when spread over every SM:
// the splits below keep every SM busy down to chunks of one k tile / one row
// per lane rather than amortising per-CTA overheads over long chunks.

// FP64 instructions issue at a small fraction of the other pipes' rate on
// this part, and an instruction predicated off still takes its issue slot,
// so the kernels below are specialised on the number of right-hand sides
// (NR, NC): every FP64 instruction issued does useful work.

template <bool UL>
__device__ __forceinline__ double load_a(const double* __restrict__ A, int64_t lda, int64_t i,
                                         int64_t k) {
  if (UL) {
    if (i < k) return 0.0;
    if (i == k) return 1.0;
  }
  return __ldg(A + i + k * lda);
}

// y = beta y + alpha s without reading y when beta = 0.
__device__ __forceinline__ void store_out(double* y, double alpha, double beta, double s) {
  *y = beta == 0.0 ? alpha * s : fma(beta, *y, alpha * s);
}

template <bool UL, int NR>
__global__ void __launch_bounds__(TN_THREADS) thin_n_kernel(int64_t M, int64_t K,
                                                            const double* __restrict__ A,
                                                            int64_t lda,
                                                            const double* __restrict__ x,
                                                            int64_t ldx, int64_t kchunk,
                                                            double alpha, double beta, double* y,
                                                            int64_t ldy, double* part) {
  __shared__ double xs[TN_KT * NR];
  __shared__ double red[4 * TN_ROWS * NR];
  const int t = threadIdx.x, il = t & (TN_ROWS - 1), kg = t >> 6;
  const int64_t i = (int64_t)blockIdx.x * TN_ROWS + il;
  const int64_t kb = (int64_t)blockIdx.y * kchunk;
  const int64_t ke = std::min<int64_t>(K, kb + kchunk);
  double acc[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) acc[c] = 0.0;
  for (int64_t kt = kb; kt < ke; kt += TN_KT) {
    const int kn = (int)std::min<int64_t>(TN_KT, ke - kt);
    __syncthreads();
    // the k tile of x, zero beyond kn (so the FMAs below need no guard)
    for (int e = t; e < TN_KT * NR; e += TN_THREADS) {
      const int kk = e % TN_KT, c = e / TN_KT;
      xs[e] = kk < kn ? x[kt + kk + (int64_t)c * ldx] : 0.0;
    }
    __syncthreads();
    if (i < M) {
      double a[16];
#pragma unroll
      for (int s = 0; s < 16; ++s) {
        const int kk = kg * 16 + s;
        a[s] = kk < kn ? load_a<UL>(A, lda, i, kt + kk) : 0.0;
      }
#pragma unroll
      for (int s = 0; s < 16; ++s)
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = fma(a[s], xs[kg * 16 + s + TN_KT * c], acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < NR; ++c) red[kg * TN_ROWS * NR + il + TN_ROWS * c] = acc[c];
  __syncthreads();
  for (int e = t; e < TN_ROWS * NR; e += TN_THREADS) {
    const int64_t row = (int64_t)blockIdx.x * TN_ROWS + (e % TN_ROWS);
    if (row >= M) continue;
    const int c = e / TN_ROWS;
    const double s = ((red[e] + red[TN_ROWS * NR + e]) + red[2 * TN_ROWS * NR + e]) +
                     red[3 * TN_ROWS * NR + e];
    if (part)
      part[(int64_t)blockIdx.y * M * NR + (int64_t)c * M + row] = s;
    else
      store_out(y + row + (int64_t)c * ldy, alpha, beta, s);
  }
}

template <bool UL, int NC>
__global__ void __launch_bounds__(TN_THREADS) thin_t_kernel(int64_t M, int64_t K,
                                                            const double* __restrict__ A,
                                                            int64_t lda,
                                                            const double* __restrict__ x,
                                                            int64_t ldx, int cbase, int nrhs,
                                                            int64_t ichunk, double alpha,
                                                            double beta, double* y, int64_t ldy,
                                                            double* part) {
  constexpr int V = 8 * NC;
  constexpr int H = halvings(V) < 5 ? halvings(V) : 5;
  constexpr int R = V >> H;                       // values a lane holds at the end
  constexpr int PLAIN = (1 << (5 - H)) - 1;       // lane bits of the whole-set steps
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t jb = (int64_t)blockIdx.x * TT_COLS + w * 8;
  const int c0 = cbase + blockIdx.z * NC;
  const int64_t ib = (int64_t)blockIdx.y * ichunk;
  const int64_t ie = std::min<int64_t>(K, ib + ichunk);
  double acc[V];
#pragma unroll
  for (int e = 0; e < V; ++e) acc[e] = 0.0;
  const int64_t jn = M - jb;  // columns of this warp that exist: min(8, jn)
#pragma unroll 4
  for (int64_t i = ib + lane; i < ie; i += 32) {
    double xv[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) xv[c] = __ldg(x + i + (int64_t)(c0 + c) * ldx);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double a = u < jn ? load_a<UL>(A, lda, i, jb + u) : 0.0;
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[u * NC + c] = fma(a, xv[c], acc[u * NC + c]);
    }
  }
  int base = 0;
  WarpSumHalves<V, 16>::run(acc, lane, base);
  if ((lane & PLAIN) == 0) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int idx = base + j, u = idx / NC, c = idx % NC;
      if (u >= jn) continue;
      if (part)
        part[(int64_t)blockIdx.y * M * nrhs + (int64_t)(c0 + c) * M + jb + u] = acc[j];
      else
        store_out(y + jb + u + (int64_t)(c0 + c) * ldy, alpha, beta, acc[j]);
    }
  }
}

// y(e) = beta y + alpha sum_g part[g][e] over the M x nrhs entries e = i + c M
// (y(i, c) at y[i + c ldy]): 32 entries per CTA, eight groups of chunks per
// entry summed in a fixed order.
__global__ void __launch_bounds__(256) thin_reduce_kernel(int64_t M, int nrhs, int splits,
                                                          const double* __restrict__ part,
                                                          double alpha, double beta, double* y,
                                                          int64_t ldy) {
  __shared__ double red[8][32];
  const int o = threadIdx.x & 31, gg = threadIdx.x >> 5;
  const int64_t tot = M * nrhs;
  const int64_t e = (int64_t)blockIdx.x * 32 + o;
  double s = 0.0;
  if (e < tot) {
#pragma unroll 4
    for (int g = gg; g < splits; g += 8) s += part[(int64_t)g * tot + e];
  }
  red[gg][o] = s;
  __syncthreads();
  if (gg == 0 && e < tot) {
    double t = red[0][o];
#pragma unroll
    for (int q = 1; q < 8; ++q) t += red[q][o];
    store_out(y + (e % M) + (e / M) * ldy, alpha, beta, t);
  }
}

// Reflector replay, middle step: p2 = op(T) p for the upper triangular b x b T,
// 16 entries of p2 per CTA (grid: ceil(b / 16) x nrhs), eight threads per entry
// (every eighth l each, then three shuffle adds).
__global__ void __launch_bounds__(128) thin_trmv_kernel(int b, const double* __restrict__ p,
                                                        const double* __restrict__ T, int64_t ldt,
                                                        int transT, double* __restrict__ p2) {
  __shared__ double ps[128];
  const int c = blockIdx.y, t = threadIdx.x;
  for (int l = t; l < b; l += 128) ps[l] = p[l + (int64_t)c * b];
  __syncthreads();
  const int i = blockIdx.x * 16 + (t >> 3), lg = t & 7;
  double s = 0.0;
  if (i < b) {
    if (!transT) {
      for (int l = i + ((lg - i) & 7); l < b; l += 8) s = fma(__ldg(T + i + (int64_t)l * ldt), ps[l], s);
    } else {
      for (int l = lg; l <= i; l += 8) s = fma(__ldg(T + l + (int64_t)i * ldt), ps[l], s);
    }
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  if (i < b && lg == 0) p2[i + (int64_t)c * b] = s;
}

// The b x b singular-vector blocks of all steps of a replay in one launch,
// out of place: xo(k + r) = sum_l op(S_i)(r, l) x(k + l) for block i (rows
// k = i nb .. k + b_i, b_i = min(nb, kmax - k), S_i = S + i nb^2 with ld nb).
// Grid: (blocks, ceil(nb / 16), nrhs); 16 rows per CTA, eight threads per row.
__global__ void __launch_bounds__(128) small_blocks_kernel(int nb, int64_t kmax,
                                                           const double* __restrict__ S, int transS,
                                                           const double* __restrict__ x, int64_t ldx,
                                                           double* __restrict__ xo, int64_t ldxo) {
  __shared__ double xs[128];
  const int64_t k = (int64_t)blockIdx.x * nb;
  const int b = (int)(kmax - k < nb ? kmax - k : nb);
  const int c = blockIdx.z, t = threadIdx.x;
  const double* xc = x + k + (int64_t)c * ldx;
  for (int l = t; l < b; l += 128) xs[l] = xc[l];
  __syncthreads();
  const double* Si = S + (int64_t)blockIdx.x * nb * nb;
  const int r = blockIdx.y * 16 + (t >> 3), lg = t & 7;
  double s = 0.0;
  if (r < b) {
    if (!transS) {
      for (int l = lg; l < b; l += 8) s = fma(__ldg(Si + r + (int64_t)l * nb), xs[l], s);
    } else {
      for (int l = lg; l < b; l += 8) s = fma(__ldg(Si + l + (int64_t)r * nb), xs[l], s);
    }
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  if (r < b && lg == 0) xo[k + r + (int64_t)c * ldxo] = s;
}

// x(0:b) <- op(S) x(0:b) for a full b x b block S, one CTA (512 threads) per
// right-hand side, four threads per entry.
__global__ void __launch_bounds__(512) thin_small_mul_kernel(int b, const double* __restrict__ S,
                                                             int64_t lds, int transS, double* x,
                                                             int64_t ldx) {
  __shared__ double xs[128];
  double* xc = x + (int64_t)blockIdx.x * ldx;
  const int t = threadIdx.x, i = t >> 2, lg = t & 3;
  if (t < b) xs[t] = xc[t];
  __syncthreads();
  double s = 0.0;
  if (i < b) {
    if (!transS) {
      for (int l = lg; l < b; l += 4) s = fma(__ldg(S + i + (int64_t)l * lds), xs[l], s);
    } else {
      for (int l = lg; l < b; l += 4) s = fma(__ldg(S + l + (int64_t)i * lds), xs[l], s);
    }
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  __syncthreads();  // every thread has read xs before x is overwritten
  if (i < b && lg == 0) xc[i] = s;
}

struct Split {
  int64_t splits, chunk;
};

// K chunks of thin_n_kernel: a multiple of the k tile, enough of them for
// kSplitTarget CTAs.
Split split_n(int64_t M, int64_t K) {
  const int64_t tiles = ceil_div(M, TN_ROWS);
  int64_t s = std::min(ceil_div(kSplitTarget, tiles), ceil_div(K, TN_KT));
  s = std::max<int64_t>(s, 1);
  const int64_t chunk = ceil_div(ceil_div(K, s), TN_KT) * TN_KT;
  return {ceil_div(K, chunk), chunk};
}

// Row chunks of thin_t_kernel: a multiple of 32 rows, enough of them for
// kSplitTarget CTAs.
Split split_t(int64_t M, int64_t K, int64_t nrhs) {
  const int64_t ctas = ceil_div(M, TT_COLS) * ceil_div(nrhs, TT_CG);
  int64_t s = std::min(ceil_div(kSplitTarget, ctas), ceil_div(K, kMinChunkT));
  s = std::max<int64_t>(s, 1);
  const int64_t chunk = ceil_div(ceil_div(K, s), 32) * 32;
  return {ceil_div(K, chunk), chunk};
}

// Calls f(std::integral_constant<int, N>) for N = n in 1..MAX.
template <int N, int MAX, class F>
void dispatch_count(int n, F&& f) {
  if constexpr (N <= MAX) {
    if (n == N) f(std::integral_constant<int, N>{});
    else dispatch_count<N + 1, MAX>(n, f);
  }
}

template <bool UL>
void launch_n(int64_t M, int64_t K, int nrhs, double alpha, const double* A, int64_t lda,
              const double* x, int64_t ldx, double beta, double* y, int64_t ldy, double* part,
              const Split& sp, cudaStream_t st) {
  const dim3 grid((unsigned)ceil_div(M, TN_ROWS), (unsigned)sp.splits);
  dispatch_count<1, kThinMaxRhs>(nrhs, [&](auto nr) {
    thin_n_kernel<UL, decltype(nr)::value><<<grid, TN_THREADS, 0, st>>>(
        M, K, A, lda, x, ldx, sp.chunk, alpha, beta, y, ldy, part);
  });
}

// nrhs = 4 q + r right-hand sides: q groups of 4 in one launch, the r left
// over in a second.
template <bool UL>
void launch_t(int64_t M, int64_t K, int nrhs, double alpha, const double* A, int64_t lda,
              const double* x, int64_t ldx, double beta, double* y, int64_t ldy, double* part,
              const Split& sp, cudaStream_t st) {
  const int q = nrhs / TT_CG, r = nrhs % TT_CG;
  const unsigned gx = (unsigned)ceil_div(M, TT_COLS), gy = (unsigned)sp.splits;
  if (q > 0)
    thin_t_kernel<UL, TT_CG><<<dim3(gx, gy, (unsigned)q), TN_THREADS, 0, st>>>(
        M, K, A, lda, x, ldx, 0, nrhs, sp.chunk, alpha, beta, y, ldy, part);
  if (r > 0)
    dispatch_count<1, TT_CG - 1>(r, [&](auto nc) {
      thin_t_kernel<UL, decltype(nc)::value><<<dim3(gx, gy, 1), TN_THREADS, 0, st>>>(
          M, K, A, lda, x, ldx, q * TT_CG, nrhs, sp.chunk, alpha, beta, y, ldy, part);
    });
}

// op(A) x into y (alpha, beta) or, with part != nullptr, into the chunks'
// partial sums part[chunk][c][i].
Status launch_thin(bool trans, bool unit_lower, int64_t M, int64_t K, int64_t nrhs, double alpha,
                   const double* A, int64_t lda, const double* x, int64_t ldx, double beta,
                   double* y, int64_t ldy, double* part, const Split& sp, cudaStream_t st) {
  TraceScope ts(trans ? kTrThinT : kTrThinN, st, 2.0 * M * K * nrhs, 8.0 * M * K);
  if (!trans) {
    if (unit_lower)
      launch_n<true>(M, K, (int)nrhs, alpha, A, lda, x, ldx, beta, y, ldy, part, sp, st);
    else
      launch_n<false>(M, K, (int)nrhs, alpha, A, lda, x, ldx, beta, y, ldy, part, sp, st);
    LLS_LAUNCHED("thin_n_kernel");
  } else {
    if (unit_lower)
      launch_t<true>(M, K, (int)nrhs, alpha, A, lda, x, ldx, beta, y, ldy, part, sp, st);
    else
      launch_t<false>(M, K, (int)nrhs, alpha, A, lda, x, ldx, beta, y, ldy, part, sp, st);
    LLS_LAUNCHED("thin_t_kernel");
  }
  return ok_status();
}

Split split_of(bool trans, int64_t M, int64_t K, int64_t nrhs) {
  return trans ? split_t(M, K, nrhs) : split_n(M, K);
}

}  // namespace

size_t thin_gemv_scratch_bytes(bool trans, int64_t M, int64_t K, int64_t nrhs) {
  if (M <= 0 || K <= 0 || nrhs <= 0) return 0;
  const Split sp = split_of(trans, M, K, nrhs);
  return sp.splits > 1 ? sizeof(double) * (size_t)sp.splits * M * nrhs : 0;
}

Status thin_gemv(bool trans, bool unit_lower, int64_t M, int64_t K, int64_t nrhs, double alpha,
                 const double* A, int64_t lda, const double* x, int64_t ldx, double beta, double* y,
                 int64_t ldy, Scratch scratch, cudaStream_t st) {
  if (M <= 0 || nrhs <= 0) return ok_status();
  if (nrhs > kThinMaxRhs) return make_error(LLS_ERR_ARG, "thin_gemv: nrhs <= 16");
  if (K <= 0) {  // y = beta y
    if (beta == 0.0) return fill_zero(M, nrhs, y, ldy, st);
    return beta == 1.0 ? ok_status() : axpy_matrix(M, nrhs, beta - 1.0, y, ldy, y, ldy, st);
  }
  if (ceil_div(M, TN_ROWS) > INT32_MAX) return make_error(LLS_ERR_ARG, "thin_gemv: too many rows");
  const Split sp = split_of(trans, M, K, nrhs);
  if (sp.splits == 1)
    return launch_thin(trans, unit_lower, M, K, nrhs, alpha, A, lda, x, ldx, beta, y, ldy, nullptr,
                       sp, st);
  if (scratch.bytes < thin_gemv_scratch_bytes(trans, M, K, nrhs))
    return make_error(LLS_ERR_NOMEM, "thin_gemv: scratch too small");
  double* part = static_cast<double*>(scratch.ptr);
  LLS_TRY(launch_thin(trans, unit_lower, M, K, nrhs, 1.0, A, lda, x, ldx, 0.0, nullptr, 0, part, sp,
                      st));
  TraceScope ts(kTrThin, st);
  thin_reduce_kernel<<<(unsigned)ceil_div(M * nrhs, 32), 256, 0, st>>>(M, (int)nrhs, (int)sp.splits,
                                                                       part, alpha, beta, y, ldy);
  LLS_LAUNCHED("thin_reduce_kernel");
  return ok_status();
}

size_t thin_scratch_bytes(int64_t M, int64_t b, int64_t nrhs) {
  if (M <= 0 || b <= 0 || nrhs <= 0) return 0;
  const Split sp = split_t(b, M, nrhs);
  return sizeof(double) * ((size_t)sp.splits * b * nrhs + 2 * (size_t)b * nrhs);
}

Status apply_reflectors_thin(int64_t M, int64_t b, int64_t nrhs, const double* W, int64_t ldw,
                             const double* T, int64_t ldt, bool transT, double* x, int64_t ldx,
                             Scratch scratch, cudaStream_t st) {
  if (M <= 0 || b <= 0 || nrhs <= 0) return ok_status();
  if (b > 128 || nrhs > kThinMaxRhs)
    return make_error(LLS_ERR_ARG, "apply_reflectors_thin: b <= 128 and nrhs <= 16");
  if (scratch.bytes < thin_scratch_bytes(M, b, nrhs))
    return make_error(LLS_ERR_NOMEM, "apply_reflectors_thin: scratch too small");
  const Split sp = split_t(b, M, nrhs);
  double* part = static_cast<double*>(scratch.ptr);
  double* p = part + (size_t)sp.splits * b * nrhs;
  double* p2 = p + (size_t)b * nrhs;
  // p = W^T x by row chunks, the chunks summed in order
  LLS_TRY(launch_thin(true, true, b, M, nrhs, 1.0, W, ldw, x, ldx, 0.0, nullptr, 0, part, sp, st));
  {
    TraceScope ts(kTrThin, st);
    thin_reduce_kernel<<<(unsigned)ceil_div(b * nrhs, 32), 256, 0, st>>>(b, (int)nrhs, (int)sp.splits,
                                                                        part, 1.0, 0.0, p, b);
    LLS_LAUNCHED("thin_reduce_kernel");
    // p2 = op(T) p
    thin_trmv_kernel<<<dim3((unsigned)ceil_div(b, 16), (unsigned)nrhs), 128, 0, st>>>(
        (int)b, p, T, ldt, transT ? 1 : 0, p2);
    LLS_LAUNCHED("thin_trmv_kernel");
  }
  // x -= W p2 (K = b <= 128: one K chunk)
  const Split one{1, b};
  return launch_thin(false, true, M, b, nrhs, -1.0, W, ldw, p2, b, 1.0, x, ldx, nullptr, one, st);
}

Status small_blocks_batched(int64_t nblk, int64_t nb, int64_t kmax, int64_t nrhs, const double* S,
                            bool transS, const double* x, int64_t ldx, double* xo, int64_t ldxo,
                            cudaStream_t st) {
  if (nblk <= 0 || nrhs <= 0) return ok_status();
  if (nb > 128) return make_error(LLS_ERR_ARG, "small_blocks_batched: nb <= 128");
  if (nblk > INT32_MAX || nrhs > 65535) return make_error(LLS_ERR_ARG, "small_blocks_batched: size");
  TraceScope ts(kTrThin, st, 2.0 * kmax * nb * nrhs, 8.0 * (double)nblk * nb * nb);
  small_blocks_kernel<<<dim3((unsigned)nblk, (unsigned)ceil_div(nb, 16), (unsigned)nrhs), 128, 0,
                        st>>>((int)nb, kmax, S, transS ? 1 : 0, x, ldx, xo, ldxo);
  LLS_LAUNCHED("small_blocks_kernel");
  return ok_status();
}

Status small_block_mul(int64_t b, int64_t nrhs, const double* S, int64_t lds, bool transS,
                       double* x, int64_t ldx, cudaStream_t st) {
  if (b <= 0 || nrhs <= 0) return ok_status();
  if (b > 128) return make_error(LLS_ERR_ARG, "small_block_mul: b <= 128");
  TraceScope ts(kTrThin, st);
  thin_small_mul_kernel<<<(unsigned)nrhs, 512, 0, st>>>((int)b, S, lds, transS ? 1 : 0, x, ldx);
  LLS_LAUNCHED("thin_small_mul_kernel");
  return ok_status();
}

}  // namespace lls
