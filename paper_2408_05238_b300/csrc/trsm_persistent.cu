// Triangular solves with T_11 (the r x r upper triangle of the factor, Fig. 4)
// for up to four right-hand sides, as one cooperative launch with a grid
// barrier per 64-row block, using the inverses of the 64 x 64 diagonal blocks
// (trsm_block_inverses): B <- R^{-1} B (blocks bottom to top) or, trans,
// B <- R^{-T} B (top to bottom).
//
// Per block q (rows j0 = 64 q .. j1):
//   -- grid barrier (the block's right-hand side is final) --
//   every CTA forms y_q = op(D_q) c_q itself (D_q staged in shared memory
//   while the barrier waited), then updates its slice of the rows still to
//   be solved: c(i) -= sum_l R(i, j0 + l) y_q(l) for i < j0, or
//   c(i) -= sum_l R(j0 + l, i) y_q(l) for i >= j1 (trans); four threads a row,
//   sixteen terms each, added by two exchanges.
// y_q goes back into B after the next barrier (every CTA has read c_q by
// then), the last block's after a final one.  Launched as kernels, the same
// solve costs two launches a block; here a block costs one barrier.
#include "internal.h"

namespace lls {
namespace {

constexpr int TP_THREADS = 256;
constexpr int TP_BLK = 64;  // the block-inverse size of trsm_block_inverses
constexpr int TP_TPR = 4;   // threads a row in the update
constexpr int TP_ROWS = TP_THREADS / TP_TPR;

struct TrsmArgs {
  int64_t r, ldr, ldb;
  const double* R;
  const double* Dinv;  // 64 x 64 blocks, column-major, zero below the diagonal
  double* B;
  int trans, G, nblk;
  GridBarrier bar;
};

__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

// Starts copying block q's inverse into shared memory (every thread its share).
__device__ __forceinline__ void stage_d(const TrsmArgs& a, int q, double* Ds) {
  const double* D = a.Dinv + (int64_t)q * TP_BLK * TP_BLK;
  for (int e = threadIdx.x; e < TP_BLK * TP_BLK; e += TP_THREADS) cp_async8(Ds + e, D + e);
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int NR>
__global__ void __launch_bounds__(TP_THREADS, 1) trsm_persistent_kernel(TrsmArgs a) {
  __shared__ double Ds[TP_BLK * TP_BLK];
  __shared__ double cs[TP_BLK * NR];
  __shared__ double ys[TP_BLK * NR];
  unsigned int epoch = 0;
  const int t = threadIdx.x;
  int prev_q = -1, prev_kb = 0;
  for (int s = 0; s < a.nblk; ++s) {
    const int q = a.trans ? s : a.nblk - 1 - s;
    const int64_t j0 = (int64_t)q * TP_BLK;
    const int kb = (int)(a.r - j0 < TP_BLK ? a.r - j0 : TP_BLK);
    stage_d(a, q, Ds);
    if (s > 0 && !grid_sync(a.bar, epoch)) {  // c_q is final
      asm volatile("cp.async.wait_all;" ::: "memory");
      return;
    }
    // the previous block's solution into B (everyone has read its c by now)
    if (blockIdx.x == 0 && prev_q >= 0)
      for (int e = t; e < prev_kb * NR; e += TP_THREADS)
        a.B[(int64_t)prev_q * TP_BLK + e % prev_kb + (int64_t)(e / prev_kb) * a.ldb] =
            ys[(e % prev_kb) * NR + e / prev_kb];
    for (int e = t; e < kb * NR; e += TP_THREADS)
      cs[(e % kb) * NR + e / kb] = __ldcg(a.B + j0 + e % kb + (int64_t)(e / kb) * a.ldb);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // y = op(D) c: four threads an entry, every fourth term each
    {
      const int i = t >> 2, lg = t & 3;
      double s1[NR];
#pragma unroll
      for (int c = 0; c < NR; ++c) s1[c] = 0.0;
      if (i < kb) {
        if (!a.trans) {
          for (int l = i + ((lg - i) & 3); l < kb; l += 4) {
            const double d = Ds[i + TP_BLK * l];
#pragma unroll
            for (int c = 0; c < NR; ++c) s1[c] = fma(d, cs[l * NR + c], s1[c]);
          }
        } else {
          for (int l = lg; l <= i; l += 4) {
            const double d = Ds[l + TP_BLK * i];
#pragma unroll
            for (int c = 0; c < NR; ++c) s1[c] = fma(d, cs[l * NR + c], s1[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        s1[c] += __shfl_xor_sync(0xffffffffu, s1[c], 1);
        s1[c] += __shfl_xor_sync(0xffffffffu, s1[c], 2);
      }
      if (i < kb && lg == 0)
#pragma unroll
        for (int c = 0; c < NR; ++c) ys[i * NR + c] = s1[c];
    }
    __syncthreads();
    // update this CTA's slice of the rows still to be solved
    const int64_t from = a.trans ? j0 + kb : 0, to = a.trans ? a.r : j0;
    if (to > from) {
      const int64_t per = (to - from + a.G - 1) / a.G;
      const int64_t lo = from + (int64_t)blockIdx.x * per;
      const int64_t hi = lo + per < to ? lo + per : to;
      const int sub = t & (TP_TPR - 1);
      const int npass = hi > lo ? (int)((hi - lo + TP_ROWS - 1) / TP_ROWS) : 0;
      for (int pass = 0; pass < npass; ++pass) {  // CTA-uniform: the exchanges need every lane
        const int64_t i = lo + (int64_t)pass * TP_ROWS + (t >> 2);
        const bool row = i < hi;
        double acc[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = 0.0;
        if (row) {
          const int l0 = sub * (TP_BLK / TP_TPR);
          if (!a.trans) {
            const double* Rp = a.R + i + (j0 + l0) * a.ldr;
#pragma unroll
            for (int u = 0; u < TP_BLK / TP_TPR; ++u)
              if (l0 + u < kb) {
                const double rv = __ldg(Rp + (int64_t)u * a.ldr);
#pragma unroll
                for (int c = 0; c < NR; ++c) acc[c] = fma(rv, ys[(l0 + u) * NR + c], acc[c]);
              }
          } else {
            const double* Rp = a.R + j0 + l0 + i * a.ldr;
#pragma unroll
            for (int u = 0; u < TP_BLK / TP_TPR; ++u)
              if (l0 + u < kb) {
                const double rv = __ldg(Rp + u);
#pragma unroll
                for (int c = 0; c < NR; ++c) acc[c] = fma(rv, ys[(l0 + u) * NR + c], acc[c]);
              }
          }
        }
#pragma unroll
        for (int c = 0; c < NR; ++c) {
          acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 1);
          acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 2);
        }
        if (row && sub == 0)
#pragma unroll
          for (int c = 0; c < NR; ++c)
            a.B[i + c * a.ldb] = __ldcg(a.B + i + c * a.ldb) - acc[c];
      }
    }
    prev_q = q;
    prev_kb = kb;
    __syncthreads();
  }
  if (!grid_sync(a.bar, epoch)) return;  // the last block's c has been read everywhere
  if (blockIdx.x == 0 && prev_q >= 0)
    for (int e = t; e < prev_kb * NR; e += TP_THREADS)
      a.B[(int64_t)prev_q * TP_BLK + e % prev_kb + (int64_t)(e / prev_kb) * a.ldb] =
          ys[(e % prev_kb) * NR + e / prev_kb];
}

int tp_ctas() {
  static int nsm = -1;
  if (nsm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) nsm = 148;
  }
  return nsm;
}

}  // namespace

Status trsm_upper_inv_persistent(int64_t r, int64_t nrhs, const double* R, int64_t ldr,
                                 const double* Dinv, double* B, int64_t ldb, bool trans,
                                 Scratch scratch, int* err, cudaStream_t st) {
  if (r <= 0 || nrhs <= 0) return ok_status();
  if (nrhs > 4) return make_error(LLS_ERR_ARG, "trsm_upper_inv_persistent: nrhs <= 4");
  if (scratch.bytes < 8) return make_error(LLS_ERR_NOMEM, "trsm_upper_inv_persistent: scratch");
  TrsmArgs a;
  a.r = r;
  a.ldr = ldr;
  a.ldb = ldb;
  a.R = R;
  a.Dinv = Dinv;
  a.B = B;
  a.trans = trans ? 1 : 0;
  a.G = tp_ctas();
  a.nblk = (int)ceil_div(r, TP_BLK);
  a.bar.count = static_cast<unsigned int*>(scratch.ptr);
  a.bar.err = err;
  a.bar.limit = g_barrier_spin_limit.load(std::memory_order_relaxed);
  LLS_CUDA(cudaMemsetAsync(scratch.ptr, 0, 8, st));
  TraceScope ts(kTrTrsmDiag, st, (double)r * r * nrhs, 4.0 * (double)r * r);
  void* args[] = {&a};
  const void* fn = nrhs == 1   ? (const void*)trsm_persistent_kernel<1>
                   : nrhs == 2 ? (const void*)trsm_persistent_kernel<2>
                   : nrhs == 3 ? (const void*)trsm_persistent_kernel<3>
                               : (const void*)trsm_persistent_kernel<4>;
  return coop_launch(fn, a.G, TP_THREADS, args, 0, st);
}

}  // namespace lls

extern "C" int lls_k_trsm_upper_blockinv(int64_t r, int64_t nrhs, const double* R, int64_t ldr,
                                         double* B, int64_t ldb, int trans, void* stream) {
  if (r < 0 || nrhs < 0 || nrhs > lls::kThinMaxRhs || ldr < (r > 1 ? r : 1) ||
      ldb < (r > 1 ? r : 1))
    return LLS_ERR_ARG;
  if (r * nrhs == 0) return LLS_OK;
  if (!R || !B) return LLS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  double* dinv = nullptr;
  int* err = nullptr;  // err[0]: the barrier flag, err[2..3]: the barrier's counter
  int code = LLS_OK;
  if (cudaMallocAsync((void**)&dinv, lls::trsm_inverse_bytes(r), st) != cudaSuccess ||
      cudaMallocAsync((void**)&err, 16, st) != cudaSuccess) {
    code = LLS_ERR_NOMEM;
  } else {
    cudaMemsetAsync(err, 0, 16, st);
    lls::Status s = lls::trsm_block_inverses(r, R, ldr, dinv, st);
    if (s.ok())
      s = nrhs <= 4 ? lls::trsm_upper_inv_persistent(r, nrhs, R, ldr, dinv, B, ldb, trans != 0,
                                                     lls::Scratch{err + 2, 8}, err, st)
                    : lls::trsm_upper_inv(r, nrhs, R, ldr, dinv, B, ldb, trans != 0, st);
    int herr = 0;
    if (s.ok()) {
      cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) s = lls::make_error(LLS_ERR_CUDA, "sync");
    }
    code = s.code;
    if (code == LLS_OK && herr) code = LLS_ERR_TIMEOUT;
  }
  if (dinv) cudaFreeAsync(dinv, st);
  if (err) cudaFreeAsync(err, st);
  return code;
}
