// Householder QR of a tall panel (unpivoted_QR of Fig. 2: steps a3 and a5)
// and the compact-WY T factor of its reflectors.
//
// The panel (m x n, n <= nb) is factored one column at a time, as in
// Golub & Van Loan Alg. 5.2.1, by G cooperating CTAs, each owning a
// contiguous slab of rows.  Per column j:
//   1. the squared norm of A(j+1:m, j) is summed per CTA and across CTAs;
//   2. every CTA derives beta = -sign(alpha) ||x||, tau = (beta - alpha)/beta
//      and the scaled vector v for its rows (LAPACK xLARFG convention,
//      tau = 0 when the column below the diagonal is zero), then forms its
//      part of the dot products v^T A(:, c) for the columns c > j;
//   3. the dot products are reduced across CTAs (CTA c mod G owns column c)
//      and every CTA updates its rows: A(:, c) -= tau (v^T A(:, c)) v.
// Reductions run in a fixed order, so every CTA derives bit-identical
// scalars and repeated runs are bit-identical.  Cross-CTA steps are joined
// by a bounded grid barrier (common.cuh) inside a cooperative launch.
#include <algorithm>
#include <mutex>

#include "internal.h"
#include "lls_kernels.h"

namespace lls {
namespace {

constexpr int PQ_THREADS = 256;
constexpr int PQ_MAX_CTAS = 256;

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
  if (!grid_sync(a.bar)) return;

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
    if (!grid_sync(a.bar)) return;

    // ---- 3a. cross-CTA reduction of the dot products (column c by CTA c mod G)
    for (int64_t c = j + 1 + cta; c < n; c += G) {
      double s = block_sum(t < G ? __ldcg(a.part_dot + (int64_t)t * n + c) : 0.0, red);
      if (t == 0) a.dot_final[c] = s;
    }
    if (!grid_sync(a.bar)) return;

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
    if (!grid_sync(a.bar)) return;
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

}  // namespace

size_t panel_qr_scratch_bytes(int64_t m, int64_t n) {
  int G = panel_ctas(m);
  return 64 + sizeof(double) * ((size_t)G + (size_t)G * n + (size_t)n);
}

Status panel_qr(int64_t m, int64_t n, double* A, int64_t lda, double* tau, Scratch scratch,
                int* err, cudaStream_t st) {
  if (m <= 0 || n <= 0) return ok_status();
  if (scratch.bytes < panel_qr_scratch_bytes(m, n))
    return make_error(LLS_ERR_NOMEM, "panel_qr: scratch too small");
  int G = panel_ctas(m);
  PanelArgs a;
  a.m = m;
  a.n = n;
  a.lda = lda;
  a.rows_per = ceil_div(m, G);
  a.A = A;
  a.tau = tau;
  char* base = static_cast<char*>(scratch.ptr);
  a.bar.count = reinterpret_cast<unsigned int*>(base);
  a.bar.gen = reinterpret_cast<unsigned int*>(base + 4);
  a.bar.err = err;
  a.part_ss = reinterpret_cast<double*>(base + 64);
  a.part_dot = a.part_ss + G;
  a.dot_final = a.part_dot + (size_t)G * n;
  size_t smem = sizeof(double) * (size_t)(a.rows_per + n);
  if (smem > 200 * 1024) return make_error(LLS_ERR_ARG, "panel_qr: panel too tall");
  LLS_CUDA(cudaMemsetAsync(base, 0, 8, st));
  if (smem > 48 * 1024)
    LLS_CUDA(cudaFuncSetAttribute(panel_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  void* args[] = {&a};
  int64_t k = std::min(m, n);
  TraceScope ts(kTrPanelQR, st, 2.0 * m * n * k - 2.0 * k * k * k / 3.0, 16.0 * m * n);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  CoopGate& gate = coop_gate();
  std::lock_guard<std::mutex> lock(gate.mu);
  int dev = 0;
  LLS_CUDA(cudaGetDevice(&dev));
  if (gate.last && gate.device == dev) LLS_CUDA(cudaStreamWaitEvent(st, gate.last, 0));
  LLS_CUDA(cudaLaunchCooperativeKernel((void*)panel_qr_kernel, dim3(G), dim3(PQ_THREADS), args,
                                       smem, st));
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

Status wy_tfactor(int64_t k, const double* S, int64_t lds, const double* tau, double* T,
                  int64_t ldt, cudaStream_t st) {
  if (k <= 0) return ok_status();
  TraceScope ts(kTrTFactor, st, (double)k * k * k / 3.0, 16.0 * k * k);
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
