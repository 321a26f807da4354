// One replay of a factor's stored block reflectors -- the step loop of the
// solve of Fig. 4 (c = U^T b, x = V z) and of the refinement's operators --
// as a single cooperative launch, for up to four right-hand sides.
//
// Per step i (k = i nb, b columns of reflectors W_i, unit lower, and their
// compact-WY factor T_i): x(k:M) <- (I - W_i op(T_i) W_i^T) x(k:M), with
// op(T) = T^T in U^T / V^T order (steps first to last) and T in U / V order
// (last to first).  Launched as a chain of small kernels each step costs four
// launches whose FP64 work is a few microseconds; here one cooperative grid
// of a CTA per SM runs every step:
//   A  each CTA sums W_i^T x over a slice of the rows (lanes along rows, 16
//      columns a warp, the lanes added by halving exchanges) into its partial;
//   -- grid barrier --
//   B  a warp per entry adds that entry's partials, in a fixed order, into p;
//   -- grid barrier --
//   C  every CTA forms p2 = op(T_i) p itself (the triangle of T_i, staged in
//      shared memory while the barriers wait), so no barrier is needed before
//   D  it updates a slice of the rows, x(r) -= W_i(r, :) p2, and goes straight
//      on to A of the next step over the same slice.
// Two grid barriers a step.  D and the next step's A cover the same rows of
// each CTA (a slice of [min(k_i, k_next), M), re-cut every step so that all
// CTAs keep working as k moves), so the CTA that updated a row is the one
// that reads it next; x, the partials and p go through global memory behind
// the barriers and are read with ld.cg (from L2, never a stale L1 line).
//
// The reflector rows of D and A stream through shared memory in 32-row x b
// chunks, four in flight, each one TMA tensor load (a 2-D map of W, chunks
// starting at even rows for the 16-byte rule); the first chunks of a step are
// issued before its barriers, so they land while the grid synchronizes.
// Entries on and above the diagonal of a step's block (other data in the
// factor's storage) are replaced by 1 and 0 as they are read.  Sums run in a
// fixed order: results are bit-identical run to run.
#include "internal.h"
#include "tcgen05.cuh"
#include "warp_sum.cuh"

namespace lls {
namespace {

constexpr int RP_THREADS = 256;
constexpr int RP_CH = 32;      // rows of a streamed chunk (a lane each)
constexpr int RP_STAGES = 4;   // chunks in flight
constexpr int RP_NB = 128;     // largest block size: 8 warps x 16 columns
constexpr int RP_TRI = RP_NB * (RP_NB + 1) / 2;  // packed upper triangle of T_i

struct ReplayArgs {
  int64_t M, kmax, ldx;
  int nb, nsteps, forward, G;
  const double* T;  // step i's T factor at T + i nb^2 (ld nb)
  double* x;
  double* part;     // [G][nb * NR]
  double* p;        // [nb * NR]
  GridBarrier bar;
};

// Shared memory: the chunk ring, T_i's triangle, D's column-group sums.
constexpr size_t rp_smem(int nr) {
  return sizeof(double) * ((size_t)RP_STAGES * RP_CH * RP_NB + RP_TRI + 8 * RP_CH * nr);
}

__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(tc::smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ int tri(int l, int j) { return j * (j + 1) / 2 + l; }

// Starts the copy of the upper triangle of step i's T factor into shared
// memory (packed by columns); cp_async_wait + __syncthreads completes it.
__device__ __forceinline__ void stage_t(const ReplayArgs& a, int i, int b, double* Ts) {
  const double* Ti = a.T + (int64_t)i * a.nb * a.nb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = w; j < b; j += RP_THREADS / 32)
    for (int l = lane; l <= j; l += 32) cp_async8(Ts + tri(l, j), Ti + l + (int64_t)j * a.nb);
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Rows of x this CTA owns from the row update of one step through the
// partial sums of the next: [from, M) cut into G equal slices.
__device__ __forceinline__ void own_rows(int64_t from, int64_t M, int G, int64_t& lo, int64_t& hi) {
  const int64_t R = (M - from + G - 1) / G;
  lo = from + (int64_t)blockIdx.x * R;
  hi = lo + R < M ? lo + R : M;
  if (lo > M) lo = M;
}

// The chunks of one step on this CTA: nD of the row update with the block at
// column kD (rows [dbeg, hi)), then nA of the next step's partial sums with
// the block at kA (rows [abeg, hi)); chunks start at even rows.
struct Stream {
  int64_t dbase, dbeg, abase, abeg, hi, kD, kA;
  int bD, bA, nD, nA;
};
struct Chunk {
  int64_t k, r0, beg, end;
  int b;
};

__device__ __forceinline__ Stream make_stream(int64_t lo, int64_t hi, int64_t kD, int bD, bool d,
                                              int64_t kA, int bA, bool an) {
  Stream s;
  s.hi = hi;
  s.kD = kD;
  s.kA = kA;
  s.bD = bD;
  s.bA = bA;
  s.dbeg = lo > kD ? lo : kD;
  s.dbase = s.dbeg & ~(int64_t)1;
  s.abeg = lo > kA ? lo : kA;
  s.abase = s.abeg & ~(int64_t)1;
  s.nD = d && hi > s.dbeg ? (int)((hi - s.dbase + RP_CH - 1) / RP_CH) : 0;
  s.nA = an && hi > s.abeg ? (int)((hi - s.abase + RP_CH - 1) / RP_CH) : 0;
  return s;
}

__device__ __forceinline__ Chunk chunk_at(const Stream& s, int q) {
  Chunk c;
  if (q < s.nD) {
    c.k = s.kD;
    c.b = s.bD;
    c.r0 = s.dbase + (int64_t)q * RP_CH;
    c.beg = s.dbeg;
  } else {
    c.k = s.kA;
    c.b = s.bA;
    c.r0 = s.abase + (int64_t)(q - s.nD) * RP_CH;
    c.beg = s.abeg;
  }
  c.end = s.hi;
  return c;
}

// Chunk number gq of the launch (a running count over all steps) goes to
// ring slot gq mod RP_STAGES; its mbarrier phase is (gq / RP_STAGES) & 1.
struct Ring {
  double* W;           // RP_STAGES slots of RP_CH x RP_NB
  uint64_t* full;      // an mbarrier a slot
  const CUtensorMap* map;
  uint32_t bytes;      // RP_CH x nb doubles a chunk
  int* fail;           // shared: a thread's chunk wait ran out
};

__device__ __forceinline__ void issue(const Ring& rg, const Chunk& c, unsigned gq) {
  const int slot = gq % RP_STAGES;
  tc::mbar_expect_tx(&rg.full[slot], rg.bytes);
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(tc::smem_u32(rg.W + slot * RP_CH * RP_NB)),
      "l"(reinterpret_cast<uint64_t>(rg.map)), "r"(tc::smem_u32(&rg.full[slot])), "r"((int)c.r0),
      "r"((int)c.k)
      : "memory");
}

// The first RP_STAGES chunks of a stream (thread 0); returns how many.
__device__ __forceinline__ int stream_first(const Ring& rg, const Stream& s, unsigned gq) {
  const int n = s.nD + s.nA < RP_STAGES ? s.nD + s.nA : RP_STAGES;
  if (threadIdx.x == 0)
    for (int q = 0; q < n; ++q) issue(rg, chunk_at(s, q), gq + q);
  return n;
}

// Waits (bounded, whatever the error word says) for the n chunks issued
// from gq on, before a CTA that leaves early lets its shared memory go.
__device__ __forceinline__ void drain(const Ring& rg, unsigned gq, int n) {
  for (int q = 0; q < n; ++q)
    for (long long it = 0; it < tc::kWaitLimit; ++it)
      if (tc::mbar_try_wait(&rg.full[(gq + q) % RP_STAGES], ((gq + q) / RP_STAGES) & 1)) break;
}

// p2 = op(T_i) p from the staged triangle: thread 4 q + s takes the pair of
// outputs q and b - 1 - q (j + 1 and b - j terms: every pair has b + 1) over
// the terms l = s mod 4, and the four are added by two exchanges.
template <int NR>
__device__ __forceinline__ void t_product(bool forward, int b, const double* Ts, const double* ps,
                                          double* p2s) {
  const int q = threadIdx.x >> 2, sub = threadIdx.x & 3;
  const int j1 = q, j2 = b - 1 - q;
  double s1[NR], s2[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) s1[c] = s2[c] = 0.0;
  if (j1 <= j2) {
    if (forward) {  // p2(j) = sum_{l <= j} T(l, j) p(l)
      for (int l = sub; l <= j1; l += 4) {
        const double tv = Ts[tri(l, j1)];
#pragma unroll
        for (int c = 0; c < NR; ++c) s1[c] = fma(tv, ps[l * NR + c], s1[c]);
      }
      for (int l = sub; l <= j2; l += 4) {
        const double tv = Ts[tri(l, j2)];
#pragma unroll
        for (int c = 0; c < NR; ++c) s2[c] = fma(tv, ps[l * NR + c], s2[c]);
      }
    } else {  // p2(j) = sum_{l >= j} T(j, l) p(l)
      for (int l = j1 + sub; l < b; l += 4) {
        const double tv = Ts[tri(j1, l)];
#pragma unroll
        for (int c = 0; c < NR; ++c) s1[c] = fma(tv, ps[l * NR + c], s1[c]);
      }
      for (int l = j2 + sub; l < b; l += 4) {
        const double tv = Ts[tri(j2, l)];
#pragma unroll
        for (int c = 0; c < NR; ++c) s2[c] = fma(tv, ps[l * NR + c], s2[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NR; ++c) {
    s1[c] += __shfl_xor_sync(0xffffffffu, s1[c], 1);
    s2[c] += __shfl_xor_sync(0xffffffffu, s2[c], 1);
    s1[c] += __shfl_xor_sync(0xffffffffu, s1[c], 2);
    s2[c] += __shfl_xor_sync(0xffffffffu, s2[c], 2);
  }
  if (sub == 0 && j1 <= j2) {
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      p2s[j1 * NR + c] = s1[c];
      if (j2 != j1) p2s[j2 * NR + c] = s2[c];
    }
  }
}

// Runs a stream whose first chunks are in flight.  D chunks: column group w
// (16 columns) and row lane give sums that the 8 groups add in order, then
// x(r) -= sum; A chunks: acc (16 columns x NR per lane) += W(r, :)^T x(r).
// Chunks that reach into the step's diagonal block read 1 on the diagonal
// and 0 above it.  False when a wait ran out.
template <int NR>
__device__ __forceinline__ bool stream_run(const ReplayArgs& a, const Ring& rg, const Stream& s,
                                           double* red, const double* p2s, double* acc,
                                           unsigned& gq) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int n = s.nD + s.nA;
  for (int q = 0; q < n; ++q, ++gq) {
    const int slot = gq % RP_STAGES;
    // a wait that runs out is acted on by the whole CTA after this chunk's
    // barrier (the threads of a CTA need not see the same outcome)
    if (!tc::mbar_wait(&rg.full[slot], (gq / RP_STAGES) & 1, a.bar.err)) *rg.fail = 1;
    const double* Wq = rg.W + slot * RP_CH * RP_NB;
    const Chunk c = chunk_at(s, q);
    const int64_t r = c.r0 + lane, rk = r - c.k;
    const bool diag = c.r0 < c.k + c.b;  // the chunk meets the unit lower triangle
    if (q < s.nD) {
      double sum[NR];
#pragma unroll
      for (int cc = 0; cc < NR; ++cc) sum[cc] = 0.0;
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int j = w * 16 + u;
        if (j < c.b) {
          double wv = Wq[lane + j * RP_CH];
          if (diag) wv = rk > j ? wv : (rk == j ? 1.0 : 0.0);
#pragma unroll
          for (int cc = 0; cc < NR; ++cc) sum[cc] = fma(wv, p2s[j * NR + cc], sum[cc]);
        }
      }
#pragma unroll
      for (int cc = 0; cc < NR; ++cc) red[(w * RP_CH + lane) * NR + cc] = sum[cc];
      __syncthreads();
      if (t < RP_CH * NR) {
        const int rr = t % RP_CH, cc = t / RP_CH;
        const int64_t rw = c.r0 + rr;
        if (rw >= c.beg && rw < c.end) {
          double tot = 0.0;
#pragma unroll
          for (int g = 0; g < 8; ++g) tot += red[(g * RP_CH + rr) * NR + cc];
          a.x[rw + cc * a.ldx] = __ldcg(a.x + rw + cc * a.ldx) - tot;
        }
      }
    } else {
      const bool in = r >= c.beg && r < c.end;
      double xv[NR];
#pragma unroll
      for (int cc = 0; cc < NR; ++cc) xv[cc] = in ? __ldcg(a.x + r + cc * a.ldx) : 0.0;
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int j = w * 16 + u;
        if (j < c.b) {
          double wv = in ? Wq[lane + j * RP_CH] : 0.0;
          if (diag) wv = rk > j ? wv : (rk == j && in ? 1.0 : 0.0);
#pragma unroll
          for (int cc = 0; cc < NR; ++cc) acc[u * NR + cc] = fma(wv, xv[cc], acc[u * NR + cc]);
        }
      }
    }
    __syncthreads();  // the slot and the group sums are free again
    if (*rg.fail) {  // the same in every thread now: let the issued chunks land, then leave
      const int left = n - q < RP_STAGES ? n - q : RP_STAGES;
      drain(rg, gq, left);
      return false;
    }
    if (t == 0 && q + RP_STAGES < n) issue(rg, chunk_at(s, q + RP_STAGES), gq + RP_STAGES);
  }
  return true;
}

// This CTA's partial of W^T x for the b columns: the lanes of each warp added
// by halving exchanges.
template <int NR>
__device__ __forceinline__ void write_partials(const ReplayArgs& a, int b, double* acc) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int V = 16 * NR;
  int base = 0;
  WarpSumHalves<V, 16>::run(acc, lane, base);
  constexpr int H = halvings(V) < 5 ? halvings(V) : 5;
  constexpr int R = V >> H;
  constexpr int PLAIN = (1 << (5 - H)) - 1;
  if ((lane & PLAIN) == 0) {
    double* out = a.part + (int64_t)blockIdx.x * a.nb * NR;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int idx = base + q, j = w * 16 + idx / NR, c = idx % NR;
      if (j < b) out[j * NR + c] = acc[q];
    }
  }
}

template <int NR>
__global__ void __launch_bounds__(RP_THREADS, 1)
    replay_kernel(ReplayArgs a, const __grid_constant__ CUtensorMap wmap) {
  extern __shared__ __align__(1024) double sm[];
  __shared__ double p2s[RP_NB * NR];
  __shared__ double ps[RP_NB * NR];
  __shared__ __align__(8) uint64_t full[RP_STAGES];
  __shared__ int s_fail;
  const Ring rg{sm, full, &wmap, (uint32_t)(sizeof(double) * RP_CH * a.nb), &s_fail};
  double* Ts = sm + RP_STAGES * RP_CH * RP_NB;
  double* red = Ts + RP_TRI;
  unsigned int epoch = 0;
  unsigned gq = 0;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  auto step_of = [&](int si) { return a.forward ? si : a.nsteps - 1 - si; };
  auto width = [&](int64_t k) { return (int)(a.kmax - k < a.nb ? a.kmax - k : a.nb); };
  double acc[16 * NR];
  if (t == 0) {
    for (int q = 0; q < RP_STAGES; ++q) tc::mbar_init(&full[q], 1);
    tc::mbar_init_fence();
    s_fail = 0;
  }
  __syncthreads();

  int64_t k = (int64_t)step_of(0) * a.nb;
  stage_t(a, step_of(0), width(k), Ts);
  {  // A of the first step
    int64_t lo, hi;
    own_rows(k, a.M, a.G, lo, hi);
    const Stream s = make_stream(lo, hi, k, width(k), false, k, width(k), true);
#pragma unroll
    for (int e = 0; e < 16 * NR; ++e) acc[e] = 0.0;
    stream_first(rg, s, gq);
    if (!stream_run<NR>(a, rg, s, red, p2s, acc, gq)) {
      cp_async_wait();
      return;
    }
    write_partials<NR>(a, width(k), acc);
  }
  for (int si = 0; si < a.nsteps; ++si) {
    const int i = step_of(si);
    const int b = width(k);
    const bool more = si + 1 < a.nsteps;
    const int64_t k2 = more ? (int64_t)step_of(si + 1) * a.nb : k;
    if (si > 0) stage_t(a, i, b, Ts);  // lands while the barriers wait
    int64_t lo, hi;
    own_rows(k < k2 ? k : k2, a.M, a.G, lo, hi);
    const Stream s = make_stream(lo, hi, k, b, true, k2, width(k2), more);
    const int issued = stream_first(rg, s, gq);  // so do the first chunks of D
    if (!grid_sync(a.bar, epoch)) {  // every partial of step i is in
      if (t == 0) drain(rg, gq, issued);
      cp_async_wait();
      return;
    }
    // ---- B: p(o) = the partials of entry o added in a fixed order, a warp an entry
    for (int o = blockIdx.x * (RP_THREADS / 32) + w; o < b * NR; o += a.G * (RP_THREADS / 32)) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int g = lane + 32 * u;
        v[u] = g < a.G ? __ldcg(a.part + (int64_t)g * a.nb * NR + o) : 0.0;
      }
      double sv = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, off);
      if (lane == 0) a.p[o] = sv;
    }
    if (!grid_sync(a.bar, epoch)) {  // p is in
      if (t == 0) drain(rg, gq, issued);
      cp_async_wait();
      return;
    }
    // ---- C: p2 = op(T_i) p in shared memory, every CTA for itself
    for (int e = t; e < b * NR; e += RP_THREADS) ps[e] = __ldcg(a.p + e);
    cp_async_wait();
    __syncthreads();
    t_product<NR>(a.forward != 0, b, Ts, ps, p2s);
    __syncthreads();
    // ---- D on this CTA's rows, then A of the next step on the same rows
#pragma unroll
    for (int e = 0; e < 16 * NR; ++e) acc[e] = 0.0;
    if (!stream_run<NR>(a, rg, s, red, p2s, acc, gq)) {
      cp_async_wait();
      return;
    }
    if (more) write_partials<NR>(a, s.bA, acc);
    __syncthreads();
    k = k2;
  }
  cp_async_wait();
}

int rp_ctas() {
  static int nsm = -1;
  if (nsm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) nsm = 148;
    if (nsm > 256) nsm = 256;  // phase B reads at most eight partials a lane
  }
  return nsm;
}

}  // namespace

size_t replay_persistent_scratch_bytes(int64_t nb, int64_t nrhs) {
  return 64 + sizeof(double) * ((size_t)rp_ctas() * nb * nrhs + (size_t)nb * nrhs);
}

bool replay_persistent_fits(int64_t nb, int64_t nrhs, const double* W, int64_t ldw, int64_t M,
                            int64_t kmax) {
  return nrhs >= 1 && nrhs <= 4 && nb >= 1 && nb <= RP_NB && ldw % 2 == 0 &&
         reinterpret_cast<uintptr_t>(W) % 16 == 0 && M < INT32_MAX && kmax < INT32_MAX;
}

Status replay_persistent(bool forward, int64_t M, int64_t nb, int64_t nsteps, int64_t kmax,
                         const double* W, int64_t ldw, const double* T, double* x, int64_t ldx,
                         int64_t nrhs, Scratch scratch, int* err, cudaStream_t st) {
  if (nsteps <= 0 || nrhs <= 0 || M <= 0) return ok_status();
  if (!replay_persistent_fits(nb, nrhs, W, ldw, M, kmax))
    return make_error(LLS_ERR_ARG, "replay_persistent: nrhs <= 4, nb <= 128, even ldw, aligned W");
  if (scratch.bytes < replay_persistent_scratch_bytes(nb, nrhs))
    return make_error(LLS_ERR_NOMEM, "replay_persistent: scratch too small");
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return make_error(LLS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  CUtensorMap wmap;
  {  // W as rows x kmax FP64, boxes of 32 rows x nb columns; rows >= M read 0
    cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)kmax};
    cuuint64_t strides[1] = {(cuuint64_t)(ldw * sizeof(double))};
    cuuint32_t box[2] = {(cuuint32_t)RP_CH, (cuuint32_t)nb};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&wmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(W), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return make_error(LLS_ERR_CUDA, "cuTensorMapEncodeTiled (reflectors) failed");
  }
  char* base = static_cast<char*>(scratch.ptr);
  ReplayArgs a;
  a.M = M;
  a.kmax = kmax;
  a.ldx = ldx;
  a.nb = (int)nb;
  a.nsteps = (int)nsteps;
  a.forward = forward ? 1 : 0;
  a.G = rp_ctas();
  a.T = T;
  a.x = x;
  a.part = reinterpret_cast<double*>(base + 64);
  a.p = a.part + (size_t)a.G * nb * nrhs;
  a.bar.count = reinterpret_cast<unsigned int*>(base);
  a.bar.err = err;
  a.bar.limit = g_barrier_spin_limit.load(std::memory_order_relaxed);
  LLS_CUDA(cudaMemsetAsync(base, 0, 8, st));
  // W_i is read twice a step (A and D): sum_i b_i (M - k_i) = kmax (M - kmax / 2) entries
  const double wsum = (double)kmax * ((double)M - 0.5 * (double)kmax);
  TraceScope ts(kTrReplay, st, 4.0 * wsum * nrhs, 16.0 * wsum);
  void* args[] = {&a, &wmap};
  const void* fn = nrhs == 1   ? (const void*)replay_kernel<1>
                   : nrhs == 2 ? (const void*)replay_kernel<2>
                   : nrhs == 3 ? (const void*)replay_kernel<3>
                               : (const void*)replay_kernel<4>;
  LLS_TRY(allow_max_dyn_smem(fn));
  return coop_launch(fn, a.G, RP_THREADS, args, rp_smem((int)nrhs), st);
}

}  // namespace lls
