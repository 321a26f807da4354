// FP64-accurate GEMM on the BF16 tensor cores (tcgen05), by exact slicing.
//
// B300's FP64 ALU gives ~1.2 TFLOP/s, its BF16 tensor cores ~1.75 PFLOP/s.
// This computes C = alpha op(A) op(B) + beta C with FP64 operands and FP64
// result at FP64-level accuracy from BF16 products that are all exact:
//
//  1. Every row i of op(A) is scaled by 2^-e_i (2^e_i > max_k |op(A)_ik|) and
//     every column j of op(B) by 2^-f_j, so each scaled entry x lies in
//     (-1, 1).  With integer arithmetic only, x * 2^56 (rounded to an integer)
//     is written in signed base 128:  x = sum_{s=1..8} d_s 2^-7s with
//     d_1 in [-128, 128] and d_2..d_8 in [-64, 63] -- integers that BF16
//     holds exactly.  The 8 digit planes ("slices") are stored K-major.
//  2. C_ij = 2^(e_i + f_j) sum_{s,t} 2^-7(s+t) sum_k d_s(i,k) d'_t(k,j).  The
//     36 products with s + t <= 9 run on tcgen05.mma kind::f16 (BF16 in,
//     FP32 accumulate in tensor memory), one FP32 accumulator per diagonal
//     D = s + t (8 of them for a 128 x 128 tile, in two passes of 4 x 128
//     TMEM columns).  Per K entry a diagonal gains at most 2^15 in
//     magnitude, so with at most 256 K entries per work item every
//     accumulator stays below 2^24: the FP32 sums
//     are exact integers.  Terms with s + t >= 10 are below 2^-55 relative
//     to the row/column scales and are dropped.
//  3. The epilogue combines the 8 exact integers into two 64-bit integers,
//     H (diagonals 2..5, unit 2^-35 of the row/column scale 2^(e_i + f_j))
//     and L (diagonals 6..9, unit 2^-63), and folds them into one,
//     v = H 2^19 + round(L 2^-9) (unit 2^-54; |H| <= K 2^35 (1 + tiny) with
//     K <= 256, so |v| < 2^63).  The only roundings are that fold (half a
//     unit, 2^-55 of the scale) and v -> FP64 (53 bits, to nearest), both at
//     FP64 GEMM accuracy.  The FP64 value is assembled from bits, then alpha
//     and beta are applied.  Longer K is split into 256-wide
//     ranges whose FP64 partial products are summed in a fixed order.
//
// Work per FP64 multiply-add: 36 BF16 multiply-adds on the tensor cores and
// a handful of integer/FP64 operations per output element, instead of K DFMAs.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "lls_kernels.h"
#include "oz_gemm.h"

namespace lls {
namespace {

constexpr int OZ_S = 8;           // slices per operand
constexpr int OZ_BM = 128;        // output rows per tile (MMA M)
constexpr int OZ_BN = 128;        // output columns per tile (MMA N)
constexpr int OZ_BK = 64;         // K per smem tile (128-byte swizzle rows)
constexpr int OZ_KC = 256;        // K per work item: keeps every FP32 sum below 2^24
constexpr int OZ_XST = 6;         // X ring depth (one 128 x 64 slice tile per stage)
constexpr int OZ_ZST = 7;         // Z ring depth (one 128 x 64 slice tile per stage)
constexpr int OZ_EPI_WARP0 = 2;  // warps 0 (TMA) and 1 (MMA issue), then the epilogue
constexpr int OZ_EPI_WARPS = 16;  // 4 lane quadrants x 4 groups of 32 columns
constexpr int OZ_EPI_COLS = OZ_BN / (OZ_EPI_WARPS / 4);  // columns per epilogue thread
constexpr int OZ_THREADS = (OZ_EPI_WARP0 + OZ_EPI_WARPS) * 32;
constexpr uint32_t OZ_TILE = OZ_BM * OZ_BK * 2;           // 16 KB, either operand
constexpr int OZ_ACC = 4;         // diagonal accumulators per pass: 4 x 128 TMEM columns
static_assert(OZ_BM == OZ_BN, "one tile shape and tensor-map box for both operands");
constexpr int kZeroExp = -4000;   // exponent of an all-zero row / column
constexpr long long kOzWaitLimit = 1LL << 24;

// ----------------------------------------------------------------------------
// Slicing.  The logical operand Op is R x K ("rows" r = output rows of A or
// output columns of B); its stored matrix is either K-contiguous
// (Op(r,k) = src[k + r ld]) or R-contiguous (Op(r,k) = src[r + k ld]).
// Unit-lower mode reads the stored matrix as unit lower trapezoidal.
// Slices: out[s][r][k], leading dimension ldk (a multiple of 8).
// ----------------------------------------------------------------------------
__device__ __forceinline__ double op_load(const double* src, int64_t ld, bool kcontig, bool ul,
                                          int64_t r, int64_t k) {
  int64_t p = kcontig ? k : r, c = kcontig ? r : k;  // stored (row, col)
  if (ul) {
    if (p < c) return 0.0;
    if (p == c) return 1.0;
  }
  return src[p + c * ld];
}

__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ int exp_of_max(unsigned long long bits) {
  // 2^e > max with e = unbiased exponent + 1 (frexp convention); zero -> sentinel
  if (bits == 0) return kZeroExp;
  int ex = (int)(bits >> 52);
  if (ex == 0) return -1022;  // subnormal maximum
  return ex - 1023 + 1;
}

// x * 2^(56 - e) rounded to an int64 X (|X| < 2^56), then 8 signed base-128
// digits, most significant first.  With the bias B = 64 (1 + 128 + ... + 128^7),
// X + B written in base 128 has the digits d_s + 64: every digit below the top
// one is a plain 7-bit field of X + B (no carries to propagate), and the top
// one is its arithmetic shift by 49.  d_1 lies in [-128, 128], d_2..d_8 in
// [-64, 63], and X = sum_s d_s 128^(8 - s) exactly.
constexpr long long kDigitBias = 0x81020408102040LL;  // 64 (128^8 - 1) / 127

__device__ __forceinline__ void make_digits(double v, int e, int d[OZ_S]) {
  unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  int ex = (int)((bits >> 52) & 0x7FF);
  long long X = 0;
  if (ex != 0 && e != kZeroExp) {
    unsigned long long mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    int sh = ex - 1075 + 56 - e;
    if (sh >= 0) X = (long long)(mant << sh);
    else if (sh > -60) X = (long long)((mant + (1ull << (-sh - 1))) >> (-sh));
    if (bits >> 63) X = -X;
  }
  const long long Y = X + kDigitBias;
  d[0] = (int)(Y >> 49) - 64;
  const unsigned int lo = (unsigned int)Y, hi = (unsigned int)((unsigned long long)Y >> 32);
#pragma unroll
  for (int s = 1; s < OZ_S; ++s) {
    const int shift = 49 - 7 * s;  // 42, 35, ..., 0
    unsigned int f;
    if (shift >= 32) f = hi >> (shift - 32);
    else if (shift + 7 <= 32) f = lo >> shift;
    else f = __funnelshift_r(lo, hi, shift);
    d[s] = (int)(f & 127u) - 64;
  }
}

// K-contiguous operand: one warp per row r; max over k, then the digits.
__global__ void oz_slice_kcontig_kernel(int64_t R, int64_t K, const double* __restrict__ src,
                                        int64_t ld, int ul, __nv_bfloat16* __restrict__ out,
                                        int64_t ldk, int* __restrict__ exps) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t plane = R * ldk;
  for (int64_t r = warp; r < R; r += nwarps) {
    unsigned long long mx = 0;
    for (int64_t k = lane; k < K; k += 32) {
      unsigned long long b = abs_bits(op_load(src, ld, true, ul != 0, r, k));
      mx = b > mx ? b : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = t > mx ? t : mx;
    }
    const int e = exp_of_max(mx);
    if (lane == 0) exps[r] = e;
    for (int64_t k = lane; k < ldk; k += 32) {
      int d[OZ_S] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (k < K) make_digits(op_load(src, ld, true, ul != 0, r, k), e, d);
#pragma unroll
      for (int s = 0; s < OZ_S; ++s) out[s * plane + r * ldk + k] = __int2bfloat16_rn(d[s]);
    }
  }
}

// K-contiguous operand by chunks: grid (K chunks of OZ_KCH, rows), so a
// handful of long rows (the b x K reflector blocks) still fills the GPU.
// Pass 1: per-row maximum of |Op(r, k)|, one atomicMax per chunk.
constexpr int OZ_KCH = 1024;

__global__ void __launch_bounds__(256) oz_rowmax_kcontig_kernel(int64_t R, int64_t K,
                                                                 const double* __restrict__ src,
                                                                 int64_t ld, int ul,
                                                                 unsigned long long* __restrict__ mx) {
  __shared__ unsigned long long red[8];
  const int64_t r = blockIdx.y;
  const int64_t k0 = (int64_t)blockIdx.x * OZ_KCH;
  unsigned long long m = 0;
  static_assert(OZ_KCH == 4 * 256, "four loads per thread and chunk");
  double v[4];  // in flight together
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t k = k0 + threadIdx.x + 256 * q;
    v[q] = k < K ? op_load(src, ld, true, ul != 0, r, k) : 0.0;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const unsigned long long b = abs_bits(v[q]);
    m = b > m ? b : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) m = red[w] > m ? red[w] : m;
    if (m) atomicMax(mx + r, m);
  }
}

// Pass 2 (after oz_exps_kernel): the digits of one chunk of one row; each
// plane's stores are contiguous in k.
__global__ void __launch_bounds__(256) oz_slice_kcontig_chunk_kernel(
    int64_t R, int64_t K, const double* __restrict__ src, int64_t ld, int ul,
    const int* __restrict__ exps, __nv_bfloat16* __restrict__ out, int64_t ldk) {
  const int64_t r = blockIdx.y;
  const int64_t k0 = (int64_t)blockIdx.x * OZ_KCH;
  const int e = exps[r];
  const int64_t plane = R * ldk;
  // two consecutive k per thread: one 4-byte store per plane (ldk and k0 are even);
  // the chunk's four loads of this thread are issued first
  double v[4];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int64_t k = k0 + 2 * threadIdx.x + 512 * q;
    v[2 * q] = k < K ? op_load(src, ld, true, ul != 0, r, k) : 0.0;
    v[2 * q + 1] = k + 1 < K ? op_load(src, ld, true, ul != 0, r, k + 1) : 0.0;
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int64_t k = k0 + 2 * threadIdx.x + 512 * q;
    if (k >= ldk) continue;
    int d0[OZ_S] = {0, 0, 0, 0, 0, 0, 0, 0}, d1[OZ_S] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (k < K) make_digits(v[2 * q], e, d0);
    if (k + 1 < K) make_digits(v[2 * q + 1], e, d1);
#pragma unroll
    for (int s = 0; s < OZ_S; ++s)
      *reinterpret_cast<__nv_bfloat162*>(out + s * plane + r * ldk + k) =
          __halves2bfloat162(__int2bfloat16_rn(d0[s]), __int2bfloat16_rn(d1[s]));
  }
}

// R-contiguous operand, pass 1: per-row maximum of |Op(r, k)| by 32 x 64 tiles.
__global__ void oz_rowmax_rcontig_kernel(int64_t R, int64_t K, const double* __restrict__ src,
                                         int64_t ld, int ul, unsigned long long* __restrict__ mx) {
  const int64_t r = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
  const int64_t k0 = (int64_t)blockIdx.y * 64;
  unsigned long long m = 0;
  if (r < R) {
    double v[8];  // 256 threads: eight k per thread, loads in flight together
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t k = k0 + (threadIdx.x >> 5) + 8 * q;
      v[q] = k < K ? op_load(src, ld, false, ul != 0, r, k) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const unsigned long long b = abs_bits(v[q]);
      m = b > m ? b : m;
    }
    if (m) atomicMax(mx + r, m);
  }
}

__global__ void oz_exps_kernel(int64_t R, const unsigned long long* __restrict__ mx,
                               int* __restrict__ exps) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < R) exps[r] = exp_of_max(mx[r]);
}

// R-contiguous operand, pass 2: digits of a 32 (r) x 32 (k) tile, transposed
// through shared memory so that the K-major slices are written coalesced.
__global__ void __launch_bounds__(256) oz_slice_rcontig_kernel(
    int64_t R, int64_t K, const double* __restrict__ src, int64_t ld, int ul,
    const int* __restrict__ exps, __nv_bfloat16* __restrict__ out, int64_t ldk) {
  __shared__ short tile[OZ_S][32][66];  // [plane][r][k], padded rows
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // 8 warps
  const int64_t r0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 64;
  {
    const int64_t r = r0 + lane;
    const int e = r < R ? exps[r] : kZeroExp;
    double v[8];  // coalesced: 32 consecutive rows per load, eight loads in flight
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t k = k0 + w + 8 * q;
      v[q] = (r < R && k < K) ? op_load(src, ld, false, ul != 0, r, k) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int kk = w + 8 * q;
      int d[OZ_S] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (r < R && k0 + kk < K) make_digits(v[q], e, d);
#pragma unroll
      for (int s = 0; s < OZ_S; ++s) tile[s][lane][kk] = (short)d[s];
    }
  }
  __syncthreads();
  const int64_t plane = R * ldk;
  for (int rr = w; rr < 32; rr += 8) {  // one 128-byte store per row and plane
    const int64_t r = r0 + rr, k = k0 + 2 * lane;
    if (r >= R || k >= ldk) continue;
#pragma unroll
    for (int s = 0; s < OZ_S; ++s)
      *reinterpret_cast<__nv_bfloat162*>(out + s * plane + r * ldk + k) = __halves2bfloat162(
          __int2bfloat16_rn(tile[s][rr][2 * lane]), __int2bfloat16_rn(tile[s][rr][2 * lane + 1]));
  }
}

// ----------------------------------------------------------------------------
// Tensor-core kernel
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  for (long long i = 0; i < kOzWaitLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 255 && *reinterpret_cast<volatile int*>(err) != 0) return false;
    if (i > 64) __nanosleep(40);
  }
  atomicExch(err, 1);
  return false;
}
// The same for the single producer and MMA-issuing threads, whose waits sit
// on the tensor pipe's critical path: no sleep between polls (try_wait
// itself suspends the thread for a while), a bounded number of polls.
__device__ bool mbar_wait_spin(uint64_t* bar, uint32_t parity, int* err) {
  for (long long i = 0; i < kOzWaitLimit / 4; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 255 && *reinterpret_cast<volatile int*>(err) != 0) return false;
  }
  atomicExch(err, 1);
  return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
constexpr uint32_t kOzIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BN >> 3) << 17) |
                              ((uint32_t)(OZ_BM >> 4) << 24);
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kOzIdesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
// v * 2^p as an FP64, assembled from bits with integer operations only (FP64
// arithmetic and conversions are scarce on this part): |v| is normalised so
// its top bit is bit 63, rounded to 53 bits (to nearest, ties away from
// zero; a carry out of the mantissa lands in the exponent), and the exponent
// set directly.  Returns false when the result would leave the normal range.
__device__ __forceinline__ bool i64_scaled(long long v, int p, double& out) {
  const unsigned long long sgn = (unsigned long long)(v >> 63);
  const unsigned long long a = ((unsigned long long)v ^ sgn) - sgn;
  if (a == 0) {
    out = 0.0;
    return true;
  }
  const int lz = __clzll((long long)a);
  const unsigned long long norm = a << lz;                       // bit 63 set
  const unsigned long long mant = (norm >> 11) + ((norm >> 10) & 1ull);  // 2^52 .. 2^53
  const int be = 63 - lz + p + 1023;                              // biased exponent
  if ((unsigned)(be - 1) >= 2045u) return false;
  out = __longlong_as_double(
      (long long)((((unsigned long long)(be - 1)) << 52) + mant + (sgn << 63)));
  return true;
}

__device__ __forceinline__ double pow2(int k) {
  if (k < -1022) return 0.0;
  if (k > 1023) k = 1023;
  return __longlong_as_double((long long)(k + 1023) << 52);
}

// Out-of-range exponents (results near under/overflow): rarely taken, kept
// out of line so the common path carries no FP64 conversion.
__device__ __noinline__ double slow_scaled(long long v, int p) {
  return (double)v * pow2(p / 2) * pow2(p - p / 2);
}

struct OzArgs {
  int M, N, K, kchunk;
  int tiles_n, splits, items;  // work items: (row tile, column tile, K range)
  const int* expX;   // per output row (M)
  const int* expZ;   // per output column (N)
  double alpha, beta;
  double* C;
  int64_t ldc;
  int transC;        // store D(i,j) at C[j + i ldc]
  double* part;      // split-K partials [split][M x N], column-major
  int* err;
};

// Persistent: one CTA per SM loops over (row tile, column tile, K range)
// items of 128 x 128 outputs.  At N = 128 an MMA reads 8 KB of operands from
// shared memory for 128 x 128 x 16 multiply-adds (N = 64 reads 6 KB for half
// of them, and shared-memory bandwidth is what bounds these MMAs), but the 8
// diagonal accumulators would need 1024 TMEM columns: each item therefore
// runs in two passes over its K range, first the diagonals D = s + t = 4..7
// (26 slice products per K tile, "pass 1" below) and then 0..3 (10
// products, "pass 0"), each into the 4 x 128 columns of tensor memory.  The
// epilogue drains the first pass into exact int64 registers (L), lets the
// second start, adds it (H), and assembles, loads and stores the FP64
// results while the next item's long first pass runs; the item's lines of C
// are prefetched into L2 before its first pass is drained.
//
// Per K tile a pass consumes its X slices s = 0, 1, ... in order and its Z
// slices from the highest t down, each Z slice last used at step s = (last
// t) - t, so both operands stream through FIFO rings of single-slice tiles:
// pass 0 loads Z3 Z2 Z1 Z0 then X0..X3; pass 1 loads Z7 Z6 Z5 Z4 X0 Z3 X1 Z2
// X2 Z1 X3 Z0 X4..X7 -- the order in which the MMA thread needs them, so the
// producer only ever waits for slots that MMAs already issued will free.
struct OzLoad {
  unsigned char z, slice;
};
__constant__ OzLoad kOzSeq0[8] = {{1, 3}, {1, 2}, {1, 1}, {1, 0}, {0, 0}, {0, 1}, {0, 2}, {0, 3}};
__constant__ OzLoad kOzSeq1[16] = {{1, 7}, {1, 6}, {1, 5}, {1, 4}, {0, 0}, {1, 3}, {0, 1}, {1, 2},
                                   {0, 2}, {1, 1}, {0, 3}, {1, 0}, {0, 4}, {0, 5}, {0, 6}, {0, 7}};

// The MMAs of one K tile of pass P.  zb: ring position of the tile's first Z
// slice (Z_t sits at zb + NZ - 1 - t); cx: next X position.
template <int P>
__device__ __forceinline__ bool oz_issue_ktile(uint32_t tmem, unsigned char* xring,
                                               unsigned char* zring, uint64_t* xfull,
                                               uint64_t* xempty, uint64_t* zfull,
                                               uint64_t* zempty, uint32_t zb, uint32_t& cx,
                                               bool first_ktile, int* err) {
  constexpr int NS = P ? 8 : 4;  // X slices and Z slices of the pass
  const uint32_t zs0 = zb % OZ_ZST;  // slot of position zb; position zb + j sits in zslot(j)
  auto zslot = [&](int j) { return zs0 + j >= OZ_ZST ? zs0 + j - OZ_ZST : zs0 + j; };
  constexpr int kNeed1[8] = {4, 5, 6, 7, 8, 8, 8, 8};
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    // Z slices first needed at step s: positions zb + have .. zb + need - 1
    const int need = P ? kNeed1[s] : 4;
    const int have = s == 0 ? 0 : (P ? kNeed1[s > 0 ? s - 1 : 0] : 4);
#pragma unroll
    for (int j = 0; j < NS; ++j)
      if (j >= have && j < need &&
          !mbar_wait_spin(&zfull[zslot(j)], ((zb + j) / OZ_ZST) & 1, err))
        return false;
    const uint32_t xs = cx % OZ_XST;
    if (!mbar_wait_spin(&xfull[xs], (cx / OZ_XST) & 1, err)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint64_t xdesc = sdesc_sw128(smem_u32(xring + xs * OZ_TILE));
    constexpr int kTlo1[8] = {4, 3, 2, 1, 0, 0, 0, 0};
    const int tlo = P ? kTlo1[s] : 0, thi = (P ? 7 : 3) - s;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (t < tlo || t > thi) continue;
      const uint64_t zdesc = sdesc_sw128(smem_u32(zring + zslot(NS - 1 - t) * OZ_TILE));
      const uint32_t acc = (uint32_t)(s + t - OZ_ACC * P);
#pragma unroll
      for (int kk = 0; kk < OZ_BK / 16; ++kk)
        mma_bf16(tmem + acc * OZ_BN, xdesc + (uint64_t)((kk * 32) >> 4),
                 zdesc + (uint64_t)((kk * 32) >> 4), (first_ktile && s == 0 && kk == 0) ? 0u : 1u);
    }
    mma_commit(&xempty[xs]);
    ++cx;
    mma_commit(&zempty[zslot(s)]);  // position zb + s: the slice whose last step this was
  }
  return true;
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_mma_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapZ,
                  OzArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* xring = smem;                     // OZ_XST x 16 KB
  unsigned char* zring = smem + OZ_XST * OZ_TILE;  // OZ_ZST x 16 KB
  __shared__ __align__(8) uint64_t xfull[OZ_XST], xempty[OZ_XST], zfull[OZ_ZST], zempty[OZ_ZST];
  __shared__ __align__(8) uint64_t tfull, tempty;
  __shared__ uint32_t s_tmem;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < OZ_XST; ++i) {
      mbar_init(&xfull[i], 1);
      mbar_init(&xempty[i], 1);
    }
    for (int i = 0; i < OZ_ZST; ++i) {
      mbar_init(&zfull[i], 1);
      mbar_init(&zempty[i], 1);
    }
    mbar_init(&tfull, 1);
    mbar_init(&tempty, OZ_EPI_WARPS);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  auto item_coords = [&](int item, int& m0, int& n0, int& kbeg, int& nkb) {
    const int ks = item % a.splits, t = item / a.splits;
    m0 = (t / a.tiles_n) * OZ_BM;
    n0 = (t % a.tiles_n) * OZ_BN;
    kbeg = ks * a.kchunk;
    nkb = (min(a.K, kbeg + a.kchunk) - kbeg + OZ_BK - 1) / OZ_BK;
  };

  if (warp == 0 && lane == 0) {
    // ---- producer: both passes' slice tiles in the MMA thread's order
    uint32_t px = 0, pz = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < a.items && ok; item += gridDim.x) {
      int m0, n0, kbeg, nkb;
      item_coords(item, m0, n0, kbeg, nkb);
      for (int pass = 0; pass < 2 && ok; ++pass) {  // diagonals 4..7, then 0..3
        const OzLoad* seq = pass ? kOzSeq0 : kOzSeq1;
        const int nseq = pass ? 8 : 16;
        for (int kb = 0; kb < nkb && ok; ++kb) {
          const int k = kbeg + kb * OZ_BK;
          for (int e = 0; e < nseq; ++e) {
            const OzLoad ld = seq[e];
            uint32_t& pos = ld.z ? pz : px;
            const uint32_t st = ld.z ? OZ_ZST : OZ_XST;
            const uint32_t slot = pos % st;
            uint64_t* emp = ld.z ? &zempty[slot] : &xempty[slot];
            uint64_t* ful = ld.z ? &zfull[slot] : &xfull[slot];
            if (pos >= st && !mbar_wait_spin(emp, ((pos / st) - 1) & 1, a.err)) {
              ok = false;
              break;
            }
            mbar_expect_tx(ful, OZ_TILE);
            tma_load_3d((ld.z ? zring : xring) + slot * OZ_TILE, ld.z ? &mapZ : &mapX, ful, k,
                        ld.z ? n0 : m0, ld.slice);
            ++pos;
          }
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: pass 0 then pass 1 of every item, each into all of TMEM
    uint32_t cx = 0, cz = 0, hs = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < a.items && ok; item += gridDim.x) {
      int m0, n0, kbeg, nkb;
      item_coords(item, m0, n0, kbeg, nkb);
      for (int pass = 0; pass < 2 && ok; ++pass, ++hs) {
        // the epilogue has drained the previous pass
        if (hs >= 1 && !mbar_wait_spin(&tempty, (hs - 1) & 1, a.err)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int kb = 0; kb < nkb && ok; ++kb) {  // diagonals 4..7, then 0..3
          ok = pass ? oz_issue_ktile<0>(tmem, xring, zring, xfull, xempty, zfull, zempty, cz, cx,
                                        kb == 0, a.err)
                    : oz_issue_ktile<1>(tmem, xring, zring, xfull, xempty, zfull, zempty, cz, cx,
                                        kb == 0, a.err);
          cz += pass ? 4 : 8;
        }
        if (ok) mma_commit(&tfull);
      }
    }
  } else if (warp >= OZ_EPI_WARP0) {
    // ---- epilogue: warp w reads TMEM lanes 32 (w mod 4) .. +31 (its rows)
    // and the 32 columns 32 ((w - 2) / 4) .. +31, in chunks of 4 (18 warps
    // put five on two SM sub-partitions, whose register files then hold 96
    // registers a thread: the 32 exact sums take 64 of them).
    const int q = warp & 3;
    const int cg0 = ((warp - OZ_EPI_WARP0) >> 2) * OZ_EPI_COLS;
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    const int bmode = a.part ? 3 : (a.beta == 0.0 ? 0 : (a.beta == 1.0 ? 1 : 2));
    const double alpha = a.alpha, beta = a.beta;
    uint32_t hs = 0;
    bool alive = true;
    for (int item = blockIdx.x; item < a.items && alive; item += gridDim.x) {
      int m0, n0, kbeg, nkb;
      item_coords(item, m0, n0, kbeg, nkb);
      if ((bmode == 1 || bmode == 2) && !a.transC) {
        // the C lines this thread will read, into L2 while the item's MMAs run
        const int ip = m0 + q * 32 + lane;
        if (ip < a.M) {
          const double* cp = a.C + ip + (int64_t)(n0 + cg0) * a.ldc;
          const int nc = min(OZ_EPI_COLS, a.N - n0 - cg0);
          for (int c = 0; c < nc; ++c)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(cp + (int64_t)c * a.ldc));
        }
      }
      long long V[OZ_EPI_COLS];
#pragma unroll
      for (int pass = 0; pass < 2; ++pass, ++hs) {
        bool ready = nkb > 0 && mbar_wait(&tfull, hs & 1, a.err);
        ready = __all_sync(0xffffffffu, ready);
        if (!ready) {  // warp-uniform: the TMEM loads below are .sync.aligned
          alive = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int ch = 0; ch < OZ_EPI_COLS / 4; ++ch) {  // 4 columns at a time
          uint32_t r[OZ_ACC][4];
#pragma unroll
          for (int d = 0; d < OZ_ACC; ++d)
            tmem_ld4(trow + (uint32_t)(d * OZ_BN + cg0 + ch * 4), r[d]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            // |acc| <= 10.5e6 < 2^24: each pair x 128 + y fits in int32
            const int x0 = __float2int_rn(__uint_as_float(r[0][c]));
            const int x1 = __float2int_rn(__uint_as_float(r[1][c]));
            const int x2 = __float2int_rn(__uint_as_float(r[2][c]));
            const int x3 = __float2int_rn(__uint_as_float(r[3][c]));
            const long long w = (long long)(x0 * 128 + x1) * 16384 + (x2 * 128 + x3);
            if (pass == 0) V[ch * 4 + c] = (w + (1LL << 8)) >> 9;  // diagonals 4..7: L
            else V[ch * 4 + c] += w * (1LL << 19);                 // diagonals 0..3: H
          }
        }
        // this pass's accumulators are drained: the next pass may start
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty);
      }
      if (!alive) break;

      const int i = m0 + q * 32 + lane;
      if (i >= a.M) continue;
      const int ei = a.expX[i];
#pragma unroll
      for (int ch = 0; ch < OZ_EPI_COLS / 4; ++ch) {  // chunks of 4 columns
        const int jb = n0 + cg0 + ch * 4;
        const int ncols = min(4, a.N - jb);
        if (ncols <= 0) break;
        double v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          v[c] = 0.0;
          const int fj = c < ncols ? a.expZ[jb + c] : kZeroExp;
          if (ei != kZeroExp && fj != kZeroExp) {
            const int p = ei + fj - 54;
            if (!i64_scaled(V[ch * 4 + c], p, v[c])) v[c] = slow_scaled(V[ch * 4 + c], p);
          }
        }
        // one loop per output mode, so no FP64 instruction of another mode
        // is issued predicated off (FP64 issue slots are scarce on this part)
        if (bmode == 3) {
          double* P = a.part + (int64_t)(item % a.splits) * a.M * a.N + i + (int64_t)jb * a.M;
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (c < ncols) P[(int64_t)c * a.M] = v[c];
        } else if (!a.transC) {
          double* cp = a.C + i + (int64_t)jb * a.ldc;
          if (bmode == 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if (c < ncols) cp[(int64_t)c * a.ldc] = alpha * v[c];
          } else if (bmode == 1) {
            double cv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) cv[c] = c < ncols ? cp[(int64_t)c * a.ldc] : 0.0;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if (c < ncols) cp[(int64_t)c * a.ldc] = fma(alpha, v[c], cv[c]);
          } else {
            double cv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) cv[c] = c < ncols ? cp[(int64_t)c * a.ldc] : 0.0;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if (c < ncols) cp[(int64_t)c * a.ldc] = fma(alpha, v[c], beta * cv[c]);
          }
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (c >= ncols) break;
            double* cp = a.C + jb + c + (int64_t)i * a.ldc;
            *cp = bmode == 0 ? alpha * v[c] : fma(alpha, v[c], (bmode == 1 ? 1.0 : beta) * *cp);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

__global__ void oz_reduce_kernel(int M, int N, int splits, const double* __restrict__ part,
                                 double alpha, double beta, double* C, int64_t ldc, int transC) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)M * N) return;
  int64_t i = idx % M, j = idx / M;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += part[(int64_t)z * M * N + idx];
  double* cp = transC ? C + j + i * ldc : C + i + j * ldc;
  *cp = (beta == 0.0) ? alpha * s : fma(alpha, s, beta * *cp);
}

// ---------------------------------------------------------------------------

// Slices [8][R][ldk] bf16 as a 3-D tensor (K, R, 8) with box (64, rows, planes).
Status make_slice_map(CUtensorMap* map, const void* base, int64_t K, int64_t R, int64_t ldk,
                      int box_rows, int box_planes) {
  EncodeTiledFn fn = tensor_map_encoder();
  if (!fn) return make_error(LLS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)R, (cuuint64_t)OZ_S};
  cuuint64_t strides[2] = {(cuuint64_t)(ldk * 2), (cuuint64_t)(R * ldk * 2)};
  cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return make_error(LLS_ERR_CUDA, "cuTensorMapEncodeTiled (slices) failed");
  return ok_status();
}

int64_t pad8(int64_t x) { return std::max<int64_t>(8, (x + 7) / 8 * 8); }

}  // namespace

size_t oz_slice_bytes(int64_t R, int64_t K) { return (size_t)OZ_S * R * pad8(K) * 2; }

size_t oz_gemm_workspace_bytes(int64_t M, int64_t N, int64_t K) {
  size_t b = oz_slice_bytes(M, K) + oz_slice_bytes(N, K) + 8 * (size_t)(M + N) + 8 * (M + N) + 1024;
  int64_t splits = (K + OZ_KC - 1) / OZ_KC;
  if (splits > 1) b += (size_t)splits * M * N * sizeof(double);
  return b;
}

// Slices of the R x K logical operand into `out` ([8][R][pad8(K)]), exponents in exps.
Status oz_slice(int64_t R, int64_t K, const double* src, int64_t ld, bool kcontig, bool unit_lower,
                __nv_bfloat16* out, int* exps, unsigned long long* maxbuf, cudaStream_t st) {
  const int64_t ldk = pad8(K);
  TraceScope ts(kTrConvert, st, 0.0, (8.0 + 16.0) * R * K);
  if (kcontig) {
    if (R > 65535) {
      int64_t warps = std::min<int64_t>(R, 148 * 64);
      oz_slice_kcontig_kernel<<<(unsigned)ceil_div(warps * 32, 256), 256, 0, st>>>(
          R, K, src, ld, unit_lower ? 1 : 0, out, ldk, exps);
      LLS_LAUNCHED("oz_slice_kcontig_kernel");
      return ok_status();
    }
    LLS_CUDA(cudaMemsetAsync(maxbuf, 0, sizeof(unsigned long long) * R, st));
    oz_rowmax_kcontig_kernel<<<dim3((unsigned)ceil_div(K, OZ_KCH), (unsigned)R), 256, 0, st>>>(
        R, K, src, ld, unit_lower ? 1 : 0, maxbuf);
    LLS_LAUNCHED("oz_rowmax_kcontig_kernel");
    oz_exps_kernel<<<(unsigned)ceil_div(R, 256), 256, 0, st>>>(R, maxbuf, exps);
    LLS_LAUNCHED("oz_exps_kernel");
    oz_slice_kcontig_chunk_kernel<<<dim3((unsigned)ceil_div(ldk, OZ_KCH), (unsigned)R), 256, 0, st>>>(
        R, K, src, ld, unit_lower ? 1 : 0, exps, out, ldk);
    LLS_LAUNCHED("oz_slice_kcontig_chunk_kernel");
    return ok_status();
  }
  LLS_CUDA(cudaMemsetAsync(maxbuf, 0, sizeof(unsigned long long) * R, st));
  dim3 g1((unsigned)ceil_div(R, 32), (unsigned)ceil_div(K, 64));
  oz_rowmax_rcontig_kernel<<<g1, 256, 0, st>>>(R, K, src, ld, unit_lower ? 1 : 0, maxbuf);
  LLS_LAUNCHED("oz_rowmax_rcontig_kernel");
  oz_exps_kernel<<<(unsigned)ceil_div(R, 256), 256, 0, st>>>(R, maxbuf, exps);
  LLS_LAUNCHED("oz_exps_kernel");
  dim3 g2((unsigned)ceil_div(R, 32), (unsigned)ceil_div(ldk, 64));
  oz_slice_rcontig_kernel<<<g2, 256, 0, st>>>(R, K, src, ld, unit_lower ? 1 : 0, exps, out, ldk);
  LLS_LAUNCHED("oz_slice_rcontig_kernel");
  return ok_status();
}

Status oz_gemm(bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t m, int64_t n, int64_t k,
               double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
               double beta, double* C, int64_t ldc, bool transC, Scratch ws, int* err,
               cudaStream_t st) {
  if (m <= 0 || n <= 0) return ok_status();
  if (k <= 0 || alpha == 0.0) {
    // nothing to add: reuse the FP64 kernel's scaling path
    return gemm(false, false, kDense, kDense, transC ? n : m, transC ? m : n, 0, 0.0, nullptr, 1,
                nullptr, 1, beta, C, ldc, Scratch{}, st);
  }
  if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX)
    return make_error(LLS_ERR_ARG, "oz_gemm: dimension too large");
  if (ws.bytes < oz_gemm_workspace_bytes(m, n, k))
    return make_error(LLS_ERR_NOMEM, "oz_gemm: workspace too small");
  char* p = static_cast<char*>(ws.ptr);
  auto take = [&](size_t bytes) {
    char* q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  auto* Xs = reinterpret_cast<__nv_bfloat16*>(take(oz_slice_bytes(m, k)));
  auto* Zs = reinterpret_cast<__nv_bfloat16*>(take(oz_slice_bytes(n, k)));
  int* ex = reinterpret_cast<int*>(take(sizeof(int) * m));
  int* fz = reinterpret_cast<int*>(take(sizeof(int) * n));
  auto* mxb = reinterpret_cast<unsigned long long*>(take(8 * (size_t)std::max(m, n)));
  const int64_t splits = (k + OZ_KC - 1) / OZ_KC;
  double* part = splits > 1 ? reinterpret_cast<double*>(take((size_t)splits * m * n * 8)) : nullptr;

  // op(A) (m x k): row i, entry kk is A[i + kk lda] (ta = 0) or A[kk + i lda] (ta = 1)
  LLS_TRY(oz_slice(m, k, A, lda, /*kcontig=*/ta, ma == kUnitLower, Xs, ex, mxb, st));
  // op(B) (k x n) as the n x k operand: column j, entry kk is B[kk + j ldb] (tb = 0).
  // A Gram product op(A) = op(B)^T reads the same stored operand the same
  // way: its slices are reused.
  const bool gram = A == B && lda == ldb && ta != tb && ma == mb && m == n;
  if (gram) {
    Zs = Xs;
    fz = ex;
  } else {
    LLS_TRY(oz_slice(n, k, B, ldb, /*kcontig=*/!tb, mb == kUnitLower, Zs, fz, mxb, st));
  }

  CUtensorMap mx, mz;
  LLS_TRY(make_slice_map(&mx, Xs, k, m, pad8(k), OZ_BM, 1));
  LLS_TRY(make_slice_map(&mz, Zs, k, n, pad8(k), OZ_BN, 1));
  OzArgs a;
  a.M = (int)m;
  a.N = (int)n;
  a.K = (int)k;
  a.kchunk = OZ_KC;
  a.tiles_n = (int)ceil_div(n, OZ_BN);
  a.splits = (int)splits;
  const int64_t items = ceil_div(m, OZ_BM) * a.tiles_n * splits;
  if (items > INT32_MAX) return make_error(LLS_ERR_ARG, "oz_gemm: too many tiles");
  a.items = (int)items;
  a.expX = ex;
  a.expZ = fz;
  a.alpha = alpha;
  a.beta = beta;
  a.C = C;
  a.ldc = ldc;
  a.transC = transC ? 1 : 0;
  a.part = part;
  a.err = err;
  const size_t smem = 1024 + (size_t)(OZ_XST + OZ_ZST) * OZ_TILE;
  LLS_TRY(allow_max_dyn_smem((const void*)oz_mma_kernel));
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      nsm = 148;
  }
  const unsigned grid = (unsigned)std::min<int64_t>(items, nsm);
  {
    TraceScope ts(kTrOzGemm, st, 2.0 * m * n * k, 16.0 * (double)(m + n) * k + 16.0 * m * n);
    oz_mma_kernel<<<grid, OZ_THREADS, smem, st>>>(mx, mz, a);
    LLS_LAUNCHED("oz_mma_kernel");
  }
  if (part) {
    TraceScope ts(kTrSmall, st);
    oz_reduce_kernel<<<(unsigned)ceil_div(m * n, 256), 256, 0, st>>>(
        (int)m, (int)n, (int)splits, part, alpha, beta, C, ldc, transC ? 1 : 0);
    LLS_LAUNCHED("oz_reduce_kernel");
  }
  return ok_status();
}

}  // namespace lls

extern "C" int lls_k_gemm_oz(int transa, int transb, int unit_lower_a, int unit_lower_b, int64_t m,
                             int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                             const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                             int* status, void* stream) {
  if (m < 0 || n < 0 || k < 0) return LLS_ERR_ARG;
  int64_t arows = transa ? k : m, brows = transb ? n : k;
  if (lda < (arows > 1 ? arows : 1) || ldb < (brows > 1 ? brows : 1) || ldc < (m > 1 ? m : 1))
    return LLS_ERR_ARG;
  if (m * n > 0 && (!C || !status || (k > 0 && (!A || !B)))) return LLS_ERR_ARG;
  if (m * n == 0) return LLS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  lls::Scratch s;
  s.bytes = lls::oz_gemm_workspace_bytes(m, n, k);
  if (cudaMallocAsync(&s.ptr, s.bytes, st) != cudaSuccess) return LLS_ERR_NOMEM;
  cudaMemsetAsync(status, 0, sizeof(int), st);
  lls::Status r = lls::oz_gemm(transa != 0, transb != 0,
                               unit_lower_a ? lls::kUnitLower : lls::kDense,
                               unit_lower_b ? lls::kUnitLower : lls::kDense, m, n, k, alpha, A, lda,
                               B, ldb, beta, C, ldc, false, s, status, st);
  cudaFreeAsync(s.ptr, st);
  return r.code;
}
