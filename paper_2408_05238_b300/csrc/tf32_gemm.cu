// FP64 GEMM on the TF32 tensor cores (tcgen05 .kind::tf32) with split
// operands: the trailing WY updates and Nullify's products of the TF32
// mixed-precision modes (steps a4, a6, a9 of Fig. 2-3).
//
// C = alpha op(A) op(B) + beta C with FP64 operands and FP64 result.  Each
// entry x of op(A) and op(B) is split, from its FP64 bits with integer
// operations only, into TF32 terms: hi = x rounded to 11 significant bits
// and lo = (x - hi) rounded to 11 bits, so |x - hi - lo| <= 2^-22 |x|.
//  * terms = 3 (3xTF32): hi*hi + hi*lo + lo*hi; the dropped lo*lo and the
//    splitting leave about 2^-21 relative to sum_k |a_k b_k|.
//  * terms = 1 (plain TF32): hi*hi only, about 2^-11 relative.
// TF32 x TF32 products (11 x 11 bits) are exact in FP32; the FP32
// accumulation in tensor memory rounds.  K is cut into ranges of TF_KC
// entries, each accumulated in FP32 and then added in FP64 in a fixed order
// (split-K partials), so one FP32 accumulation never spans more than TF_KC
// terms.  Entries must lie inside FP32's range (|x| < 2^128; entries below
// 2^-126 are flushed to zero): a larger entry becomes Inf and the result
// non-finite.
//
// The tensor-core kernel is persistent: one CTA per SM loops over (row tile,
// column tile, K range) items.  Warp 0 (one lane) streams the TF32 planes of
// 128 rows of op(A) and 128 columns of op(B) through a ring of shared-memory
// stages with TMA (SWIZZLE_128B: 32 FP32 = 128 bytes of K per row); warp 1
// (one lane) issues tcgen05.mma (K = 8 per instruction) into one of two
// 128-column FP32 accumulators in tensor memory; warps 4..11 drain the other
// accumulator (FP32 -> FP64 from bits, alpha, beta, store) while the next
// item's MMAs run.  Every wait is bounded (tcgen05.cuh).
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "lls_kernels.h"
#include "tcgen05.cuh"
#include "tf32_gemm.h"

namespace lls {
namespace {

constexpr int TF_BM = 128;                 // rows of op(A) per item (MMA M)
constexpr int TF_BN = 128;                 // columns of op(B) per item (MMA N)
constexpr int TF_BK = 32;                  // K per stage: 32 FP32 = one 128-byte swizzle row
constexpr int TF_KC = 1024;                // K per FP32 accumulation (one split)
constexpr int TF_THREADS = 384;            // warps 0 (TMA), 1 (MMA), 2 (TMEM), 4..11 (epilogue)
constexpr int TF_EPI_WARP0 = 4;
constexpr int TF_EPI_WARPS = 8;
constexpr uint32_t TF_PLANE = TF_BM * TF_BK * 4;   // 16 KB: one plane of one operand tile
constexpr int TF_ACC_COLS = TF_BN;                 // TMEM columns per accumulator
constexpr int kTfSplitChunk = 1024;                // K per CTA of the K-contiguous split
static_assert(TF_BM == TF_BN, "one tensor-map box height serves both operands");

constexpr int stages_for(int P) { return P == 2 ? 3 : 6; }
constexpr size_t smem_for(int P) { return 1024 + (size_t)stages_for(P) * 2 * P * TF_PLANE; }

// ---------------------------------------------------------------------------
// Splitting FP64 -> TF32 terms (FP32 bit patterns whose low 13 mantissa bits
// are zero), integer arithmetic only.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double op_load(const double* src, int64_t ld, bool kcontig, bool ul,
                                          int64_t r, int64_t k) {
  const int64_t p = kcontig ? k : r, c = kcontig ? r : k;  // stored (row, column)
  if (ul) {
    if (p < c) return 0.0;
    if (p == c) return 1.0;
  }
  return src[p + c * ld];
}

// The split is integer work on the FP64 bits, and the split passes are bound
// by it rather than by memory, so it works on 32-bit words: hi keeps the top
// 10 explicit mantissa bits (bits 19..10 of the high word), rounded to
// nearest even on the 42 bits below; lo = x - hi is those 42 bits (or 2^42
// minus them when hi rounded up, with the sign flipped) times 2^(E - 1075),
// rounded to 11 significant bits the same way.  Identical bit patterns to a
// 64-bit formulation of the same roundings (checked on tens of millions of
// values, ties and carries included).
template <int P>
__device__ __forceinline__ void tf32_split(double x, uint32_t t[P]) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t w1 = (uint32_t)(u >> 32), w0 = (uint32_t)u;
  const uint32_t sgn = w1 & 0x80000000u;
  const int E = (int)((w1 >> 20) & 0x7FFu);
#pragma unroll
  for (int p = 0; p < P; ++p) t[p] = sgn;
  if (E == 0) return;  // zero or FP64 subnormal: below FP32's range
  if (E == 0x7FF) {    // Inf stays Inf, NaN stays NaN
    t[0] = sgn | 0x7F800000u | ((((w1 & 0xFFFFFu) | w0) != 0u) ? 0x400000u : 0u);
    return;
  }
  uint32_t mh = (w1 >> 10) & 0x3FFu;
  const uint32_t r1 = w1 & 0x3FFu;  // top 10 of the 42 dropped bits
  const bool up = r1 > 0x200u || (r1 == 0x200u && (w0 != 0u || (mh & 1u) != 0u));
  int eh = E - 1023 + 127;
  if (up && ++mh == 1024u) {
    mh = 0;
    ++eh;
  }
  if (eh >= 255) {
    t[0] = sgn | 0x7F800000u;
    return;
  }
  if (eh <= 0) return;  // below FP32's normal range: flushed
  t[0] = sgn | ((uint32_t)eh << 23) | (mh << 13);
  if (P == 1) return;
  uint32_t rh = r1, rl = w0, lsgn = sgn;
  if (up) {  // hi > |x|: the remainder is 2^42 - (r1:w0), of the opposite sign
    rl = 0u - w0;
    rh = 0x400u - r1 - (w0 != 0u ? 1u : 0u);
    lsgn ^= 0x80000000u;
  }
  if ((rh | rl) == 0u) return;
  const int pos = rh != 0u ? 63 - __clz(rh) : 31 - __clz(rl);  // leading bit of rh:rl
  const int sh = pos - 10;                                      // keep 11 bits
  const unsigned long long v = ((unsigned long long)rh << 32) | rl;
  uint32_t d;
  if (sh > 0) {
    d = (uint32_t)(v >> sh);
    const unsigned long long rr = v & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rr > half || (rr == half && (d & 1u) != 0u)) ++d;
  } else {
    d = (uint32_t)(v << (-sh));
  }
  int el = E - 1075 + sh + 10 + 127;
  if (d == 2048u) {
    d = 1024u;
    ++el;
  }
  if (el <= 0) return;
  t[P - 1] = lsgn | ((uint32_t)el << 23) | ((d - 1024u) << 13);
}

// K-contiguous operand (Op(r, k) = src[k + r ld]): block (chunk, row), two
// consecutive k per thread, one 8-byte store per plane.
template <int P>
__global__ void __launch_bounds__(256) tf_split_kcontig_kernel(int64_t R, int64_t K,
                                                                const double* __restrict__ src,
                                                                int64_t ld, int ul,
                                                                uint32_t* __restrict__ out,
                                                                int64_t ldk) {
  const int64_t k0 = (int64_t)blockIdx.x * kTfSplitChunk;
  const int64_t plane = R * ldk;
  static_assert(kTfSplitChunk == 2 * 512, "two passes of 512 entries per chunk");
  for (int64_t r = blockIdx.y; r < R; r += gridDim.y) {
    double v[4];  // the chunk's four loads of this thread in flight together
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
      uint32_t t0[P], t1[P];
      tf32_split<P>(v[2 * q], t0);
      tf32_split<P>(v[2 * q + 1], t1);
#pragma unroll
      for (int p = 0; p < P; ++p)
        *reinterpret_cast<uint2*>(out + p * plane + r * ldk + k) = make_uint2(t0[p], t1[p]);
    }
  }
}

// R-contiguous operand (Op(r, k) = src[r + k ld]): a 64 (r) x 64 (k) tile read
// along r (512 contiguous bytes a column, 16 loads in flight a thread),
// transposed through shared memory and written along k.
template <int P>
__global__ void __launch_bounds__(256) tf_split_rcontig_kernel(int64_t R, int64_t K,
                                                                const double* __restrict__ src,
                                                                int64_t ld, int ul,
                                                                uint32_t* __restrict__ out,
                                                                int64_t ldk) {
  __shared__ uint32_t tile[P][64][65];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // 8 warps
  const int64_t r0 = (int64_t)blockIdx.x * 64, k0 = (int64_t)blockIdx.y * 64;
  {
    double v[16];  // all sixteen loads in flight before any split
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t k = k0 + w + 8 * q;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t r = r0 + lane + 32 * h;
        v[2 * q + h] = (r < R && k < K) ? op_load(src, ld, false, ul != 0, r, k) : 0.0;
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t t[P];
        tf32_split<P>(v[2 * q + h], t);
#pragma unroll
        for (int p = 0; p < P; ++p) tile[p][lane + 32 * h][w + 8 * q] = t[p];
      }
  }
  __syncthreads();
  const int64_t plane = R * ldk;
  for (int rr = w; rr < 64; rr += 8) {
    const int64_t r = r0 + rr, k = k0 + 2 * lane;
    if (r >= R || k >= ldk) continue;
#pragma unroll
    for (int p = 0; p < P; ++p)
      *reinterpret_cast<uint2*>(out + p * plane + r * ldk + k) =
          make_uint2(tile[p][rr][2 * lane], tile[p][rr][2 * lane + 1]);
  }
}

// ---------------------------------------------------------------------------
// Tensor-core kernel
// ---------------------------------------------------------------------------
struct TfArgs {
  int M, N, K, splits, tiles_n, items;
  double alpha, beta;
  double* C;
  int64_t ldc;
  double* part;  // split-K partials [split][M x N] (column-major), or null
  int* err;
};

// An FP32 value (bits) as an FP64, from bits (FP32 subnormals flush to zero).
__device__ __forceinline__ double f32_bits_to_f64(uint32_t b) {
  const unsigned long long s = (unsigned long long)(b >> 31) << 63;
  const uint32_t e = (b >> 23) & 0xFFu;
  if (e == 0) return __longlong_as_double((long long)s);
  const unsigned long long ee = e == 0xFFu ? 0x7FFull : (unsigned long long)(e + 896u);
  return __longlong_as_double(
      (long long)(s | (ee << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

template <int P>
__global__ void __launch_bounds__(TF_THREADS, 1)
    tf32_mma_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapZ,
                    TfArgs a) {
  constexpr int S = stages_for(P);
  constexpr uint32_t STAGE_BYTES = 2 * P * TF_PLANE;
  constexpr uint32_t ID = tc::idesc(2, TF_BM, TF_BN);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[S], empty[S], tfull[2], tempty[2];
  __shared__ uint32_t s_tmem;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&tfull[i], 1);
      tc::mbar_init(&tempty[i], TF_EPI_WARPS);
    }
    tc::mbar_init_fence();
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&s_tmem)),
                 "r"(2 * TF_ACC_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;

  auto item_coords = [&](int item, int& m0, int& n0, int& kbeg, int& nkb) {
    const int ks = item % a.splits, t = item / a.splits;
    m0 = (t / a.tiles_n) * TF_BM;
    n0 = (t % a.tiles_n) * TF_BN;
    kbeg = ks * TF_KC;
    nkb = (min(a.K, kbeg + TF_KC) - kbeg + TF_BK - 1) / TF_BK;
  };

  if (warp == 0 && lane == 0) {
    // ---- producer: per stage the P planes of the X tile and of the Z tile
    uint32_t it = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < a.items && ok; item += gridDim.x) {
      int m0, n0, kbeg, nkb;
      item_coords(item, m0, n0, kbeg, nkb);
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = it % S;
        if (it >= (uint32_t)S && !tc::mbar_wait_spin(&empty[s], ((it / S) - 1) & 1, a.err)) {
          ok = false;
          break;
        }
        unsigned char* st = smem + (size_t)s * STAGE_BYTES;
        tc::mbar_expect_tx(&full[s], STAGE_BYTES);
        tc::tma_load_3d(st, &mapX, &full[s], kbeg + kb * TF_BK, m0, 0);
        tc::tma_load_3d(st + P * TF_PLANE, &mapZ, &full[s], kbeg + kb * TF_BK, n0, 0);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: item number li accumulates into TMEM buffer li % 2
    uint32_t it = 0;
    bool ok = true;
    int li = 0;
    for (int item = blockIdx.x; item < a.items && ok; item += gridDim.x, ++li) {
      int m0, n0, kbeg, nkb;
      item_coords(item, m0, n0, kbeg, nkb);
      const int ab = li & 1;
      if (li >= 2 && !tc::mbar_wait_spin(&tempty[ab], ((li >> 1) - 1) & 1, a.err)) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const uint32_t d = tmem + (uint32_t)(ab * TF_ACC_COLS);
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = it % S;
        if (!tc::mbar_wait_spin(&full[s], (it / S) & 1, a.err)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t sb = tc::smem_u32(smem + (size_t)s * STAGE_BYTES);
        const uint64_t xd = tc::sdesc_sw128(sb), zd = tc::sdesc_sw128(sb + P * TF_PLANE);
        // terms: (lo, hi), (hi, lo), (hi, hi) for P = 2; (hi, hi) for P = 1
#pragma unroll
        for (int term = 0; term < (P == 2 ? 3 : 1); ++term) {
          const int px = (P == 2 && term == 0) ? 1 : 0;
          const int pz = (P == 2 && term == 1) ? 1 : 0;
#pragma unroll
          for (int kk = 0; kk < TF_BK / 8; ++kk) {
            const uint32_t acc = (kb == 0 && term == 0 && kk == 0) ? 0u : 1u;
            tc::mma_tf32(d, xd + (uint64_t)((px * TF_PLANE + kk * 32) >> 4),
                         zd + (uint64_t)((pz * TF_PLANE + kk * 32) >> 4), ID, acc);
          }
        }
        tc::mma_commit(&empty[s]);
      }
      if (!ok) break;
      tc::mma_commit(&tfull[ab]);
    }
  } else if (warp >= TF_EPI_WARP0) {
    // ---- epilogue: warp w reads TMEM lanes 32 (w mod 4) .. +31 (its rows)
    // and the 64 columns 64 ((w - 4) / 4) .. +63 of the accumulator
    const int q = warp & 3, ch = (warp - TF_EPI_WARP0) >> 2;
    const bool use_c = a.part == nullptr && a.beta != 0.0;
    int li = 0;
    for (int item = blockIdx.x; item < a.items; item += gridDim.x, ++li) {
      int m0, n0, kbeg, nkb;
      item_coords(item, m0, n0, kbeg, nkb);
      const int ab = li & 1;
      if (use_c) {
        // the C lines this thread will read, into L2 while the item's MMAs run
        // (read from DRAM in dependent chunks, they made the epilogue the
        // bound of the rank-b updates)
        const int ip = m0 + q * 32 + lane, jp = n0 + ch * 64;
        if (ip < a.M) {
          const double* cp = a.C + ip + (int64_t)jp * a.ldc;
          const int nc = min(64, a.N - jp);
          for (int c = 0; c < nc; ++c)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(cp + (int64_t)c * a.ldc));
        }
      }
      bool ready = tc::mbar_wait(&tfull[ab], (li >> 1) & 1, a.err);
      ready = __all_sync(0xffffffffu, ready);
      if (!ready) break;  // warp-uniform: the TMEM loads below are .sync.aligned
      tc::fence_after_sync();
      uint32_t v[64];
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * TF_ACC_COLS + ch * 64);
#pragma unroll
      for (int c = 0; c < 4; ++c) tc::tmem_ld16(taddr + (uint32_t)(c * 16), v + c * 16);
      tc::tmem_wait_ld();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[ab]);  // the accumulator may be refilled
      const int i = m0 + q * 32 + lane;
      const int jb = n0 + ch * 64;
      if (i < a.M) {
        const int ncols = min(64, a.N - jb);
        if (a.part) {
          double* P_ = a.part + (int64_t)(item % a.splits) * a.M * a.N + i + (int64_t)jb * a.M;
#pragma unroll
          for (int c = 0; c < 64; ++c)
            if (c < ncols) P_[(int64_t)c * a.M] = f32_bits_to_f64(v[c]);
        } else {
          double* cp = a.C + i + (int64_t)jb * a.ldc;
          const double alpha = a.alpha, beta = a.beta;
#pragma unroll
          for (int c0 = 0; c0 < 64; c0 += 16) {
            double cv[16];
#pragma unroll
            for (int c = 0; c < 16; ++c)
              cv[c] = (use_c && c0 + c < ncols) ? cp[(int64_t)(c0 + c) * a.ldc] : 0.0;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              if (c0 + c < ncols) {
                const double x = f32_bits_to_f64(v[c0 + c]);
                cp[(int64_t)(c0 + c) * a.ldc] =
                    !use_c ? alpha * x : (beta == 1.0 ? fma(alpha, x, cv[c]) : fma(alpha, x, beta * cv[c]));
              }
            }
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 2) {
    tc::fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * TF_ACC_COLS));
  }
}

__global__ void tf_reduce_kernel(int M, int N, int splits, const double* __restrict__ part,
                                 double alpha, double beta, double* C, int64_t ldc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)M * N) return;
  const int64_t i = idx % M, j = idx / M;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += part[(int64_t)z * M * N + idx];
  double* cp = C + i + j * ldc;
  *cp = beta == 0.0 ? alpha * s : fma(alpha, s, beta * *cp);
}

// ---------------------------------------------------------------------------

// Planes [P][R][ldk] FP32 as a 3-D tensor (K, R, P) with box (32, 128, P).
Status make_plane_map(CUtensorMap* map, const void* base, int64_t K, int64_t R, int64_t ldk, int P) {
  EncodeTiledFn fn = tensor_map_encoder();
  if (!fn) return make_error(LLS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)R, (cuuint64_t)P};
  cuuint64_t strides[2] = {(cuuint64_t)(ldk * 4), (cuuint64_t)(R * ldk * 4)};
  cuuint32_t box[3] = {(cuuint32_t)TF_BK, (cuuint32_t)TF_BM, (cuuint32_t)P};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return make_error(LLS_ERR_CUDA, "cuTensorMapEncodeTiled (TF32 planes) failed");
  return ok_status();
}

int64_t pad4(int64_t x) { return std::max<int64_t>(4, (x + 3) / 4 * 4); }

int num_sms() {
  static int n = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 148;
  });
  return n;
}

size_t plane_bytes(int64_t R, int64_t K, int P) { return (size_t)P * R * pad4(K) * 4; }

template <int P>
Status split_operand(int64_t R, int64_t K, const double* src, int64_t ld, bool kcontig, bool ul,
                     uint32_t* out, cudaStream_t st) {
  const int64_t ldk = pad4(K);
  TraceScope ts(kTrConvert, st, 0.0, (8.0 + 4.0 * P) * R * K);
  if (kcontig) {
    dim3 g((unsigned)ceil_div(ldk, kTfSplitChunk), (unsigned)std::min<int64_t>(R, 65535));
    tf_split_kcontig_kernel<P><<<g, 256, 0, st>>>(R, K, src, ld, ul ? 1 : 0, out, ldk);
    LLS_LAUNCHED("tf_split_kcontig_kernel");
  } else {
    dim3 g((unsigned)ceil_div(R, 64), (unsigned)ceil_div(ldk, 64));
    if (g.y > 65535u) return make_error(LLS_ERR_ARG, "tf32_gemm: K too large");
    tf_split_rcontig_kernel<P><<<g, 256, 0, st>>>(R, K, src, ld, ul ? 1 : 0, out, ldk);
    LLS_LAUNCHED("tf_split_rcontig_kernel");
  }
  return ok_status();
}

template <int P>
Status tf32_gemm_p(bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t m, int64_t n,
                   int64_t k, double alpha, const double* A, int64_t lda, const double* B,
                   int64_t ldb, double beta, double* C, int64_t ldc, Scratch ws, int* err,
                   cudaStream_t st) {
  char* p = static_cast<char*>(ws.ptr);
  auto take = [&](size_t bytes) {
    char* q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  auto* Xs = reinterpret_cast<uint32_t*>(take(plane_bytes(m, k, P)));
  auto* Zs = reinterpret_cast<uint32_t*>(take(plane_bytes(n, k, P)));
  const int64_t splits = ceil_div(k, TF_KC);
  double* part = splits > 1 ? reinterpret_cast<double*>(take((size_t)splits * m * n * 8)) : nullptr;

  // op(A) (m x k): row i, entry kk is A[i + kk lda] (ta = 0) or A[kk + i lda] (ta = 1)
  LLS_TRY(split_operand<P>(m, k, A, lda, /*kcontig=*/ta, ma == kUnitLower, Xs, st));
  // op(B) (k x n) as the n x k operand; a Gram product reuses the planes
  const bool gram = A == B && lda == ldb && ta != tb && ma == mb && m == n;
  if (gram) Zs = Xs;
  else LLS_TRY(split_operand<P>(n, k, B, ldb, /*kcontig=*/!tb, mb == kUnitLower, Zs, st));

  CUtensorMap mx, mz;
  LLS_TRY(make_plane_map(&mx, Xs, k, m, pad4(k), P));
  LLS_TRY(make_plane_map(&mz, Zs, k, n, pad4(k), P));
  TfArgs a;
  a.M = (int)m;
  a.N = (int)n;
  a.K = (int)k;
  a.splits = (int)splits;
  a.tiles_n = (int)ceil_div(n, TF_BN);
  const int64_t items = ceil_div(m, TF_BM) * a.tiles_n * splits;
  if (items > INT32_MAX) return make_error(LLS_ERR_ARG, "tf32_gemm: too many tiles");
  a.items = (int)items;
  a.alpha = alpha;
  a.beta = beta;
  a.C = C;
  a.ldc = ldc;
  a.part = part;
  a.err = err;
  LLS_TRY(allow_max_dyn_smem((const void*)tf32_mma_kernel<P>));
  const int grid = (int)std::min<int64_t>(items, num_sms());
  {
    TraceScope ts(kTrTf32Gemm, st, 2.0 * m * n * k, 4.0 * P * (double)(m + n) * k + 16.0 * m * n);
    tf32_mma_kernel<P><<<grid, TF_THREADS, smem_for(P), st>>>(mx, mz, a);
    LLS_LAUNCHED("tf32_mma_kernel");
  }
  if (part) {
    TraceScope ts(kTrSmall, st);
    tf_reduce_kernel<<<(unsigned)ceil_div(m * n, 256), 256, 0, st>>>((int)m, (int)n, (int)splits,
                                                                     part, alpha, beta, C, ldc);
    LLS_LAUNCHED("tf_reduce_kernel");
  }
  return ok_status();
}

}  // namespace

size_t tf32_gemm_workspace_bytes(int64_t m, int64_t n, int64_t k, int terms) {
  const int P = terms == 3 ? 2 : 1;
  size_t b = plane_bytes(m, k, P) + plane_bytes(n, k, P) + 1024;
  const int64_t splits = ceil_div(k, TF_KC);
  if (splits > 1) b += (size_t)splits * m * n * sizeof(double);
  return b;
}

Status tf32_gemm(bool ta, bool tb, OperandMode ma, OperandMode mb, int64_t m, int64_t n, int64_t k,
                 double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                 double beta, double* C, int64_t ldc, int terms, Scratch ws, int* err,
                 cudaStream_t st) {
  if (m <= 0 || n <= 0) return ok_status();
  if (terms != 1 && terms != 3) return make_error(LLS_ERR_ARG, "tf32_gemm: terms must be 1 or 3");
  if (k <= 0 || alpha == 0.0)  // nothing to add: the FP64 kernel's scaling path
    return gemm(false, false, kDense, kDense, m, n, 0, 0.0, nullptr, 1, nullptr, 1, beta, C, ldc,
                Scratch{}, st);
  if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX)
    return make_error(LLS_ERR_ARG, "tf32_gemm: dimension too large");
  if (ws.bytes < tf32_gemm_workspace_bytes(m, n, k, terms))
    return make_error(LLS_ERR_NOMEM, "tf32_gemm: workspace too small");
  if (terms == 3)
    return tf32_gemm_p<2>(ta, tb, ma, mb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, err, st);
  return tf32_gemm_p<1>(ta, tb, ma, mb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, err, st);
}

}  // namespace lls

extern "C" int lls_k_gemm_tf32(int transa, int transb, int unit_lower_a, int unit_lower_b,
                               int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                               int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                               int64_t ldc, int terms, int* status, void* stream) {
  if (m < 0 || n < 0 || k < 0 || (terms != 1 && terms != 3)) return LLS_ERR_ARG;
  const int64_t arows = transa ? k : m, brows = transb ? n : k;
  if (lda < (arows > 1 ? arows : 1) || ldb < (brows > 1 ? brows : 1) || ldc < (m > 1 ? m : 1))
    return LLS_ERR_ARG;
  if (m * n > 0 && (!C || !status || (k > 0 && (!A || !B)))) return LLS_ERR_ARG;
  if (m * n == 0) return LLS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  lls::Scratch s;
  s.bytes = lls::tf32_gemm_workspace_bytes(m, n, k, terms);
  if (cudaMallocAsync(&s.ptr, s.bytes, st) != cudaSuccess) return LLS_ERR_NOMEM;
  cudaMemsetAsync(status, 0, sizeof(int), st);
  lls::Status r = lls::tf32_gemm(transa != 0, transb != 0,
                                 unit_lower_a ? lls::kUnitLower : lls::kDense,
                                 unit_lower_b ? lls::kUnitLower : lls::kDense, m, n, k, alpha, A,
                                 lda, B, ldb, beta, C, ldc, terms, s, status, st);
  cudaFreeAsync(s.ptr, st);
  return r.code;
}
