// BF16 tensor-core GEMM on sm_103a (tcgen05 + TMA + TMEM): D = X^T Z.
//
// X is K x M and Z is K x N, both column-major BF16 (K contiguous), so both
// operands are "K-major" for the MMA; D is M x N FP32 (column-major), either
// written directly or as split-K partial sums.  Used for the sampling
// products Y = (A^T A)^q A^T G of Fig. 2 in mixed precision (step a2): X is a
// BF16 copy of the trailing block A_BR (or of its transpose), Z the sketch or
// the previous product.
//
// One CTA computes a 128 x N tile (N <= 128, padded to 16) over a range of
// K.  Warp 0 (one lane) streams 128 x 64 tiles of X and N x 64 tiles of Z
// into a ring of shared-memory stages with TMA (SWIZZLE_128B, 64 BF16 = 128
// bytes of K per row); warp 1 (one lane) issues tcgen05.mma kind::f16
// (BF16 inputs, FP32 accumulation in tensor memory) four K = 16 slices per
// stage and releases the stage with tcgen05.commit; then all four warps read
// their 32-lane quarter of the accumulator with tcgen05.ld and store it.
// Every mbarrier wait has an iteration limit: on running out the CTA raises
// *err, skips the rest, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "lls_kernels.h"
#include "tc_gemm.h"

namespace lls {
namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;          // 64 bf16 = 128 bytes: one swizzle row
constexpr int TC_STAGES = 6;
constexpr int TC_THREADS = 128;
constexpr long long kWaitLimit = 1LL << 24;

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

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false (and *err raised) when the limit runs out or another
// thread already gave up.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  for (long long i = 0; i < kWaitLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 255 && *reinterpret_cast<volatile int*>(err) != 0) return false;
    if (i > 64) __nanosleep(40);
  }
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, SWIZZLE_128B, 8-row atoms of
// 1024 bytes (stride byte offset), sm_100 descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // version
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B BF16,
// both K-major, M x N tile.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
  int M, N, Ntile, K;
  int kchunk;          // K per split (multiple of TC_BK)
  float* D;            // output (splits == 1) or partials [split][ldd * N]
  int64_t ldd;
  int* err;
  uint32_t tmem_cols;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_bf16_kernel(const __grid_constant__ CUtensorMap mapX,
                        const __grid_constant__ CUtensorMap mapZ, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned ring: stage s holds X (128 x 64) then Z (Ntile x 64)
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t xbytes = TC_BM * TC_BK * 2;
  const uint32_t zbytes = (uint32_t)a.Ntile * TC_BK * 2;
  const uint32_t stage_bytes = xbytes + zbytes;
  __shared__ __align__(8) uint64_t full_bar[TC_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[TC_STAGES];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t s_tmem;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TC_BM;
  const int kbeg = blockIdx.y * a.kchunk;
  const int kend = min(a.K, kbeg + a.kchunk);
  const int nk = (kend - kbeg + TC_BK - 1) / TC_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % TC_STAGES;
      const uint32_t round = (uint32_t)(kt / TC_STAGES);
      if (kt >= TC_STAGES && !mbar_wait(&empty_bar[s], (round - 1) & 1, a.err)) break;
      unsigned char* xs = smem + s * stage_bytes;
      unsigned char* zs = xs + xbytes;
      mbar_expect_tx(&full_bar[s], stage_bytes);
      const int kc = kbeg + kt * TC_BK;
      tma_load_2d(xs, &mapX, &full_bar[s], kc, m0);
      tma_load_2d(zs, &mapZ, &full_bar[s], kc, 0);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = idesc_bf16(TC_BM, a.Ntile);
    bool ok = true;
    for (int kt = 0; kt < nk && ok; ++kt) {
      const int s = kt % TC_STAGES;
      const uint32_t round = (uint32_t)(kt / TC_STAGES);
      if (!mbar_wait(&full_bar[s], round & 1, a.err)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t xaddr = smem_u32(smem + s * stage_bytes);
      const uint32_t zaddr = xaddr + xbytes;
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk) {
        // advance 16 BF16 = 32 bytes along K inside the 128-byte swizzle row
        mma_bf16(tmem, sdesc_sw128(xaddr + kk * 32), sdesc_sw128(zaddr + kk * 32), idesc,
                 (kt > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&empty_bar[s]);
    }
    if (ok) mma_commit(&done_bar);
  }

  // ---- epilogue: every warp reads its 32 accumulator lanes
  __syncwarp();
  bool ready = nk > 0 && mbar_wait(&done_bar, 0, a.err);
  ready = __all_sync(0xffffffffu, ready);  // tcgen05.ld needs the whole warp
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ready) {
    const int row = m0 + warp * 32 + lane;
    float* D = a.D + (int64_t)blockIdx.y * a.ldd * a.N;
    for (int c0 = 0; c0 < a.Ntile; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < a.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < a.N) D[row + (int64_t)(c0 + j) * a.ldd] = v[j];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols));
  }
}

__global__ void splitk_sum_f32_kernel(int M, int N, int splits, const float* __restrict__ part,
                                      int64_t ldp, float* __restrict__ D, int64_t ldd) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)M * N) return;
  int64_t i = idx % M, j = idx / M;
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += part[(int64_t)z * ldp * N + i + j * ldp];
  D[i + j * ldd] = s;
}

// ---------------------------------------------------------------------------
// Tensor maps via the driver entry point (no link-time libcuda dependency).
// ---------------------------------------------------------------------------

// rows x cols column-major bf16 matrix (rows contiguous = K), box 64 x box_cols.
Status make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
                int box_cols) {
  EncodeTiledFn fn = tensor_map_encoder();
  if (!fn) return make_error(LLS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * 2) % 16)
    return make_error(LLS_ERR_ARG, "bf16 operand must be 16-byte aligned with ld % 8 == 0");
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_cols};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return make_error(LLS_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return ok_status();
}

int num_sms() {
  static int n = -1;
  if (n < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 148;
  }
  return n;
}

}  // namespace

size_t tc_gemm_smem_bytes(int Ntile) {
  return 1024 + (size_t)TC_STAGES * (TC_BM * TC_BK * 2 + (size_t)Ntile * TC_BK * 2);
}

int tc_gemm_splits(int M, int K) {
  int tiles = (M + TC_BM - 1) / TC_BM;
  int ktiles = (K + TC_BK - 1) / TC_BK;
  int s = std::max(1, (num_sms() + tiles - 1) / tiles);
  s = std::min(s, std::max(1, ktiles / 4));  // at least 4 K tiles per split
  return std::min(s, 32);
}

size_t tc_gemm_scratch_bytes(int M, int N, int K) {
  int s = tc_gemm_splits(M, K);
  return s > 1 ? (size_t)s * M * N * sizeof(float) : 0;
}

Status tc_gemm_bf16(int M, int N, int K, const void* X, int64_t ldx, const void* Z, int64_t ldz,
                    float* D, int64_t ldd, Scratch scratch, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return ok_status();
  if (N > 128) return make_error(LLS_ERR_ARG, "tc_gemm_bf16: N > 128");
  const int Ntile = (N + 15) / 16 * 16;
  if (K <= 0) {
    LLS_CUDA(cudaMemset2DAsync(D, ldd * sizeof(float), 0, M * sizeof(float), N, st));
    return ok_status();
  }
  CUtensorMap mx, mz;
  LLS_TRY(make_map(&mx, X, K, M, ldx, TC_BM));
  LLS_TRY(make_map(&mz, Z, K, N, ldz, Ntile));
  int splits = tc_gemm_splits(M, K);
  if (splits > 1 && scratch.bytes < (size_t)splits * M * N * sizeof(float)) splits = 1;
  int ktiles = (K + TC_BK - 1) / TC_BK;
  int kchunk = ((ktiles + splits - 1) / splits) * TC_BK;
  splits = (K + kchunk - 1) / kchunk;  // every split has at least one K tile
  TcArgs a;
  a.M = M;
  a.N = N;
  a.Ntile = Ntile;
  a.K = K;
  a.kchunk = kchunk;
  a.err = err;
  uint32_t cols = 32;
  while (cols < (uint32_t)Ntile) cols <<= 1;
  a.tmem_cols = cols;
  if (splits > 1) {
    a.D = static_cast<float*>(scratch.ptr);
    a.ldd = M;
  } else {
    a.D = D;
    a.ldd = ldd;
  }
  size_t smem = tc_gemm_smem_bytes(Ntile);
  LLS_TRY(allow_max_dyn_smem((const void*)tc_gemm_bf16_kernel));
  dim3 grid((M + TC_BM - 1) / TC_BM, splits);
  {
    TraceScope ts(kTrBf16Gemm, st, 2.0 * M * N * K, 2.0 * ((double)M * K + (double)K * N) + 4.0 * M * N);
    tc_gemm_bf16_kernel<<<grid, TC_THREADS, smem, st>>>(mx, mz, a);
    LLS_LAUNCHED("tc_gemm_bf16_kernel");
  }
  if (splits > 1) {
    TraceScope ts(kTrSmall, st);
    splitk_sum_f32_kernel<<<(unsigned)ceil_div((int64_t)M * N, 256), 256, 0, st>>>(
        M, N, splits, static_cast<const float*>(scratch.ptr), M, D, ldd);
    LLS_LAUNCHED("splitk_sum_f32_kernel");
  }
  return ok_status();
}

}  // namespace lls

extern "C" int lls_k_gemm_bf16_tn(int64_t M, int64_t N, int64_t K, const void* X, int64_t ldx,
                                  const void* Z, int64_t ldz, float* D, int64_t ldd, int* status,
                                  void* stream) {
  if (M < 0 || N < 0 || K < 0 || N > 128 || M > INT32_MAX || K > INT32_MAX) return LLS_ERR_ARG;
  if (ldx < (K > 1 ? K : 1) || ldz < (K > 1 ? K : 1) || ldd < (M > 1 ? M : 1)) return LLS_ERR_ARG;
  if (M * N > 0 && (!D || !status || (K > 0 && (!X || !Z)))) return LLS_ERR_ARG;
  if (M * N == 0) return LLS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  lls::Scratch s;
  size_t need = lls::tc_gemm_scratch_bytes((int)M, (int)N, (int)K);
  if (need) {
    if (cudaMallocAsync(&s.ptr, need, st) != cudaSuccess) return LLS_ERR_NOMEM;
    s.bytes = need;
  }
  cudaMemsetAsync(status, 0, sizeof(int), st);
  lls::Status r = lls::tc_gemm_bf16((int)M, (int)N, (int)K, X, ldx, Z, ldz, D, ldd, s, status, st);
  if (s.ptr) cudaFreeAsync(s.ptr, st);
  return r.code;
}
