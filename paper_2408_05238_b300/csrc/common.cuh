// Internal helpers shared by the library's CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "lls.h"
#include "trace.h"

namespace lls {

// Status with a message, carried through the host driver.
struct Status {
  int code = LLS_OK;
  int arg = 0;
  std::string msg;
  bool ok() const { return code >= 0; }
};

inline Status ok_status() { return Status{}; }
inline Status make_error(int code, const std::string& msg, int arg = 0) {
  Status s;
  s.code = code;
  s.arg = arg;
  s.msg = msg;
  return s;
}

inline Status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return ok_status();
  return make_error(e == cudaErrorMemoryAllocation ? LLS_ERR_NOMEM : LLS_ERR_CUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
}

#define LLS_TRY(expr)                  \
  do {                                 \
    ::lls::Status _s = (expr);         \
    if (!_s.ok()) return _s;           \
  } while (0)

#define LLS_CUDA(call) LLS_TRY(::lls::cuda_status((call), #call))

// Launch check after a <<<>>> launch.
#define LLS_LAUNCHED(name)                                     \
  do {                                                         \
    ::lls::g_launches.fetch_add(1, std::memory_order_relaxed); \
    LLS_CUDA(cudaGetLastError());                              \
  } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// Device-side grid barrier for cooperative launches.  Every waiting CTA
// spins with a bounded number of polls; on running out it raises *err and
// returns false, so a kernel can exit instead of hanging.  The state is two
// words (arrival count, generation) that must be zero before the launch.
// ---------------------------------------------------------------------------
constexpr long long kBarrierSpinLimit = 1LL << 22;  // a few seconds of polling at most

struct GridBarrier {
  unsigned int* count;
  unsigned int* gen;
  int* err;
};

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int* p) {
  return *reinterpret_cast<const volatile unsigned int*>(p);
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

__device__ inline bool grid_sync(const GridBarrier& bar) {
  __syncthreads();
  __shared__ int s_fail;
  if (threadIdx.x == 0) {
    s_fail = 0;
    unsigned int g = ld_volatile_u32(bar.gen);
    __threadfence();
    unsigned int arrived = atomicAdd(bar.count, 1u);
    if (arrived == gridDim.x * gridDim.y * gridDim.z - 1) {
      atomicExch(bar.count, 0u);
      __threadfence();
      atomicAdd(bar.gen, 1u);
    } else {
      long long it = 0;
      while (ld_volatile_u32(bar.gen) == g) {
        if (++it > kBarrierSpinLimit || ld_volatile_i32(bar.err) != 0) {
          atomicExch(bar.err, 1);
          s_fail = 1;
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return s_fail == 0;
}

// Warp and block reductions (fixed order, so every CTA that reduces the same
// inputs gets bit-identical results).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace lls
