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

// Guard-word debug mode (guard.cu, lls_debug_guard): buffers allocated
// while it is on carry guard bytes on both sides, checked after every launch.
extern std::atomic<int> g_guard_mode;
Status guard_alloc(size_t need, void** user);
void guard_free(void* user);
void guard_after_launch(const char* name);

// Launch check after a <<<>>> launch.
#define LLS_LAUNCHED(name)                                          \
  do {                                                              \
    ::lls::g_launches.fetch_add(1, std::memory_order_relaxed);      \
    LLS_CUDA(cudaGetLastError());                                   \
    if (::lls::g_guard_mode.load(std::memory_order_relaxed))        \
      ::lls::guard_after_launch(name);                              \
  } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// Device-side grid barrier for cooperative launches.  Every waiting CTA
// spins with a bounded number of polls; on running out it raises *err and
// returns false, so a kernel can exit instead of hanging.  The state is one
// arrival-count word that must be zero before the launch.
// ---------------------------------------------------------------------------
constexpr long long kBarrierSpinLimit = 1LL << 22;  // a few seconds of polling at most

// limit: polls a waiting CTA makes before it gives up; launchers take it
// from g_barrier_spin_limit (kBarrierSpinLimit unless a test lowered it
// through lls_debug_barrier_limit).
struct GridBarrier {
  unsigned int* count;
  int* err;
  long long limit = kBarrierSpinLimit;
};

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int* p) {
  return *reinterpret_cast<const volatile unsigned int*>(p);
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// Grid-wide barrier on a monotonically increasing arrival counter (reset to
// 0 before each launch; a launch passes at most 2^31 / CTAs barriers).  Each
// CTA counts its own barriers in `epoch` (a variable of the calling kernel,
// starting at 0), so thread 0 arrives with a fire-and-forget release add and
// waits, with acquire loads, until the counter reaches (epoch + 1) x CTAs.
// The wait is bounded (bar.limit polls); on expiry, or when another
// CTA has already failed, it sets *err and every thread of the CTA gets false.
__device__ inline bool grid_sync(const GridBarrier& bar, unsigned int& epoch) {
  __syncthreads();
  __shared__ int s_fail;
  if (threadIdx.x == 0) {
    s_fail = 0;
    const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int target = (epoch + 1) * nb;
    // release: this CTA's writes, ordered before it by the __syncthreads above,
    // are visible to whoever acquires the count (no separate fence needed)
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar.count) : "memory");
    long long it = 0;
    for (;;) {
      unsigned int cur;
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(bar.count) : "memory");
      if ((int)(cur - target) >= 0) break;
      if (++it > bar.limit || ((it & 255) == 0 && ld_volatile_i32(bar.err) != 0)) {
        atomicExch(bar.err, 1);
        s_fail = 1;
        break;
      }
      if (it > 4096) __nanosleep(64);
    }
  }
  ++epoch;
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
