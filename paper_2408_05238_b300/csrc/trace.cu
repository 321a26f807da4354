#include <cstring>

#include "lls.h"
#include "solver.h"
#include "trace.h"

namespace lls {

thread_local Tracer* g_tracer = nullptr;
std::atomic<int64_t> g_launches{0};
std::atomic<int64_t> g_allocs{0};
std::atomic<long long> g_barrier_spin_limit{kBarrierSpinLimit};

const char* trace_kind_name(int k) {
  static const char* names[kTrCount] = {"dgemm_kernel",      "splitk_reduce_kernel",
                                        "panel_qr_kernel",   "wy_tfactor_kernel",
                                        "sketch_kernel",     "jacobi_svd_kernel",
                                        "small_kernels",     "bf16_gemm_kernel",
                                        "convert_kernels",   "oz_mma_kernel",
                                        "tf32_mma_kernel",   "batched_factor_kernel",
                                        "thin_small_kernels", "thin_n_kernel",
                                        "thin_t_kernel",     "trsm_diag_kernel",
                                        "bf16_convert_kernels", "replay_kernel",
                                        "phase:sample",
                                        "phase:qr_y",
                                        "phase:right_update", "phase:panel",
                                        "phase:left_update", "phase:block_svd",
                                        "phase:rank",        "phase:nullify",
                                        "phase:solve",       "phase:refine"};
  return (k >= 0 && k < kTrCount) ? names[k] : "unknown";
}

cudaEvent_t Tracer::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Tracer::flush() {
  for (auto& r : recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess &&
        cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      launches[r.kind] += 1;
      seconds[r.kind] += ms * 1e-3;
      flops[r.kind] += r.flops;
      bytes[r.kind] += r.bytes;
    }
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  recs.clear();
}

void Tracer::reset() {
  flush();
  std::memset(launches, 0, sizeof(launches));
  std::memset(seconds, 0, sizeof(seconds));
  std::memset(flops, 0, sizeof(flops));
  std::memset(bytes, 0, sizeof(bytes));
}

Tracer::~Tracer() {
  for (auto& r : recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : pool) cudaEventDestroy(e);
}

}  // namespace lls

extern "C" {

int lls_trace_enable(lls_handle hh, int on) {
  lls::Handle* h = reinterpret_cast<lls::Handle*>(hh);
  if (!h) return LLS_ERR_ARG;
  if (on && !h->tracer) h->tracer.reset(new lls::Tracer());
  if (h->tracer) h->tracer->reset();
  h->trace_on = on != 0;
  return LLS_OK;
}

int lls_trace_read(lls_handle hh, lls_trace_stat* out, int64_t max, int64_t* count) {
  lls::Handle* h = reinterpret_cast<lls::Handle*>(hh);
  if (!h || !count || (max > 0 && !out)) return LLS_ERR_ARG;
  *count = 0;
  if (!h->tracer) return LLS_OK;
  h->tracer->flush();
  int64_t c = 0;
  for (int k = 0; k < lls::kTrCount; ++k) {
    if (!h->tracer->launches[k]) continue;
    if (c < max) {
      lls_trace_stat& s = out[c];
      std::memset(&s, 0, sizeof(s));
      std::strncpy(s.name, lls::trace_kind_name(k), sizeof(s.name) - 1);
      s.launches = h->tracer->launches[k];
      s.seconds = h->tracer->seconds[k];
      s.flops = h->tracer->flops[k];
      s.bytes = h->tracer->bytes[k];
    }
    ++c;
  }
  *count = c;
  return LLS_OK;
}

int64_t lls_launch_count(void) { return lls::g_launches.load(); }
int64_t lls_alloc_count(void) { return lls::g_allocs.load(); }

}  // extern "C"
