// lls_k_panel_qr_noalloc: the Householder panel QR with its scratch in a
// fixed device array owned by the library, for callers that must not
// allocate device memory (see include/lls_kernels.h).
//
// Scratch of the cooperative panel kernels: the grid-barrier arrival
// counter and the partial sums (for the shared-memory kernel two buffers of
// one value per CTA and column, two copies of one row and two of the column
// totals; for the global-memory kernel one norm per CTA, one dot product per
// CTA and column and one reduced dot per column).  A barrier time-out is
// reported in the caller's status word, not in the array.  The array is
// sized by panel_qr.cu's own layout for its largest grid (kPanelMaxCtas
// CTAs) and 128 columns: 528,512 bytes (about 516 KiB).
#include <mutex>

#include "internal.h"
#include "lls_kernels.h"

namespace {

constexpr int64_t kNoAllocMaxCols = 128;
constexpr size_t kNoAllocBytes = lls::panel_qr_scratch_layout_bytes(lls::kPanelMaxCtas, kNoAllocMaxCols);
static_assert(kNoAllocBytes == 528512, "documented size of the fixed scratch array");

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_panel_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (the name is only a host-side stand-in, not a device address).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LLS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return LLS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_panel_scratch);
    if (e != cudaSuccess || !p) return LLS_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return LLS_OK;
}

}  // namespace

extern "C" int lls_k_panel_qr_noalloc(int64_t m, int64_t n, double* A, int64_t lda, double* tau,
                                      int* status, void* stream) {
  if (m < 0 || n < 0 || lda < (m > 1 ? m : 1)) return LLS_ERR_ARG;
  if (n > kNoAllocMaxCols) return LLS_ERR_CAPACITY;
  if (m == 0 || n == 0) return LLS_OK;
  if (!A || !tau || !status) return LLS_ERR_ARG;
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != LLS_OK) return rc;
  lls::Scratch s{base, kNoAllocBytes};
  if (lls::panel_qr_scratch_bytes(m, n) > s.bytes) return LLS_ERR_CAPACITY;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return LLS_ERR_CUDA;
  return lls::panel_qr(m, n, A, lda, tau, s, status, st).code;
}
