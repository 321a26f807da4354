// CUDA runtime stand-ins for the host harness (test infrastructure): device
// memory is host memory, copies are memmove, streams are synchronous.  Fresh
// allocations are filled with NaN.
#include <cuda_runtime_api.h>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <cstdio>
extern "C" {
void** __cudaRegisterFatBinary(void*) { static void* h = nullptr; return &h; }
void __cudaRegisterFatBinaryEnd(void**) {}
void __cudaUnregisterFatBinary(void**) {}
}

cudaError_t cudaDeviceSynchronize() { return cudaSuccess; }
cudaError_t cudaFree(void* p) { free(p); return cudaSuccess; }
cudaError_t cudaFreeAsync(void* p, cudaStream_t) { free(p); return cudaSuccess; }
cudaError_t cudaFreeHost(void* p) { free(p); return cudaSuccess; }
const char* cudaGetErrorString(cudaError_t) { return "stand-in runtime"; }
cudaError_t cudaGetLastError() { return cudaSuccess; }
// poison fresh allocations so that reads of unwritten memory show up
static void* pmalloc(size_t n) {
  void* p = malloc(n);
  double* d = (double*)p;
  for (size_t i = 0; i < n / 8; ++i) d[i] = std::nan("");
  return p;
}
cudaError_t cudaMalloc(void** p, size_t n) { *p = pmalloc(n); return cudaSuccess; }
cudaError_t cudaMallocAsync(void** p, size_t n, cudaStream_t) { *p = pmalloc(n); return cudaSuccess; }
cudaError_t cudaMallocHost(void** p, size_t n) { *p = pmalloc(n); return cudaSuccess; }
cudaError_t cudaMemcpy(void* d, const void* s, size_t n, cudaMemcpyKind) { memmove(d, s, n); return cudaSuccess; }
cudaError_t cudaMemcpyAsync(void* d, const void* s, size_t n, cudaMemcpyKind, cudaStream_t) {
  memmove(d, s, n);
  return cudaSuccess;
}
cudaError_t cudaMemcpy2DAsync(void* d, size_t dp, const void* s, size_t sp, size_t w, size_t h,
                              cudaMemcpyKind, cudaStream_t) {
  for (size_t r = 0; r < h; ++r) memmove((char*)d + r * dp, (const char*)s + r * sp, w);
  return cudaSuccess;
}
cudaError_t cudaMemsetAsync(void* p, int v, size_t n, cudaStream_t) { memset(p, v, n); return cudaSuccess; }
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }

cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t) { return cudaSuccess; }
