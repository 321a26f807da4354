// Gaussian sketch G of Fig. 2 (generate_iid_stdnorm_matrix, step a1).
//
// Counter-based: entry (p, j) of the sketch of step `step` is a pure
// function of (seed, step, p, j), so the matrix is generated in parallel,
// needs no state between steps and is identical for every launch shape.
// Generator: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// two 64 x 64 -> 128-bit products of counter words 0 and 2, a permutation and
// an xor with the key, which is bumped by the two Weyl constants between
// rounds.  Block (g, j) has counter (g, j, step, 0), key (seed, 0); its four
// words give two Box-Muller pairs, i.e. rows 4g..4g+3 of column j.
#include <cuda_bf16.h>

#include "internal.h"
#include "lls_kernels.h"
#include "philox.cuh"

namespace lls {
namespace {

using namespace rng;


__global__ void philox_raw_kernel(uint64_t seed, uint64_t step, int64_t groups, int64_t cols,
                                  uint64_t* out) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= groups * cols) return;
  int64_t g = idx % groups, j = idx / groups;
  U64x4 w = philox4x64_10((uint64_t)g, (uint64_t)j, step, 0ull, seed, 0ull);
#pragma unroll
  for (int e = 0; e < 4; ++e) out[4 * idx + e] = w.w[e];
}

__global__ void sketch_kernel(uint64_t seed, uint64_t step, int64_t rows, int64_t cols,
                              double* G, int64_t ldg) {
  int64_t groups = (rows + 3) / 4;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= groups * cols) return;
  int64_t g = idx % groups, j = idx / groups;
  double z[4];
  block_normals(seed, step, (uint64_t)g, (uint64_t)j, z);
  double* col = G + j * ldg;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    int64_t p = 4 * g + e;
    if (p < rows) col[p] = z[e];
  }
}

__global__ void sketch_bf16_kernel(uint64_t seed, uint64_t step, int64_t rows, int64_t cols,
                                   __nv_bfloat16* G, int64_t ldg) {
  int64_t groups = (rows + 3) / 4;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= groups * cols) return;
  int64_t g = idx % groups, j = idx / groups;
  double z[4];
  block_normals(seed, step, (uint64_t)g, (uint64_t)j, z);
  __nv_bfloat16* col = G + j * ldg;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    int64_t p = 4 * g + e;
    if (p < rows) col[p] = __double2bfloat16(z[e]);
  }
}

}  // namespace

Status launch_philox_raw(uint64_t seed, int64_t step, int64_t groups, int64_t cols,
                         uint64_t* out, cudaStream_t st) {
  int64_t total = groups * cols;
  if (total <= 0) return ok_status();
  philox_raw_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(seed, (uint64_t)step,
                                                                    groups, cols, out);
  LLS_LAUNCHED("philox_raw_kernel");
  return ok_status();
}

Status launch_sketch(uint64_t seed, int64_t step, int64_t rows, int64_t cols, double* G,
                     int64_t ldg, cudaStream_t st) {
  int64_t total = ceil_div(rows, 4) * cols;
  if (rows <= 0 || cols <= 0) return ok_status();
  TraceScope ts(kTrSketch, st, 0.0, 8.0 * rows * cols);
  sketch_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(seed, (uint64_t)step, rows,
                                                                cols, G, ldg);
  LLS_LAUNCHED("sketch_kernel");
  return ok_status();
}

Status launch_sketch_bf16(uint64_t seed, int64_t step, int64_t rows, int64_t cols, void* G,
                          int64_t ldg, cudaStream_t st) {
  int64_t total = ceil_div(rows, 4) * cols;
  if (rows <= 0 || cols <= 0) return ok_status();
  TraceScope ts(kTrSketch, st, 0.0, 2.0 * rows * cols);
  sketch_bf16_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(
      seed, (uint64_t)step, rows, cols, static_cast<__nv_bfloat16*>(G), ldg);
  LLS_LAUNCHED("sketch_bf16_kernel");
  return ok_status();
}

}  // namespace lls

extern "C" int lls_k_philox(uint64_t seed, int64_t step, int64_t groups, int64_t cols,
                            uint64_t* out, void* stream) {
  if (groups < 0 || cols < 0 || step < 0) return LLS_ERR_ARG;
  if (groups * cols > 0 && !out) return LLS_ERR_ARG;
  return lls::launch_philox_raw(seed, step, groups, cols, out, (cudaStream_t)stream).code;
}

extern "C" int lls_k_sketch(uint64_t seed, int64_t step, int64_t rows, int64_t cols,
                            double* G, int64_t ldg, void* stream) {
  if (rows < 0 || cols < 0 || step < 0 || ldg < (rows > 1 ? rows : 1)) return LLS_ERR_ARG;
  if (rows * cols > 0 && !G) return LLS_ERR_ARG;
  return lls::launch_sketch(seed, step, rows, cols, G, ldg, (cudaStream_t)stream).code;
}
