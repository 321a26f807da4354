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

namespace lls {
namespace {

struct U64x4 {
  uint64_t w[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                                uint64_t c3, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  U64x4 o;
  o.w[0] = c0;
  o.w[1] = c1;
  o.w[2] = c2;
  o.w[3] = c3;
  return o;
}

// Four normals of block (g, j), in row order 4g .. 4g+3.
__device__ __forceinline__ void block_normals(uint64_t seed, uint64_t step, uint64_t g,
                                              uint64_t j, double z[4]) {
  U64x4 w = philox4x64_10(g, j, step, 0ull, seed, 0ull);
  const double scale = 1.1102230246251565e-16;  // 2^-53
  const double two_pi = 6.283185307179586;      // fl(2 pi)
  double u0 = ((double)(w.w[0] >> 11) + 1.0) * scale;
  double t1 = (double)(w.w[1] >> 11) * scale;
  double u2 = ((double)(w.w[2] >> 11) + 1.0) * scale;
  double t3 = (double)(w.w[3] >> 11) * scale;
  double r0 = sqrt(-2.0 * log(u0));
  double r2 = sqrt(-2.0 * log(u2));
  double a1 = two_pi * t1, a3 = two_pi * t3;
  z[0] = r0 * cos(a1);
  z[1] = r0 * sin(a1);
  z[2] = r2 * cos(a3);
  z[3] = r2 * sin(a3);
}

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
