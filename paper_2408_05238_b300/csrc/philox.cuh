// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the Box-Muller
// normals of the Gaussian sketch (Fig. 2, generate_iid_stdnorm_matrix):
// shared by the sketch kernels (sketch.cu) and the persistent batched
// factorization (batched_factor.cu), so both draw the same G.
#pragma once

#include <stdint.h>

namespace lls {
namespace rng {

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

}  // namespace rng
}  // namespace lls
