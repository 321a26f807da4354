// Warp-level sums of several FP64 values per lane with few FP64 adds.
#pragma once

namespace lls {

// Sum of V values per lane over the 32 lanes of a warp with FP64 adds on
// halves: while V is even, each step keeps half of the values (the lane's
// bit at the step's offset picks which) and adds the partner's copy of
// them, so a lane does V/2 + V/4 + ... adds instead of 5 V; the remaining
// offsets add whole sets.  Afterwards the lane holds the sums of the
// original values base .. base + V / 2^halvings - 1.
template <int V, int OFF>
struct WarpSumHalves {
  static __device__ __forceinline__ void run(double* v, int lane, int& base) {
    if constexpr (OFF == 0) {
      return;
    } else if constexpr (V % 2 == 0) {
      const bool up = (lane & OFF) != 0;
#pragma unroll
      for (int j = 0; j < V / 2; ++j) {
        const double send = up ? v[j] : v[j + V / 2];
        const double keep = up ? v[j + V / 2] : v[j];
        v[j] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
      }
      if (up) base += V / 2;
      WarpSumHalves<V / 2, OFF / 2>::run(v, lane, base);
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], OFF);
      WarpSumHalves<V, OFF / 2>::run(v, lane, base);
    }
  }
};
// Halvings of a V-value sum over 32 lanes (at most 5) and what remains.
constexpr int halvings(int V) { return (V % 2 == 0 && V > 1) ? 1 + (halvings(V / 2) < 4 ? halvings(V / 2) : 4) : 0; }

}  // namespace lls
