// Mixed-precision sampling (step a2 in BF16).  Placeholder until the
// tcgen05 kernels land: the mode is rejected.
#include "solver.h"

namespace lls {

Status sample_bf16(Handle&, const double*, int64_t, int64_t, int64_t, int64_t, int, uint64_t,
                   int64_t, double*, int64_t) {
  return make_error(LLS_ERR_ARG, "mixed precision sampling is not available in this build", 2);
}

}  // namespace lls
