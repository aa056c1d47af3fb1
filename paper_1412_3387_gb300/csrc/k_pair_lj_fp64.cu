// Pair kernels of one form (LJ, FP64); see pair_impl.cuh.
#include "pair_impl.cuh"

namespace mdgb {
MDGB_PAIR_FORM(kLJ, false)
}  // namespace mdgb
