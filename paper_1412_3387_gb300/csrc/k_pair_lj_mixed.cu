// Pair kernels of one form (LJ, mixed precision); see pair_impl.cuh.
#include "pair_impl.cuh"

namespace mdgb {
MDGB_PAIR_FORM(kLJ, true)
}  // namespace mdgb
