// Pair kernels of one form (DPD, mixed precision); see pair_impl.cuh.
#include "pair_impl.cuh"

namespace mdgb {
MDGB_PAIR_FORM(kDPD, true)
}  // namespace mdgb
