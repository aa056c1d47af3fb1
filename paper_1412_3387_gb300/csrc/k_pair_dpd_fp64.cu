// Pair kernels of one form (DPD, FP64); see pair_impl.cuh.
#include "pair_impl.cuh"

namespace mdgb {
MDGB_PAIR_FORM(kDPD, false)
}  // namespace mdgb
