// Pair kernels of one form (Gaussian, FP64); see pair_impl.cuh.
#include "pair_impl.cuh"

namespace mdgb {
MDGB_PAIR_FORM(kGauss, false)
}  // namespace mdgb
