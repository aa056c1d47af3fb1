// Pair kernels of one form (Gaussian, mixed precision); see pair_impl.cuh.
#include "pair_impl.cuh"

namespace mdgb {
MDGB_PAIR_FORM(kGauss, true)
}  // namespace mdgb
