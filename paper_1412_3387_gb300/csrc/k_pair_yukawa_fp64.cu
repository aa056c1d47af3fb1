// Pair kernels of one form (Yukawa, FP64); see pair_impl.cuh.
#include "pair_impl.cuh"

namespace mdgb {
MDGB_PAIR_FORM(kYukawa, false)
}  // namespace mdgb
