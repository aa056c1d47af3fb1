// Pair kernels of one form (Morse, FP64); see pair_impl.cuh.
#include "pair_impl.cuh"

namespace mdgb {
MDGB_PAIR_FORM(kMorse, false)
}  // namespace mdgb
