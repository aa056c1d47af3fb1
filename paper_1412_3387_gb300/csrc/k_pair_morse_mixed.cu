// Pair kernels of one form (Morse, mixed precision); see pair_impl.cuh.
#include "pair_impl.cuh"

namespace mdgb {
MDGB_PAIR_FORM(kMorse, true)
}  // namespace mdgb
