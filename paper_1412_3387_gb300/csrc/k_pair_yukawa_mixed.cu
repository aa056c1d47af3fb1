// Pair kernels of one form (Yukawa, mixed precision); see pair_impl.cuh.
#include "pair_impl.cuh"

namespace mdgb {
MDGB_PAIR_FORM(kYukawa, true)
}  // namespace mdgb
