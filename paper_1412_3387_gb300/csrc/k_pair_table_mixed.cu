// Pair kernels of one form (tabulated, mixed precision); see pair_impl.cuh.
#include "pair_impl.cuh"

namespace mdgb {
MDGB_PAIR_FORM(kTable, true)
}  // namespace mdgb
