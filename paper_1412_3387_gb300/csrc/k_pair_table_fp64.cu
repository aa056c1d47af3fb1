// Pair kernels of one form (tabulated, FP64); see pair_impl.cuh.
#include "pair_impl.cuh"

namespace mdgb {
MDGB_PAIR_FORM(kTable, false)
}  // namespace mdgb
