// Pair forces: dispatch over the (potential, precision) forms, each compiled
// in its own translation unit from pair_impl.cuh.
#include "md_internal.cuh"

namespace mdgb {

constexpr int kLJ = 0, kDPD = 1;

template <int POT, bool MIXED>
cudaError_t launch_pair_form(const KArgs &a, Launch l, int want_virial, cudaStream_t st);
template <int POT, bool MIXED>
int max_block_pair_form(int w, int want_virial);
template <int POT, bool MIXED>
void pair_form_attributes();

void pair_init_attributes() {
  pair_form_attributes<kLJ, true>();
  pair_form_attributes<kLJ, false>();
  pair_form_attributes<kDPD, true>();
  pair_form_attributes<kDPD, false>();
}

cudaError_t launch_pair(const KArgs &a, Launch l, int want_virial, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const bool m = a.mixed != 0;
  if (a.pair == kLJ)
    return m ? launch_pair_form<kLJ, true>(a, l, want_virial, st)
             : launch_pair_form<kLJ, false>(a, l, want_virial, st);
  return m ? launch_pair_form<kDPD, true>(a, l, want_virial, st)
           : launch_pair_form<kDPD, false>(a, l, want_virial, st);
}

int max_block_pair(const KArgs &a, int w, int want_virial) {
  const bool m = a.mixed != 0;
  if (a.pair == kLJ)
    return m ? max_block_pair_form<kLJ, true>(w, want_virial)
             : max_block_pair_form<kLJ, false>(w, want_virial);
  return m ? max_block_pair_form<kDPD, true>(w, want_virial)
           : max_block_pair_form<kDPD, false>(w, want_virial);
}

}  // namespace mdgb
