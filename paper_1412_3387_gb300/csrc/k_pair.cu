// Pair forces: dispatch over the (potential, precision) forms, each compiled
// in its own translation unit from pair_impl.cuh.
#include "md_internal.cuh"

namespace mdgb {

constexpr int kLJ = 0, kDPD = 1, kGauss = 2, kMorse = 3, kYukawa = 4, kTable = 5;

template <int POT, bool MIXED>
cudaError_t launch_pair_form(const KArgs &a, Launch l, int want_virial, cudaStream_t st);
template <int POT, bool MIXED>
int max_block_pair_form(int w, int want_virial);
template <int POT, bool MIXED>
void pair_form_attributes();

template <int POT>
void form_attributes() {
  pair_form_attributes<POT, true>();
  pair_form_attributes<POT, false>();
}

void pair_init_attributes() {
  form_attributes<kLJ>();
  form_attributes<kDPD>();
  form_attributes<kGauss>();
  form_attributes<kMorse>();
  form_attributes<kYukawa>();
  form_attributes<kTable>();
}

template <int POT>
cudaError_t launch_pot(const KArgs &a, Launch l, int want_virial, cudaStream_t st) {
  return a.mixed ? launch_pair_form<POT, true>(a, l, want_virial, st)
                 : launch_pair_form<POT, false>(a, l, want_virial, st);
}

cudaError_t launch_pair(const KArgs &a, Launch l, int want_virial, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  if (a.half && !a.mixed) {
    // half list: both particles of a pair add into their sums
    cudaError_t e = cudaMemsetAsync(a.force, 0, sizeof(double) * 4 * (size_t)a.n, st);
    if (e == cudaSuccess && want_virial)
      e = cudaMemsetAsync(a.virial, 0, sizeof(double) * 6 * (size_t)a.n, st);
    if (e != cudaSuccess) return e;
  }
  switch (a.pair) {
    case kLJ: return launch_pot<kLJ>(a, l, want_virial, st);
    case kDPD: return launch_pot<kDPD>(a, l, want_virial, st);
    case kGauss: return launch_pot<kGauss>(a, l, want_virial, st);
    case kMorse: return launch_pot<kMorse>(a, l, want_virial, st);
    case kYukawa: return launch_pot<kYukawa>(a, l, want_virial, st);
    case kTable: return launch_pot<kTable>(a, l, want_virial, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int POT>
int max_block_pot(const KArgs &a, int w, int want_virial) {
  return a.mixed ? max_block_pair_form<POT, true>(w, want_virial)
                 : max_block_pair_form<POT, false>(w, want_virial);
}

int max_block_pair(const KArgs &a, int w, int want_virial) {
  switch (a.pair) {
    case kLJ: return max_block_pot<kLJ>(a, w, want_virial);
    case kDPD: return max_block_pot<kDPD>(a, w, want_virial);
    case kGauss: return max_block_pot<kGauss>(a, w, want_virial);
    case kMorse: return max_block_pot<kMorse>(a, w, want_virial);
    case kYukawa: return max_block_pot<kYukawa>(a, w, want_virial);
    case kTable: return max_block_pot<kTable>(a, w, want_virial);
    default: return 0;
  }
}

}  // namespace mdgb
