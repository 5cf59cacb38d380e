// tm_dslash_pair_f32.cu -- instantiation of the two-sites-per-thread hopping kernel for TM_F32
// spinor storage (all three link formats and every epilogue), as its own translation unit.
#include "tm_dslash_pair.cuh"

namespace tmq {
tm_status hop_pair_launch_f32(tm_lattice lat, const HopArgs& a, cudaStream_t s) {
  return hop_pair_launch_prec<TM_F32>(lat, a, s);
}
}  // namespace tmq
