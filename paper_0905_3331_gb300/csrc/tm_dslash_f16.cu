// tm_dslash_f16.cu -- instantiation of the hopping kernel for TM_F16 spinor storage
// (all three link formats and every epilogue), compiled as its own translation unit.
#include "tm_dslash.cuh"

namespace tmq {
tm_status hop_launch_f16(tm_lattice lat, const HopArgs& a, cudaStream_t s) { return hop_launch_prec<TM_F16>(lat, a, s); }
}  // namespace tmq
