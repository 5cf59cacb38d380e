// tm_dslash_f64.cu -- instantiation of the hopping kernel for TM_F64 spinor storage
// (all three link formats and every epilogue), compiled as its own translation unit.
#include "tm_dslash.cuh"

namespace tmq {
tm_status hop_launch_f64(tm_lattice lat, const HopArgs& a, cudaStream_t s) { return hop_launch_prec<TM_F64>(lat, a, s); }
}  // namespace tmq
