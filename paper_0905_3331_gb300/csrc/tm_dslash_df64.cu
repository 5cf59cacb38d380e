// tm_dslash_df64.cu -- instantiation of the hopping kernel for TM_DF64 (double-float) storage
// and arithmetic: 18-real links, one thread per site, every epilogue.  (The double-word
// arithmetic makes each kernel several times larger than its FP32 sibling, so only this
// one configuration is built.)
#include "tm_dslash.cuh"

namespace tmq {
tm_status hop_launch_df64(tm_lattice lat, const HopArgs& a, cudaStream_t s) {
  if (a.nreal != 18) return set_error(TM_ERR_UNSUPPORTED, "double-float storage supports 18-real links only");
  return hop_launch_tps<TM_DF64, 18, 1, false>(lat, a, s);
}
}  // namespace tmq
