// tm_doublet.cuh -- shared declarations of the doublet operator (eq. Dh): the flavour-matrix
// epilogue and the two-flavour hopping launch.
#pragma once

#include "tm_internal.cuh"

namespace tmq {

// out_f = [G] ( sum_g P[c][f][g] y_g + Q[c][f][g] z_g ),  c = chirality (0: spins 0,1; 1: spins 2,3),
// P and Q complex 2x2 flavour matrices, G = gamma5 tau1 when `swap` is set.
struct DCoef {
  double P[2][2][2][2];  // [chirality][f_out][f_in][re, im]
  double Q[2][2][2][2];
  int swap;
  // the same rounded to FP32 once on the host (dcoef_finish), for the FP32 arithmetic of the
  // reduced-precision kernels: GB300 converts FP64 to FP32 on its narrow FP64 pipe
  float fP[2][2][2][2], fQ[2][2][2][2];
};
inline DCoef dcoef_finish(DCoef c) {
  constexpr int N = (int)(sizeof(c.P) / sizeof(c.P[0][0][0][0]));
  static_assert(sizeof(c.fP) / sizeof(c.fP[0][0][0][0]) == N && sizeof(c.Q) == sizeof(c.P), "coefficient sizes");
  for (int i = 0; i < N; ++i) {
    (&c.fP[0][0][0][0])[i] = (float)(&c.P[0][0][0][0])[i];
    (&c.fQ[0][0][0][0])[i] = (float)(&c.Q[0][0][0][0])[i];
  }
  return c;
}
// A coefficient as a complex number of the kernel's arithmetic type.
template <typename R>
__device__ __forceinline__ cpx<R> dco(const double (&d)[2], const float (&f)[2]) {
  if constexpr (sizeof(R) == 4)
    return mk<R>(f[0], f[1]);
  else
    return mk<R>((R)d[0], (R)d[1]);
}

// One two-flavour hopping application with the flavour epilogue (z = H in):
//   mode 0: out = epi;  1: out = epi, sum ||out||^2;  2: out (= r, FP64 for FP64 storage, FP32
//   otherwise) -= alpha epi, sum ||r||^2.  Fields are two one-flavour half fields back to back
//   (stride = bytes of one), r with rstride.
struct DHopArgs {
  int prec, nreal, out_parity;
  const void* in;
  size_t stride;
  void* out;
  size_t out_stride;
  const void* y;  // or null
  DCoef co;
  int mode;
  const CGState* alpha_src;  // mode 2: alpha from the state (1 if null)
  Reduce red;                // modes 1, 2
  const int* skip;
};

// Both flavours of each output site in one thread: each link is loaded once for the two
// flavours.  Storage TM_F64 (18-real links) and TM_F32 (18, 12, 8).
tm_status dhop_launch(tm_lattice lat, const DHopArgs& a, cudaStream_t s);

}  // namespace tmq
