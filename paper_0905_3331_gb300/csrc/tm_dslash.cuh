// tm_dslash.cuh -- the hopping kernel H_{p,1-p} (eq. eo0 bracket, Sec. 4.1) with fused
// site-diagonal epilogues (eq. eo2, eo3) and fused FP64 reductions.
//
// One thread computes one output site of one right-hand side:
//   out(x) = sum_mu [ U_mu(x) (1 + gamma_mu) in(x + mu^) + U_mu(x - mu^)^dag (1 - gamma_mu) in(x - mu^) ]
// For each of the 8 hops the neighbour spinor is projected onto two spin components first
// (Sec. 4.1: (1 +- gamma_mu) psi has two independent spin components), the two colour
// vectors are multiplied by the link, and the lower two spin components are rebuilt from
// the upper two.  The projections below follow from the gamma matrices of App. A, with
// s = +1 for the forward hop (1 + gamma_mu) and s = -1 for the backward hop (1 - gamma_mu):
//   mu = t: h0 = p0 - s p2,   h1 = p1 - s p3;   out2 += -s U h0,  out3 += -s U h1
//   mu = x: h0 = p0 - i s p3, h1 = p1 - i s p2; out2 += i s U h1, out3 += i s U h0
//   mu = y: h0 = p0 - s p3,   h1 = p1 + s p2;   out2 += s U h1,   out3 += -s U h0
//   mu = z: h0 = p0 - i s p2, h1 = p1 + i s p3; out2 += i s U h0, out3 += -i s U h1
// and out0 += U h0, out1 += U h1 in every direction (U^dag for the backward hops).  Fermions
// are antiperiodic in time (Sec. 2.4): the hop across t = T-1 <-> 0 is multiplied by -1.
#pragma once

#include "tm_internal.cuh"

namespace tmq {

constexpr int HOP_NT = 128;  // threads per block of the batched and doublet hopping kernels
// The one-flavour hopping kernel runs hop_spb(TPS) output sites per block with TPS threads each:
// 64 sites (32 with 4 threads per site, whose partial sums would not fit the static shared
// memory otherwise).  1024 blocks for 16^3 x 32 spread evenly over 152 SMs (6.7 per SM) where
// 128-site blocks left a 3-vs-4-block imbalance.
constexpr int hop_spb(int tps) { return tps == 4 ? 32 : 64; }

template <typename R, int MU, int S>
__device__ __forceinline__ void project(const cpx<R> p[12], cpx<R> h0[3], cpx<R> h1[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cpx<R> p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
    if (MU == 0) {
      h0[c] = (S > 0) ? p0 - p2 : p0 + p2;
      h1[c] = (S > 0) ? p1 - p3 : p1 + p3;
    } else if (MU == 1) {
      h0[c] = (S > 0) ? p0 - times_i(p3) : p0 + times_i(p3);
      h1[c] = (S > 0) ? p1 - times_i(p2) : p1 + times_i(p2);
    } else if (MU == 2) {
      h0[c] = (S > 0) ? p0 - p3 : p0 + p3;
      h1[c] = (S > 0) ? p1 + p2 : p1 - p2;
    } else {
      h0[c] = (S > 0) ? p0 - times_i(p2) : p0 + times_i(p2);
      h1[c] = (S > 0) ? p1 + times_i(p3) : p1 - times_i(p3);
    }
  }
}

template <typename R, int MU, int S>
__device__ __forceinline__ void accumulate(cpx<R> acc[12], const cpx<R> u0[3], const cpx<R> u1[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc[a] = acc[a] + u0[a];
    acc[3 + a] = acc[3 + a] + u1[a];
    if (MU == 0) {
      acc[6 + a] = (S > 0) ? acc[6 + a] - u0[a] : acc[6 + a] + u0[a];
      acc[9 + a] = (S > 0) ? acc[9 + a] - u1[a] : acc[9 + a] + u1[a];
    } else if (MU == 1) {
      acc[6 + a] = (S > 0) ? acc[6 + a] + times_i(u1[a]) : acc[6 + a] - times_i(u1[a]);
      acc[9 + a] = (S > 0) ? acc[9 + a] + times_i(u0[a]) : acc[9 + a] - times_i(u0[a]);
    } else if (MU == 2) {
      acc[6 + a] = (S > 0) ? acc[6 + a] + u1[a] : acc[6 + a] - u1[a];
      acc[9 + a] = (S > 0) ? acc[9 + a] - u0[a] : acc[9 + a] + u0[a];
    } else {
      acc[6 + a] = (S > 0) ? acc[6 + a] + times_i(u0[a]) : acc[6 + a] - times_i(u0[a]);
      acc[9 + a] = (S > 0) ? acc[9 + a] - times_i(u1[a]) : acc[9 + a] + times_i(u1[a]);
    }
  }
}

template <typename R>
__device__ __forceinline__ void su3_mul2(const Mat3<R>& U, const cpx<R> h0[3], const cpx<R> h1[3],
                                         cpx<R> u0[3], cpx<R> u1[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u0[a] = U.m[a][0] * h0[0] + U.m[a][1] * h0[1] + U.m[a][2] * h0[2];
    u1[a] = U.m[a][0] * h1[0] + U.m[a][1] * h1[1] + U.m[a][2] * h1[2];
  }
}

// u = U^dag h for two colour vectors
template <typename R>
__device__ __forceinline__ void su3_adj_mul2(const Mat3<R>& U, const cpx<R> h0[3], const cpx<R> h1[3],
                                             cpx<R> u0[3], cpx<R> u1[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u0[a] = cjmul(U.m[0][a], h0[0]) + cjmul(U.m[1][a], h0[1]) + cjmul(U.m[2][a], h0[2]);
    u1[a] = cjmul(U.m[0][a], h1[0]) + cjmul(U.m[1][a], h1[1]) + cjmul(U.m[2][a], h1[2]);
  }
}

// ------------------------------------------------------------ direction pairs ---
// The forward and backward hops of one direction mu reach the lower two spin components of the
// output through the same fixed map P_mu (the +1 column of the table at the top) with opposite
// signs: upper += u+ + u-, lower += P_mu (u+ - u-), u+- = U(+-) h(+-) the two-spinor results of
// the hops.  So a pair forms s = u+ + u- by continuing the FMA chains of u+ with the backward
// products, d = 2 u+ - s with one FMA per real, and adds s and P_mu d to the accumulator: 12 +
// 12 adds per real pair instead of 2 x 24, and every colour row is one FMA chain (the product
// form a*b + c*d + ... with separate multiplies and adds took 30% DMUL and 43% DADD of the FP64
// pipe).  FP64 / FP32 / FP16 storage; double-float keeps the per-hop form (no fused FMA).

// u = U h for two colour vectors, each real part one chain
template <typename R>
__device__ __forceinline__ void su3_mul2_fma(const Mat3<R>& U, const cpx<R> h0[3], const cpx<R> h1[3], cpx<R> u0[3],
                                             cpx<R> u1[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R r0 = U.m[a][0].re * h0[0].re, i0 = U.m[a][0].re * h0[0].im;
    R r1 = U.m[a][0].re * h1[0].re, i1 = U.m[a][0].re * h1[0].im;
    r0 = fmadd(-U.m[a][0].im, h0[0].im, r0);
    i0 = fmadd(U.m[a][0].im, h0[0].re, i0);
    r1 = fmadd(-U.m[a][0].im, h1[0].im, r1);
    i1 = fmadd(U.m[a][0].im, h1[0].re, i1);
#pragma unroll
    for (int b = 1; b < 3; ++b) {
      r0 = fmadd(U.m[a][b].re, h0[b].re, r0);
      r0 = fmadd(-U.m[a][b].im, h0[b].im, r0);
      i0 = fmadd(U.m[a][b].re, h0[b].im, i0);
      i0 = fmadd(U.m[a][b].im, h0[b].re, i0);
      r1 = fmadd(U.m[a][b].re, h1[b].re, r1);
      r1 = fmadd(-U.m[a][b].im, h1[b].im, r1);
      i1 = fmadd(U.m[a][b].re, h1[b].im, i1);
      i1 = fmadd(U.m[a][b].im, h1[b].re, i1);
    }
    u0[a] = mk<R>(r0, i0);
    u1[a] = mk<R>(r1, i1);
  }
}

// s = u + U^dag h for two colour vectors: the chains continue from u
template <typename R>
__device__ __forceinline__ void su3_adj_mul2_add(const Mat3<R>& U, const cpx<R> h0[3], const cpx<R> h1[3],
                                                 const cpx<R> u0[3], const cpx<R> u1[3], cpx<R> s0[3],
                                                 cpx<R> s1[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R r0 = u0[a].re, i0 = u0[a].im, r1 = u1[a].re, i1 = u1[a].im;
#pragma unroll
    for (int b = 0; b < 3; ++b) {  // conj(U[b][a]) h[b]
      r0 = fmadd(U.m[b][a].re, h0[b].re, r0);
      r0 = fmadd(U.m[b][a].im, h0[b].im, r0);
      i0 = fmadd(U.m[b][a].re, h0[b].im, i0);
      i0 = fmadd(-U.m[b][a].im, h0[b].re, i0);
      r1 = fmadd(U.m[b][a].re, h1[b].re, r1);
      r1 = fmadd(U.m[b][a].im, h1[b].im, r1);
      i1 = fmadd(U.m[b][a].re, h1[b].im, i1);
      i1 = fmadd(-U.m[b][a].im, h1[b].re, i1);
    }
    s0[a] = mk<R>(r0, i0);
    s1[a] = mk<R>(r1, i1);
  }
}

// Projection of one hop's neighbour spinor with the FP16 per-site norm and the boundary sign.
template <int PREC, int MU, int S>
__device__ __forceinline__ void project_scaled(const cpx<typename SpinorFmt<PREC>::real> p[12],
                                               typename SpinorFmt<PREC>::real scale, bool negate,
                                               cpx<typename SpinorFmt<PREC>::real> h0[3],
                                               cpx<typename SpinorFmt<PREC>::real> h1[3]) {
  typedef typename SpinorFmt<PREC>::real R;
  project<R, MU, S>(p, h0, h1);
  if (SpinorFmt<PREC>::has_norm) {
    const R f = (MU == 0 && negate) ? -scale : scale;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h0[c] = f * h0[c];
      h1[c] = f * h1[c];
    }
  } else if (MU == 0 && negate) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h0[c] = mk<R>(-h0[c].re, -h0[c].im);
      h1[c] = mk<R>(-h1[c].re, -h1[c].im);
    }
  }
}

// First half of a pair: u = U_mu(x) (1 + gamma_mu) in(x + mu^), projected, with the link given
// as a matrix (pair_fwd below reconstructs it from its stored words first).
template <int PREC, int MU>
__device__ __forceinline__ void pair_fwd_mat(cpx<typename SpinorFmt<PREC>::real> u0[3],
                                             cpx<typename SpinorFmt<PREC>::real> u1[3],
                                             const Mat3<typename SpinorFmt<PREC>::real>& U,
                                             const cpx<typename SpinorFmt<PREC>::real> p[12],
                                             typename SpinorFmt<PREC>::real scale, bool negate) {
  typedef typename SpinorFmt<PREC>::real R;
  cpx<R> h0[3], h1[3];
  project_scaled<PREC, MU, +1>(p, scale, negate, h0, h1);
  su3_mul2_fma(U, h0, h1, u0, u1);
}

// ---- FP16 storage: the projection straight from the stored half words.  Each projected real
// a +- b of two stored halves is one conversion of b and one mixed-precision add of a
// (add/sub.rn.f32.f16: a half operand, FP32 result), not two conversions and an FP32 add: 12 FP32
// pipe instructions per hop fewer.  The sum is exact in FP32 as in the converted form (two
// halves), so the results are bitwise those of the converted projection.
__device__ __forceinline__ unsigned short lo16(unsigned int w) { return (unsigned short)(w & 0xffffu); }
__device__ __forceinline__ unsigned short hi16(unsigned int w) { return (unsigned short)(w >> 16); }
__device__ __forceinline__ float cvt16(unsigned short a) { return __half2float(__ushort_as_half(a)); }
__device__ __forceinline__ float hadd32(unsigned short a, float c) {
  float d;
  asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
  return d;
}
__device__ __forceinline__ float hsub32(unsigned short a, float c) {
  float d;
  asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
  return d;
}
// a + q b for complex halves a, b (re low, im high) and q = +1 (Q 0), -1 (1), +i (2), -i (3)
template <int Q>
__device__ __forceinline__ cpx<float> padd16(unsigned int a, unsigned int b) {
  if (Q == 0) return mk<float>(hadd32(lo16(a), cvt16(lo16(b))), hadd32(hi16(a), cvt16(hi16(b))));
  if (Q == 1) return mk<float>(hsub32(lo16(a), cvt16(lo16(b))), hsub32(hi16(a), cvt16(hi16(b))));
  if (Q == 2) return mk<float>(hsub32(lo16(a), cvt16(hi16(b))), hadd32(hi16(a), cvt16(lo16(b))));
  return mk<float>(hadd32(lo16(a), cvt16(hi16(b))), hsub32(hi16(a), cvt16(lo16(b))));
}
// (1 + S gamma_MU) p projected (the table at the top), p the 12 half words of a site
template <int MU, int S>
__device__ __forceinline__ void project16(const unsigned int w[12], cpx<float> h0[3], cpx<float> h1[3]) {
  constexpr int Q0 = MU == 0 || MU == 2 ? (S > 0 ? 1 : 0) : (S > 0 ? 3 : 2);
  constexpr int Q1 = MU == 0 ? (S > 0 ? 1 : 0) : (MU == 1 ? (S > 0 ? 3 : 2) : (MU == 2 ? (S > 0 ? 0 : 1) : (S > 0 ? 2 : 3)));
  constexpr int J0 = (MU == 0 || MU == 3) ? 6 : 9;  // partner of p0: p2 or p3
  constexpr int J1 = (MU == 0 || MU == 3) ? 9 : 6;  // partner of p1: p3 or p2
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    h0[c] = padd16<Q0>(w[c], w[J0 + c]);
    h1[c] = padd16<Q1>(w[3 + c], w[J1 + c]);
  }
}

template <int MU, int S>
__device__ __forceinline__ void project16_scaled(const unsigned int w[13], bool negate, cpx<float> h0[3], cpx<float> h1[3]) {
  project16<MU, S>(w, h0, h1);
  const float n = __uint_as_float(w[12]);
  const float f = (MU == 0 && negate) ? -n : n;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    h0[c] = f * h0[c];
    h1[c] = f * h1[c];
  }
}

template <int PREC, int NREAL, int MU>
__device__ __forceinline__ void pair_fwd(cpx<typename SpinorFmt<PREC>::real> u0[3],
                                         cpx<typename SpinorFmt<PREC>::real> u1[3],
                                         const RawWords<NREAL * LinkStore<PREC>::size>& raw,
                                         const cpx<typename SpinorFmt<PREC>::real> p[12],
                                         typename SpinorFmt<PREC>::real scale, bool negate) {
  typedef typename SpinorFmt<PREC>::real R;
  Mat3<R> U;
  LinkRecon<R, typename LinkStore<PREC>::type, NREAL>::unpack(raw, U);
  pair_fwd_mat<PREC, MU>(u0, u1, U, p, scale, negate);
}

// Second half: the backward hop U_mu(x - mu^)^dag (1 - gamma_mu) in(x - mu^) completes the pair,
// which is added to the accumulator (written, for the first pair of the accumulator).
// The backward hop from its projected half spinor (h0, h1) onward.
template <typename R, int MU, bool FIRST>
__device__ __forceinline__ void pair_bwd_proj(cpx<R> acc[12], const cpx<R> u0[3], const cpx<R> u1[3], const Mat3<R>& U,
                                              const cpx<R> h0[3], const cpx<R> h1[3]) {
  cpx<R> s0[3], s1[3];
  su3_adj_mul2_add(U, h0, h1, u0, u1, s0, s1);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const cpx<R> d0 = mk<R>(fmadd(R(2), u0[a].re, -s0[a].re), fmadd(R(2), u0[a].im, -s0[a].im));
    const cpx<R> d1 = mk<R>(fmadd(R(2), u1[a].re, -s1[a].re), fmadd(R(2), u1[a].im, -s1[a].im));
    cpx<R> l2, l3;  // P_mu d
    if (MU == 0) {
      l2 = mk<R>(-d0.re, -d0.im);
      l3 = mk<R>(-d1.re, -d1.im);
    } else if (MU == 1) {
      l2 = times_i(d1);
      l3 = times_i(d0);
    } else if (MU == 2) {
      l2 = d1;
      l3 = mk<R>(-d0.re, -d0.im);
    } else {
      l2 = times_i(d0);
      l3 = mk<R>(d1.im, -d1.re);  // -i d1
    }
    if (FIRST) {
      acc[a] = s0[a];
      acc[3 + a] = s1[a];
      acc[6 + a] = l2;
      acc[9 + a] = l3;
    } else {
      acc[a] = acc[a] + s0[a];
      acc[3 + a] = acc[3 + a] + s1[a];
      acc[6 + a] = acc[6 + a] + l2;
      acc[9 + a] = acc[9 + a] + l3;
    }
  }
}

template <int PREC, int MU, bool FIRST>
__device__ __forceinline__ void pair_bwd_mat(cpx<typename SpinorFmt<PREC>::real> acc[12],
                                             const cpx<typename SpinorFmt<PREC>::real> u0[3],
                                             const cpx<typename SpinorFmt<PREC>::real> u1[3],
                                             const Mat3<typename SpinorFmt<PREC>::real>& U,
                                             const cpx<typename SpinorFmt<PREC>::real> p[12],
                                             typename SpinorFmt<PREC>::real scale, bool negate) {
  typedef typename SpinorFmt<PREC>::real R;
  cpx<R> h0[3], h1[3];
  project_scaled<PREC, MU, -1>(p, scale, negate, h0, h1);
  pair_bwd_proj<R, MU, FIRST>(acc, u0, u1, U, h0, h1);
}

template <int PREC, int NREAL, int MU, bool FIRST>
__device__ __forceinline__ void pair_bwd(cpx<typename SpinorFmt<PREC>::real> acc[12],
                                         const cpx<typename SpinorFmt<PREC>::real> u0[3],
                                         const cpx<typename SpinorFmt<PREC>::real> u1[3],
                                         const RawWords<NREAL * LinkStore<PREC>::size>& raw,
                                         const cpx<typename SpinorFmt<PREC>::real> p[12],
                                         typename SpinorFmt<PREC>::real scale, bool negate) {
  typedef typename SpinorFmt<PREC>::real R;
  Mat3<R> U;
  LinkRecon<R, typename LinkStore<PREC>::type, NREAL>::unpack(raw, U);
  pair_bwd_mat<PREC, MU, FIRST>(acc, u0, u1, U, p, scale, negate);
}

// Both hops of direction mu, loads then arithmetic.
template <int PREC, int NREAL, int MU, bool FIRST>
__device__ __forceinline__ void hop_pair(cpx<typename SpinorFmt<PREC>::real> acc[12], const void* in, int h,
                                         int nbf, const char* slabf, int lif, bool negf, int nbb, const char* slabb,
                                         int lib, bool negb) {
  typedef typename SpinorFmt<PREC>::real R;
  constexpr int BYTES = NREAL * LinkStore<PREC>::size;
  const RawWords<BYTES> rf = load_raw<BYTES>(slabf, h, lif);
  const RawWords<BYTES> rb = load_raw<BYTES>(slabb, h, lib);
  cpx<R> u0[3], u1[3];
  if constexpr (PREC == TM_F16) {
    unsigned int w[13];
    cpx<float> h0[3], h1[3];
    Mat3<float> U;
    SpinorFmt<TM_F16>::load_words(in, h, nbf, w);
    project16_scaled<MU, +1>(w, negf, h0, h1);
    LinkRecon<float, __half, NREAL>::unpack(rf, U);
    su3_mul2_fma(U, h0, h1, u0, u1);
    SpinorFmt<TM_F16>::load_words(in, h, nbb, w);
    project16_scaled<MU, -1>(w, negb, h0, h1);
    LinkRecon<float, __half, NREAL>::unpack(rb, U);
    pair_bwd_proj<float, MU, FIRST>(acc, u0, u1, U, h0, h1);
  } else {
    cpx<R> p[12];
    R scale;
    SpinorFmt<PREC>::load_unscaled(in, h, nbf, p, scale);
    pair_fwd<PREC, NREAL, MU>(u0, u1, rf, p, scale, negf);
    SpinorFmt<PREC>::load_unscaled(in, h, nbb, p, scale);
    pair_bwd<PREC, NREAL, MU, FIRST>(acc, u0, u1, rb, p, scale, negb);
  }
}

// One hop.  Forward (S = +1): link U_mu(x) from the output parity's slab at the output site.
// Backward (S = -1): link U_mu(x - mu^) from the other parity's slab at the neighbour's index,
// applied as its adjoint -- the same stored link serves both hops, so the operator keeps
// gamma5-hermiticity exactly in every storage format.  hop_apply does the arithmetic on the
// loaded link words and neighbour spinor (FP16: unscaled, with its per-site norm).
template <int PREC, int NREAL, int MU, int S>
__device__ __forceinline__ void hop_apply(cpx<typename SpinorFmt<PREC>::real> acc[12],
                                          const RawWords<NREAL * LinkStore<PREC>::size>& raw,
                                          const cpx<typename SpinorFmt<PREC>::real> p[12],
                                          typename SpinorFmt<PREC>::real scale, bool negate) {
  typedef typename SpinorFmt<PREC>::real R;
  typedef typename LinkStore<PREC>::type St;
  cpx<R> h0[3], h1[3];
  project<R, MU, S>(p, h0, h1);
  if (SpinorFmt<PREC>::has_norm) {
    // FP16 per-site norm and the boundary sign, applied to the 6 projected components
    const R f = (MU == 0 && negate) ? -scale : scale;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h0[c] = f * h0[c];
      h1[c] = f * h1[c];
    }
  } else if (MU == 0 && negate) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h0[c] = R(-1) * h0[c];
      h1[c] = R(-1) * h1[c];
    }
  }
  Mat3<R> U;
  LinkRecon<R, St, NREAL>::unpack(raw, U);
  cpx<R> u0[3], u1[3];
  if (S > 0)
    su3_mul2(U, h0, h1, u0, u1);
  else
    su3_adj_mul2(U, h0, h1, u0, u1);
  accumulate<R, MU, S>(acc, u0, u1);
}

template <int PREC, int NREAL, int MU, int S>
__device__ __forceinline__ void hop_dir(cpx<typename SpinorFmt<PREC>::real> acc[12], const void* in, int h,
                                        int nbi, const char* slab, int link_index, bool negate) {
  typedef typename SpinorFmt<PREC>::real R;
  constexpr int BYTES = NREAL * LinkStore<PREC>::size;
  RawWords<BYTES> raw = load_raw<BYTES>(slab, h, link_index);
  cpx<R> p[12];
  R scale;
  SpinorFmt<PREC>::load_unscaled(in, h, nbi, p, scale);
  hop_apply<PREC, NREAL, MU, S>(acc, raw, p, scale, negate);
}

// Software-pipelined form (FP32 / FP16 storage, one thread per site): the link and spinor
// words of the next hop are loaded before the current hop's arithmetic, so each thread keeps
// two hops' loads in flight instead of waiting out eight load latencies one after another.
// For lattices that fill less than a wave the launch time is this per-thread chain.
template <int PREC, int NREAL>
struct HopWords {
  RawWords<NREAL * LinkStore<PREC>::size> link;
  unsigned int sp[SpinorFmt<PREC>::bytes_per_site / 4];
};

template <int PREC, int NREAL>
__device__ __forceinline__ void hop_fetch(HopWords<PREC, NREAL>& d, const char* in, int h, int nbi,
                                          const char* slab, int link_index) {
  d.link = load_raw<NREAL * LinkStore<PREC>::size>(slab, h, link_index);
  SpinorFmt<PREC>::load_words(in, h, nbi, d.sp);
}

template <int PREC, int NREAL>
__device__ __forceinline__ void hop_all_pipelined(cpx<typename SpinorFmt<PREC>::real> acc[12], const Geom& g,
                                                  int cb, const SiteCoord& c, const int nb[8], const char* inr,
                                                  const char* lf, const char* lo, size_t slab) {
  typedef typename SpinorFmt<PREC>::real R;
  const bool tfwd = (c.t == g.T - 1), tbwd = (c.t == 0);
  HopWords<PREC, NREAL> A, B;  // forward and backward hop of the current direction
  cpx<R> u0[3], u1[3], p[12];
  R scale;
  hop_fetch(A, inr, g.h, nb[0], lf + 0 * slab, cb);
  hop_fetch(B, inr, g.h, nb[4], lo + 0 * slab, nb[4]);
#define TM_PIPE_FWD(MU, NEG)                                                  \
  if constexpr (PREC == TM_F16) {                                             \
    cpx<float> h0[3], h1[3];                                                  \
    Mat3<float> U;                                                            \
    project16_scaled<MU, +1>(A.sp, NEG, h0, h1);                              \
    LinkRecon<float, __half, NREAL>::unpack(A.link, U);                       \
    su3_mul2_fma(U, h0, h1, u0, u1);                                          \
  } else {                                                                    \
    SpinorFmt<PREC>::unpack_words(A.sp, p, scale);                            \
    pair_fwd<PREC, NREAL, MU>(u0, u1, A.link, p, scale, NEG);                 \
  }
#define TM_PIPE_BWD(MU, FIRST, NEG)                                           \
  if constexpr (PREC == TM_F16) {                                             \
    cpx<float> h0[3], h1[3];                                                  \
    Mat3<float> U;                                                            \
    project16_scaled<MU, -1>(B.sp, NEG, h0, h1);                              \
    LinkRecon<float, __half, NREAL>::unpack(B.link, U);                       \
    pair_bwd_proj<float, MU, FIRST>(acc, u0, u1, U, h0, h1);                  \
  } else {                                                                    \
    SpinorFmt<PREC>::unpack_words(B.sp, p, scale);                            \
    pair_bwd<PREC, NREAL, MU, FIRST>(acc, u0, u1, B.link, p, scale, NEG);     \
  }
  TM_PIPE_FWD(0, tfwd)
  hop_fetch(A, inr, g.h, nb[1], lf + 1 * slab, cb);
  TM_PIPE_BWD(0, true, tbwd)
  hop_fetch(B, inr, g.h, nb[5], lo + 1 * slab, nb[5]);
  TM_PIPE_FWD(1, false)
  hop_fetch(A, inr, g.h, nb[2], lf + 2 * slab, cb);
  TM_PIPE_BWD(1, false, false)
  hop_fetch(B, inr, g.h, nb[6], lo + 2 * slab, nb[6]);
  TM_PIPE_FWD(2, false)
  hop_fetch(A, inr, g.h, nb[3], lf + 3 * slab, cb);
  TM_PIPE_BWD(2, false, false)
  hop_fetch(B, inr, g.h, nb[7], lo + 3 * slab, nb[7]);
  TM_PIPE_FWD(3, false)
  TM_PIPE_BWD(3, false, false)
#undef TM_PIPE_FWD
#undef TM_PIPE_BWD
}

// MODE 0: out = epi(hop).  MODE 1: same plus sum ||out||^2.
// MODE 2: out buffer holds r (FP64 for FP64 storage, FP32 otherwise); r <- r - alpha * epi(hop),
// plus sum ||r||^2.
// MODE 3 (with y, FP64): out = D t with t = c hop + E y, plus sum ||t - M out||^2 with M the
// inverse of D (coef.m): the residual of the site-diagonal solve M out = t that produced out,
// from the hopping sum already in registers.
//
// TPS (threads per site) = 1, 2 or 4.  With TPS > 1 the 8 hops of a site are split over TPS
// warps of the block (part q takes the directions q*4/TPS .. (q+1)*4/TPS - 1, both hops of
// each), so the branch on the part is warp-uniform; the partial sums meet in shared memory,
// are added in part order 0, 1, ..., and part q finishes the storage blocks
// [NBLK q / TPS, NBLK (q + 1) / TPS) of the site.  More threads per site give more memory
// requests in flight for lattices too small to fill the GPU with one thread per site.
template <int PREC, int NREAL, int TPS>
__device__ __forceinline__ void hop_part(cpx<typename SpinorFmt<PREC>::real> acc[12], const Geom& g, int cb,
                                         const SiteCoord& c, const int nb[8], const char* inr, const char* lf,
                                         const char* lo, size_t slab, int part) {
  const bool tfwd = (c.t == g.T - 1), tbwd = (c.t == 0);
  if constexpr (PREC == TM_DF64) {  // per hop (no fused multiply-add for double-float)
    if (TPS == 1 || part == 0 || (TPS == 2 && part == 0)) {
      hop_dir<PREC, NREAL, 0, +1>(acc, inr, g.h, nb[0], lf + 0 * slab, cb, tfwd);
      hop_dir<PREC, NREAL, 0, -1>(acc, inr, g.h, nb[4], lo + 0 * slab, nb[4], tbwd);
    }
    if (TPS == 1 || (TPS == 2 && part == 0) || (TPS == 4 && part == 1)) {
      hop_dir<PREC, NREAL, 1, +1>(acc, inr, g.h, nb[1], lf + 1 * slab, cb, false);
      hop_dir<PREC, NREAL, 1, -1>(acc, inr, g.h, nb[5], lo + 1 * slab, nb[5], false);
    }
    if (TPS == 1 || (TPS == 2 && part == 1) || (TPS == 4 && part == 2)) {
      hop_dir<PREC, NREAL, 2, +1>(acc, inr, g.h, nb[2], lf + 2 * slab, cb, false);
      hop_dir<PREC, NREAL, 2, -1>(acc, inr, g.h, nb[6], lo + 2 * slab, nb[6], false);
    }
    if (TPS == 1 || (TPS == 2 && part == 1) || (TPS == 4 && part == 3)) {
      hop_dir<PREC, NREAL, 3, +1>(acc, inr, g.h, nb[3], lf + 3 * slab, cb, false);
      hop_dir<PREC, NREAL, 3, -1>(acc, inr, g.h, nb[7], lo + 3 * slab, nb[7], false);
    }
  } else {
    // direction pairs; the first pair of a part writes the accumulator
    if (TPS == 1 || part == 0)
      hop_pair<PREC, NREAL, 0, true>(acc, inr, g.h, nb[0], lf + 0 * slab, cb, tfwd, nb[4], lo + 0 * slab, nb[4], tbwd);
    if (TPS == 1 || (TPS == 2 && part == 0))
      hop_pair<PREC, NREAL, 1, false>(acc, inr, g.h, nb[1], lf + 1 * slab, cb, false, nb[5], lo + 1 * slab, nb[5], false);
    if (TPS == 4 && part == 1)
      hop_pair<PREC, NREAL, 1, true>(acc, inr, g.h, nb[1], lf + 1 * slab, cb, false, nb[5], lo + 1 * slab, nb[5], false);
    if (TPS == 1)
      hop_pair<PREC, NREAL, 2, false>(acc, inr, g.h, nb[2], lf + 2 * slab, cb, false, nb[6], lo + 2 * slab, nb[6], false);
    if ((TPS == 2 && part == 1) || (TPS == 4 && part == 2))
      hop_pair<PREC, NREAL, 2, true>(acc, inr, g.h, nb[2], lf + 2 * slab, cb, false, nb[6], lo + 2 * slab, nb[6], false);
    if (TPS == 1 || (TPS == 2 && part == 1))
      hop_pair<PREC, NREAL, 3, false>(acc, inr, g.h, nb[3], lf + 3 * slab, cb, false, nb[7], lo + 3 * slab, nb[7], false);
    if (TPS == 4 && part == 3)
      hop_pair<PREC, NREAL, 3, true>(acc, inr, g.h, nb[3], lf + 3 * slab, cb, false, nb[7], lo + 3 * slab, nb[7], false);
  }
}

// FP32 / FP16 storage with one thread per site: a register budget for 12 blocks of 64 threads
// per SM with 12-real links (80 per thread instead of 86-92).  The kernel is memory-latency
// bound and the extra warps win over a few spilled bytes (FP32/12: 32^3 x 64 118 -> 113 us,
// 16^3 x 32 18.9 -> 17.6 us per launch).  8- and 18-real links get 10 blocks (96 registers):
// at 80 their direction pairs spilled 84-156 bytes (FP32/8 on 32^3 x 64: 115 -> 107 us with
// 96, FP32/18: 157 -> 140 us).  FP64 and double-float keep their full budget (ALU bound).
// The software-pipelined form holds two hops' words (72 more registers for FP32/12): a budget
// for HOP_PIPE_BLOCKS blocks per SM.
#ifndef HOP_PIPE_BLOCKS
#define HOP_PIPE_BLOCKS 7
#endif
#ifndef HOP_BLOCKS_12
#define HOP_BLOCKS_12 12
#endif
#ifndef HOP_BLOCKS_OTHER
#define HOP_BLOCKS_OTHER 10
#endif
constexpr int hop_min_blocks(int prec, int nreal, int tps, bool pipe) {
  return pipe ? HOP_PIPE_BLOCKS
              : ((tps == 1 && (prec == TM_F32 || prec == TM_F16)) ? (nreal == 12 ? HOP_BLOCKS_12 : HOP_BLOCKS_OTHER) : 1);
}

// Which block of which right-hand side a block of the hopping kernel computes: the CUDA grid's
// (block x of gridDim.x, right-hand side y), read where used like the kernel's own indices ...
struct GridBlock {
  __device__ __forceinline__ int bid() const { return blockIdx.x; }
  __device__ __forceinline__ int nblocks() const { return gridDim.x; }
  __device__ __forceinline__ int rhs() const { return blockIdx.y; }
};
// ... or a block of a batched solver's work list (right-hand side 0 of one system's fields)
struct ListBlock {
  int b, n;
  __device__ __forceinline__ int bid() const { return b; }
  __device__ __forceinline__ int nblocks() const { return n; }
  __device__ __forceinline__ int rhs() const { return 0; }
};

// The body of the hopping kernels: output sites [bid SPB, (bid + 1) SPB) of right-hand side rhs
// (fields at in + rhs in_stride, ...), block bid of nblocks (from B).  alpha (MODE 2): r -= alpha o
// with alpha = alpha_sign * alpha_src[rhs].alpha, or alpha_sign without alpha_src; the norms of
// MODE >= 1 go to the reduction red of system rhs.  Shared by hop_kernel and the batched solver's
// kernel.  The field pointers are formed where they are used, as from a kernel's parameters, so
// that they hold no registers across the hops.
template <int PREC, int NREAL, bool HAS_Y, int MODE, int TPS, bool PIPE, class Blk, int SPB = hop_spb(TPS)>
__device__ __forceinline__ void hop_sites(const Geom g, const int out_parity, const char* __restrict__ links,
                                          const void* in, size_t in_stride, void* out, size_t out_stride,
                                          const void* y, size_t y_stride, const EpiCoef coef,
                                          const CGState* alpha_src, const double alpha_sign, const Reduce red,
                                          const Blk B) {
  typedef typename SpinorFmt<PREC>::real R;
  typedef SpinorFmt<PREC> F;
  constexpr int NT = SPB * TPS;            // threads per block (SPB sites per block)
  constexpr int WPP = (NT / 32) / TPS;     // warps per part
  constexpr int STRIDE = 25;               // 24 reals per site, padded against bank conflicts
  __shared__ double sh[NT / 32];
  __shared__ R part_acc[TPS > 1 ? TPS * SPB * STRIDE : 1];
  __shared__ float part_max[(TPS > 1 && F::has_norm) ? TPS * SPB : 1];
  const int warp = threadIdx.x >> 5;
  const int part = (TPS == 1) ? 0 : warp / WPP;
  const int sib = (TPS == 1) ? threadIdx.x : (warp % WPP) * 32 + (threadIdx.x & 31);
  const int rhs = B.rhs();
  const int cb = B.bid() * SPB + sib;
  const bool active = cb < g.h;
  cpx<R> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = mk<R>(R(0), R(0));
  if (active) {
    const SiteCoord c = site_of(g, cb, out_parity);
    int nb[8];
    neighbours(g, cb, c, nb);
    const char* inr = static_cast<const char*>(in) + (size_t)rhs * in_stride;
    const size_t slab = link_bytes(PREC, NREAL) * (size_t)g.h;
    const char* lf = links + (size_t)(out_parity * 4) * slab;        // U_mu(x), x of this parity
    const char* lo = links + (size_t)((1 - out_parity) * 4) * slab;  // U_mu(y), y of the other parity
    if constexpr (PIPE)
      hop_all_pipelined<PREC, NREAL>(acc, g, cb, c, nb, inr, lf, lo, slab);
    else
      hop_part<PREC, NREAL, TPS>(acc, g, cb, c, nb, inr, lf, lo, slab, part);
  }
  // this thread's share of the site's storage blocks
  const int kb = (TPS == 1) ? 0 : F::CPB * ((F::NBLK * part) / TPS);
  const int ke = (TPS == 1) ? 12 : F::CPB * ((F::NBLK * (part + 1)) / TPS);
  if (TPS > 1) {
    R* mine = part_acc + (part * SPB + sib) * STRIDE;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      mine[2 * k] = acc[k].re;
      mine[2 * k + 1] = acc[k].im;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 12; ++k)
      if (k >= kb && k < ke) {
        cpx<R> sum = mk<R>(part_acc[sib * STRIDE + 2 * k], part_acc[sib * STRIDE + 2 * k + 1]);
#pragma unroll
        for (int q = 1; q < TPS; ++q) {
          const R* o = part_acc + (q * SPB + sib) * STRIDE;
          sum = sum + mk<R>(o[2 * k], o[2 * k + 1]);
        }
        acc[k] = sum;
      }
  }
  typedef typename SiteSum<R>::type SR;
  SR nrm = SR(0);
  // epilogue: o_s = D_s (c acc_s + E_s y_s) on components [kb, ke), evaluated as
  // (D_s c) acc_s + (D_s E_s) y_s with the two coefficients formed once in FP64 (24 multiplies
  // per site fewer); MODE 3 needs t = c acc + E y itself and keeps the factored form
  constexpr bool F32A = sizeof(R) == 4;  // FP32 arithmetic: the host-folded FP32 coefficients
  const R cc = (R)coef.c;
  const cpx<R> Du = mk<R>((R)coef.d_up_re, (R)coef.d_up_im), Dl = mk<R>((R)coef.d_lo_re, (R)coef.d_lo_im);
  const cpx<R> DCu = F32A ? mk<R>((R)coef.f_dcu_re, (R)coef.f_dcu_im)
                          : mk<R>((R)(coef.d_up_re * coef.c), (R)(coef.d_up_im * coef.c));
  const cpx<R> DCl = F32A ? mk<R>((R)coef.f_dcl_re, (R)coef.f_dcl_im)
                          : mk<R>((R)(coef.d_lo_re * coef.c), (R)(coef.d_lo_im * coef.c));
  cpx<R> o[12];
  if (HAS_Y) {
    const cpx<R> Eu = mk<R>((R)coef.e_up_re, (R)coef.e_up_im), El = mk<R>((R)coef.e_lo_re, (R)coef.e_lo_im);
    const cpx<R> DEu = F32A ? mk<R>((R)coef.f_deu_re, (R)coef.f_deu_im)
                            : mk<R>((R)(coef.d_up_re * coef.e_up_re - coef.d_up_im * coef.e_up_im),
                                    (R)(coef.d_up_re * coef.e_up_im + coef.d_up_im * coef.e_up_re));
    const cpx<R> DEl = F32A ? mk<R>((R)coef.f_del_re, (R)coef.f_del_im)
                            : mk<R>((R)(coef.d_lo_re * coef.e_lo_re - coef.d_lo_im * coef.e_lo_im),
                                    (R)(coef.d_lo_re * coef.e_lo_im + coef.d_lo_im * coef.e_lo_re));
    cpx<R> yv[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) yv[k] = mk<R>(R(0), R(0));
    if (active) F::load_range(static_cast<const char*>(y) + (size_t)rhs * y_stride, g.h, cb, yv, kb, ke);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      if (MODE == 3) {
        const cpx<R> t = cc * acc[k] + ((k < 6) ? Eu : El) * yv[k];
        o[k] = ((k < 6) ? Du : Dl) * t;
        if (k >= kb && k < ke) {
          const cpx<R> M = (k < 6) ? mk<R>((R)coef.m_up_re, (R)coef.m_up_im) : mk<R>((R)coef.m_lo_re, (R)coef.m_lo_im);
          nrm += (SR)norm2(t - M * o[k]);
        }
      } else {
        o[k] = ((k < 6) ? DCu : DCl) * acc[k] + ((k < 6) ? DEu : DEl) * yv[k];
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = ((k < 6) ? DCu : DCl) * acc[k];
  }
  char* outr = static_cast<char*>(out) + (size_t)rhs * out_stride;
  if (MODE == 2) {
    if (active) {
      // (FP32 arithmetic: the sign, +-1, applied after the rounding, with the same result)
      const R al = F32A ? (alpha_src ? (R)alpha_sign * (R)alpha_src[rhs].alpha : (R)alpha_sign)
                        : (R)(alpha_src ? alpha_sign * alpha_src[rhs].alpha : alpha_sign);
      constexpr int PR = ResidPrec<PREC>::value;
      cpx<R> r[12];
      SpinorFmt<PR>::load_range(outr, g.h, cb, r, kb, ke);
#pragma unroll
      for (int k = 0; k < 12; ++k)
        if (k >= kb && k < ke) {
          r[k] = r[k] - al * o[k];
          nrm += (SR)norm2(r[k]);
        }
      SpinorFmt<PR>::store_range(outr, g.h, cb, r, kb, ke, 0.f, false);
    }
  } else {
    float m = 0.f;
    if (F::has_norm) {  // the site's FP16 norm needs all of its components
#pragma unroll
      for (int k = 0; k < 12; ++k)
        if (k >= kb && k < ke) m = fmaxf(m, fmaxf(fabsf((float)o[k].re), fabsf((float)o[k].im)));
      if (TPS > 1) {
        part_max[part * SPB + sib] = m;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TPS; ++q) m = fmaxf(m, part_max[q * SPB + sib]);
      }
    }
    if (active) {
      if (MODE == 1) {
#pragma unroll
        for (int k = 0; k < 12; ++k)
          if (k >= kb && k < ke) nrm += (SR)norm2(o[k]);
      }
      F::store_range(outr, g.h, cb, o, kb, ke, m, part == 0);
    }
  }
  if (MODE >= 1) {
    const double bs = block_sum<NT>(nrm, sh);  // SR: FP32 for FP32 arithmetic
    grid_reduce<NT>(red, rhs, B.nblocks(), B.bid(), bs, sh);
  }
}

template <int PREC, int NREAL, bool HAS_Y, int MODE, int TPS, bool PIPE>
__global__ void __launch_bounds__(hop_spb(TPS) * TPS, hop_min_blocks(PREC, NREAL, TPS, PIPE)) hop_kernel(const Geom g, const int out_parity,
                                                     const char* __restrict__ links, const void* in,
                                                     size_t in_stride, void* out, size_t out_stride,
                                                     const void* y, size_t y_stride, const EpiCoef coef,
                                                     const CGState* alpha_src, const double alpha_sign,
                                                     const Reduce red, const int* skip) {
  pdl_wait();
  pdl_allow();
  if (skip != nullptr && *skip != 0) return;
  hop_sites<PREC, NREAL, HAS_Y, MODE, TPS, PIPE>(g, out_parity, links, in, in_stride, out, out_stride, y, y_stride, coef,
                                                 alpha_src, alpha_sign, red, GridBlock{});
}

// the two-sites-per-thread kernel (tm_dslash_pair.cuh), instantiated in its own units
tm_status hop_pair_launch_f32(tm_lattice lat, const HopArgs& a, cudaStream_t s);
tm_status hop_pair_launch_f16(tm_lattice lat, const HopArgs& a, cudaStream_t s);

template <int PREC, int NREAL, int TPS, bool PIPE>
tm_status hop_launch_tps(tm_lattice lat, const HopArgs& a, cudaStream_t s) {
  const Geom& g = lat->geom;
  constexpr int SPB = hop_spb(TPS), NT = SPB * TPS;
  dim3 grid((g.h + SPB - 1) / SPB, a.nrhs);
  const char* links = static_cast<const char*>(lat->links[PREC][link_index(NREAL)]);
  const bool has_y = a.y != nullptr;
#define TM_HOP_ARGS                                                                                      \
  g, a.out_parity, links, a.in, a.in_stride, a.out, a.out_stride, a.y, a.y_stride, a.coef, a.alpha_src, \
      a.alpha_sign, a.red, a.skip
  if (!has_y && a.mode == 0)
    launch_pdl(hop_kernel<PREC, NREAL, false, 0, TPS, PIPE>, grid, dim3(NT), s, TM_HOP_ARGS);
  else if (!has_y && a.mode == 1)
    launch_pdl(hop_kernel<PREC, NREAL, false, 1, TPS, PIPE>, grid, dim3(NT), s, TM_HOP_ARGS);
  else if (has_y && a.mode == 0)
    launch_pdl(hop_kernel<PREC, NREAL, true, 0, TPS, PIPE>, grid, dim3(NT), s, TM_HOP_ARGS);
  else if (has_y && a.mode == 1)
    launch_pdl(hop_kernel<PREC, NREAL, true, 1, TPS, PIPE>, grid, dim3(NT), s, TM_HOP_ARGS);
  else if (has_y && a.mode == 2)
    launch_pdl(hop_kernel<PREC, NREAL, true, 2, TPS, PIPE>, grid, dim3(NT), s, TM_HOP_ARGS);
  else if (has_y && a.mode == 3 && PREC == TM_F64) {
    if constexpr (PREC == TM_F64) launch_pdl(hop_kernel<PREC, NREAL, true, 3, TPS, PIPE>, grid, dim3(NT), s, TM_HOP_ARGS);
  } else
    return set_error(TM_ERR_ARG, "hopping: unsupported epilogue combination");
#undef TM_HOP_ARGS
  count_launch();
  return cuda_check(cudaGetLastError(), "hopping kernel launch");
}

template <int PREC, int NREAL>
tm_status hop_launch_t(tm_lattice lat, const HopArgs& a, cudaStream_t s) {
  switch (lat->hop_tps[PREC][link_index(NREAL)]) {
    case 2:
      return hop_launch_tps<PREC, NREAL, 2, false>(lat, a, s);
    case 4:
      return hop_launch_tps<PREC, NREAL, 4, false>(lat, a, s);
    case TM_HOP_PIPELINED:
      if constexpr (PREC == TM_F32 || PREC == TM_F16) return hop_launch_tps<PREC, NREAL, 1, true>(lat, a, s);
      return hop_launch_tps<PREC, NREAL, 1, false>(lat, a, s);
    case TM_HOP_PAIRED:
      if constexpr (PREC == TM_F32) return hop_pair_launch_f32(lat, a, s);
      if constexpr (PREC == TM_F16) return hop_pair_launch_f16(lat, a, s);
      return hop_launch_tps<PREC, NREAL, 1, false>(lat, a, s);
    default:
      return hop_launch_tps<PREC, NREAL, 1, false>(lat, a, s);
  }
}

template <int PREC>
tm_status hop_launch_prec(tm_lattice lat, const HopArgs& a, cudaStream_t s) {
  switch (a.nreal) {
    case 18:
      return hop_launch_t<PREC, 18>(lat, a, s);
    case 12:
      return hop_launch_t<PREC, 12>(lat, a, s);
    case 8:
      return hop_launch_t<PREC, 8>(lat, a, s);
    default:
      return set_error(TM_ERR_ARG, "hopping: link format %d not one of 18, 12, 8", a.nreal);
  }
}

tm_status hop_launch_f64(tm_lattice lat, const HopArgs& a, cudaStream_t s);
tm_status hop_launch_df64(tm_lattice lat, const HopArgs& a, cudaStream_t s);
tm_status hop_launch_f32(tm_lattice lat, const HopArgs& a, cudaStream_t s);
tm_status hop_launch_f16(tm_lattice lat, const HopArgs& a, cudaStream_t s);

}  // namespace tmq
