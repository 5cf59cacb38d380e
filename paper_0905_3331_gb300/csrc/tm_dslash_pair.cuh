// tm_dslash_pair.cuh -- the hopping kernel with two output sites per thread and packed FP32
// arithmetic (FP32 and FP16 storage).
//
// The arithmetic is that of the one-site kernel -- the spin projection before the SU(3)
// multiply (Sec. 4.1), direction pairs whose forward and backward hops share the FMA chains,
// links reconstructed from 18, 12 or 8 stored reals, the epilogue out = D (c H in + E y) and the
// fused reductions -- carried out on pairs (site A, site B) of the two-lane type f2, so one
// packed instruction serves both sites.  The units tm_dslash_pair_f32.cu and
// tm_dslash_pair_f16.cu instantiate it.  With FP16 storage the one-site kernel is bound by
// instruction issue, not by memory (ncu on 32^3 x 64: 69-73% issue-active, 31-48% of DRAM
// bandwidth, ~1900 instructions per site with 12-real links); the pairs halve the issue slots of
// the FP32 work.
// Thread t of block b computes sites A = 128 b + t and B = A + 64: each warp's loads of either
// site are 32 consecutive sites of a storage block, one coalesced request as before.
#pragma once

#include "tm_dslash.cuh"

namespace tmq {

constexpr int PAIR_NT = 64;  // threads per block; 2 * PAIR_NT output sites per block
#ifndef HOP_PAIR_BLOCKS
#define HOP_PAIR_BLOCKS 5
#endif

// Spinor of sites ia (lane x) and ib (lane y), unscaled, with their FP16 norms (1 for FP32).
template <int PREC>
__device__ __forceinline__ void load_spinor_pair(const void* in, int h, int ia, int ib, cpx<f2> p[12], f2& scale) {
  cpx<float> a[12], b[12];
  float sa, sb;
  SpinorFmt<PREC>::load_unscaled(in, h, ia, a, sa);
  SpinorFmt<PREC>::load_unscaled(in, h, ib, b, sb);
#pragma unroll
  for (int k = 0; k < 12; ++k) p[k] = mk<f2>(f2(a[k].re, b[k].re), f2(a[k].im, b[k].im));
  scale = f2(sa, sb);
}

// Links (slab, ia) and (slab, ib) reconstructed as a pair of matrices.
template <int PREC, int NREAL>
__device__ __forceinline__ void load_link_pair(const char* slab, int h, int ia, int ib, Mat3<f2>& U) {
  typedef typename LinkStore<PREC>::type S;
  constexpr int BYTES = NREAL * LinkStore<PREC>::size;
  const RawWords<BYTES> ra = load_raw<BYTES>(slab, h, ia);
  const RawWords<BYTES> rb = load_raw<BYTES>(slab, h, ib);
  LinkRecon<f2, S, NREAL>::from_reals(
      [&](int k) { return f2((float)RawGet<S, BYTES>::get(ra, k), (float)RawGet<S, BYTES>::get(rb, k)); }, U);
}

// Both hops of direction MU for the pair: u+- = U(+-) (1 +- gamma_MU) in(x +- MU^) projected,
// scaled by each neighbour's norm and boundary sign (ff, fb), combined into the accumulator as in
// pair_fwd / pair_bwd.
template <int PREC, int NREAL, int MU, bool FIRST>
__device__ __forceinline__ void hop_pair2(cpx<f2> acc[12], const void* in, int h, int nfa, int nfb, const char* slabf,
                                          int lfa, int lfb, f2 sgnf, int nba, int nbb, const char* slabb, int lba,
                                          int lbb, f2 sgnb) {
  cpx<f2> p[12];
  f2 scale;
  cpx<f2> h0[3], h1[3], u0[3], u1[3];
  {
    Mat3<f2> U;
    load_link_pair<PREC, NREAL>(slabf, h, lfa, lfb, U);
    load_spinor_pair<PREC>(in, h, nfa, nfb, p, scale);
    project<f2, MU, +1>(p, h0, h1);
    const f2 f = SpinorFmt<PREC>::has_norm ? scale * sgnf : sgnf;
    if (SpinorFmt<PREC>::has_norm || MU == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        h0[c] = f * h0[c];
        h1[c] = f * h1[c];
      }
    }
    su3_mul2_fma(U, h0, h1, u0, u1);
  }
  Mat3<f2> U;
  load_link_pair<PREC, NREAL>(slabb, h, lba, lbb, U);
  load_spinor_pair<PREC>(in, h, nba, nbb, p, scale);
  project<f2, MU, -1>(p, h0, h1);
  const f2 f = SpinorFmt<PREC>::has_norm ? scale * sgnb : sgnb;
  if (SpinorFmt<PREC>::has_norm || MU == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h0[c] = f * h0[c];
      h1[c] = f * h1[c];
    }
  }
  cpx<f2> s0[3], s1[3];
  su3_adj_mul2_add(U, h0, h1, u0, u1, s0, s1);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const cpx<f2> d0 = mk<f2>(fmadd(f2(2.f), u0[a].re, -s0[a].re), fmadd(f2(2.f), u0[a].im, -s0[a].im));
    const cpx<f2> d1 = mk<f2>(fmadd(f2(2.f), u1[a].re, -s1[a].re), fmadd(f2(2.f), u1[a].im, -s1[a].im));
    cpx<f2> l2, l3;  // P_mu d
    if (MU == 0) {
      l2 = mk<f2>(-d0.re, -d0.im);
      l3 = mk<f2>(-d1.re, -d1.im);
    } else if (MU == 1) {
      l2 = times_i(d1);
      l3 = times_i(d0);
    } else if (MU == 2) {
      l2 = d1;
      l3 = mk<f2>(-d0.re, -d0.im);
    } else {
      l2 = times_i(d0);
      l3 = mk<f2>(d1.im, -d1.re);
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

// Modes and arguments as hop_kernel (MODE 0, 1, 2; MODE 3 is FP64 only).
template <int PREC, int NREAL, bool HAS_Y, int MODE>
__global__ void __launch_bounds__(PAIR_NT, HOP_PAIR_BLOCKS)
    hop_pair_kernel(const Geom g, const int out_parity, const char* __restrict__ links, const void* in,
                    size_t in_stride, void* out, size_t out_stride, const void* y, size_t y_stride, const EpiCoef coef,
                    const CGState* alpha_src, const double alpha_sign, const Reduce red, const int* skip) {
  typedef SpinorFmt<PREC> F;
  __shared__ double sh[PAIR_NT / 32];
  pdl_wait();
  pdl_allow();
  if (skip != nullptr && *skip != 0) return;
  const int rhs = blockIdx.y;
  const int cba = blockIdx.x * (2 * PAIR_NT) + threadIdx.x;
  const bool act_a = cba < g.h;
  const bool act_b = cba + PAIR_NT < g.h;
  const int cbb = act_b ? cba + PAIR_NT : cba;  // an idle lane B repeats site A (loads stay in bounds)
  cpx<f2> acc[12];
  if (act_a) {
    const SiteCoord ca = site_of(g, cba, out_parity), cb = site_of(g, cbb, out_parity);
    int na[8], nb[8];
    neighbours(g, cba, ca, na);
    neighbours(g, cbb, cb, nb);
    const char* inr = static_cast<const char*>(in) + (size_t)rhs * in_stride;
    const size_t slab = link_bytes(PREC, NREAL) * (size_t)g.h;
    const char* lf = links + (size_t)(out_parity * 4) * slab;        // U_mu(x), x of this parity
    const char* lo = links + (size_t)((1 - out_parity) * 4) * slab;  // U_mu(y), y of the other parity
    // antiperiodic time direction: the hop across t = T-1 <-> 0 carries -1 (Sec. 2.4)
    const f2 tf(ca.t == g.T - 1 ? -1.f : 1.f, cb.t == g.T - 1 ? -1.f : 1.f);
    const f2 tb(ca.t == 0 ? -1.f : 1.f, cb.t == 0 ? -1.f : 1.f);
    const f2 one(1.f);
    hop_pair2<PREC, NREAL, 0, true>(acc, inr, g.h, na[0], nb[0], lf + 0 * slab, cba, cbb, tf, na[4], nb[4],
                                    lo + 0 * slab, na[4], nb[4], tb);
    hop_pair2<PREC, NREAL, 1, false>(acc, inr, g.h, na[1], nb[1], lf + 1 * slab, cba, cbb, one, na[5], nb[5],
                                     lo + 1 * slab, na[5], nb[5], one);
    hop_pair2<PREC, NREAL, 2, false>(acc, inr, g.h, na[2], nb[2], lf + 2 * slab, cba, cbb, one, na[6], nb[6],
                                     lo + 2 * slab, na[6], nb[6], one);
    hop_pair2<PREC, NREAL, 3, false>(acc, inr, g.h, na[3], nb[3], lf + 3 * slab, cba, cbb, one, na[7], nb[7],
                                     lo + 3 * slab, na[7], nb[7], one);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = mk<f2>(f2(0.f), f2(0.f));
  }
  // epilogue o_s = D_s (c acc_s + E_s y_s) = (D_s c) acc_s + (D_s E_s) y_s, per chirality
  const cpx<f2> DCu = mk<f2>(f2(coef.f_dcu_re), f2(coef.f_dcu_im));  // folded on the host (epi_finish)
  const cpx<f2> DCl = mk<f2>(f2(coef.f_dcl_re), f2(coef.f_dcl_im));
  cpx<f2> o[12];
  if (HAS_Y) {
    const cpx<f2> DEu = mk<f2>(f2(coef.f_deu_re), f2(coef.f_deu_im));
    const cpx<f2> DEl = mk<f2>(f2(coef.f_del_re), f2(coef.f_del_im));
    cpx<float> ya[12], yb[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) ya[k] = yb[k] = mk<float>(0.f, 0.f);
    if (act_a) {
      const char* yr = static_cast<const char*>(y) + (size_t)rhs * y_stride;
      F::load_range(yr, g.h, cba, ya, 0, 12);
      F::load_range(yr, g.h, cbb, yb, 0, 12);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const cpx<f2> yv = mk<f2>(f2(ya[k].re, yb[k].re), f2(ya[k].im, yb[k].im));
      o[k] = (k < 6 ? DCu : DCl) * acc[k] + (k < 6 ? DEu : DEl) * yv;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = (k < 6 ? DCu : DCl) * acc[k];
  }
  float nrm = 0.f;  // this thread's own sites, in FP32 (reading of Sec. 4.1's precisions, FP64 across threads)
  char* outr = static_cast<char*>(out) + (size_t)rhs * out_stride;
  cpx<float> oa[12], ob[12];
  if (MODE == 2) {
    if (act_a) {
      const f2 al(alpha_src ? (float)alpha_sign * (float)alpha_src[rhs].alpha : (float)alpha_sign);
      constexpr int PR = ResidPrec<PREC>::value;
      cpx<float> ra[12], rb[12];
      SpinorFmt<PR>::load_range(outr, g.h, cba, ra, 0, 12);
      SpinorFmt<PR>::load_range(outr, g.h, cbb, rb, 0, 12);
      f2 n2(0.f);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        cpx<f2> r = mk<f2>(f2(ra[k].re, rb[k].re), f2(ra[k].im, rb[k].im));
        r = mk<f2>(fmadd(-al, o[k].re, r.re), fmadd(-al, o[k].im, r.im));
        n2 = n2 + norm2(r);
        oa[k] = mk<float>(r.re.v.x, r.im.v.x);
        ob[k] = mk<float>(r.re.v.y, r.im.v.y);
      }
      nrm = n2.v.x + (act_b ? n2.v.y : 0.f);
      SpinorFmt<PR>::store_range(outr, g.h, cba, oa, 0, 12, 0.f, false);
      if (act_b) SpinorFmt<PR>::store_range(outr, g.h, cbb, ob, 0, 12, 0.f, false);
    }
  } else if (act_a) {
    float ma = 0.f, mb = 0.f;
    f2 n2(0.f);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      oa[k] = mk<float>(o[k].re.v.x, o[k].im.v.x);
      ob[k] = mk<float>(o[k].re.v.y, o[k].im.v.y);
      if (F::has_norm) {
        ma = fmaxf(ma, fmaxf(fabsf(oa[k].re), fabsf(oa[k].im)));
        mb = fmaxf(mb, fmaxf(fabsf(ob[k].re), fabsf(ob[k].im)));
      }
      if (MODE == 1) n2 = n2 + norm2(o[k]);
    }
    if (MODE == 1) nrm = n2.v.x + (act_b ? n2.v.y : 0.f);
    F::store_range(outr, g.h, cba, oa, 0, 12, ma, true);
    if (act_b) F::store_range(outr, g.h, cbb, ob, 0, 12, mb, true);
  }
  if (MODE >= 1) {
    const double bs = block_sum<PAIR_NT>(nrm, sh);
    grid_reduce<PAIR_NT>(red, rhs, gridDim.x, blockIdx.x, bs, sh);
  }
}

template <int PREC, int NREAL>
tm_status hop_pair_launch_t(tm_lattice lat, const HopArgs& a, cudaStream_t s) {
  const Geom& g = lat->geom;
  dim3 grid((g.h + 2 * PAIR_NT - 1) / (2 * PAIR_NT), a.nrhs);
  const char* links = static_cast<const char*>(lat->links[PREC][link_index(NREAL)]);
  const bool has_y = a.y != nullptr;
#define TM_PAIR_ARGS                                                                                     \
  g, a.out_parity, links, a.in, a.in_stride, a.out, a.out_stride, a.y, a.y_stride, a.coef, a.alpha_src, \
      a.alpha_sign, a.red, a.skip
  if (!has_y && a.mode == 0)
    launch_pdl(hop_pair_kernel<PREC, NREAL, false, 0>, grid, dim3(PAIR_NT), s, TM_PAIR_ARGS);
  else if (!has_y && a.mode == 1)
    launch_pdl(hop_pair_kernel<PREC, NREAL, false, 1>, grid, dim3(PAIR_NT), s, TM_PAIR_ARGS);
  else if (has_y && a.mode == 0)
    launch_pdl(hop_pair_kernel<PREC, NREAL, true, 0>, grid, dim3(PAIR_NT), s, TM_PAIR_ARGS);
  else if (has_y && a.mode == 1)
    launch_pdl(hop_pair_kernel<PREC, NREAL, true, 1>, grid, dim3(PAIR_NT), s, TM_PAIR_ARGS);
  else if (has_y && a.mode == 2)
    launch_pdl(hop_pair_kernel<PREC, NREAL, true, 2>, grid, dim3(PAIR_NT), s, TM_PAIR_ARGS);
  else
    return set_error(TM_ERR_ARG, "hopping: unsupported epilogue combination");
#undef TM_PAIR_ARGS
  count_launch();
  return cuda_check(cudaGetLastError(), "hopping kernel launch");
}

template <int PREC>
tm_status hop_pair_launch_prec(tm_lattice lat, const HopArgs& a, cudaStream_t s) {
  switch (a.nreal) {
    case 18:
      return hop_pair_launch_t<PREC, 18>(lat, a, s);
    case 12:
      return hop_pair_launch_t<PREC, 12>(lat, a, s);
    case 8:
      return hop_pair_launch_t<PREC, 8>(lat, a, s);
    default:
      return set_error(TM_ERR_ARG, "hopping: link format %d not one of 18, 12, 8", a.nreal);
  }
}

}  // namespace tmq
