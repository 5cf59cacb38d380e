// tm_dslash_doublet.cu -- the hopping term of the doublet operator (eq. Dh) for both flavours
// at once, with the flavour-mixing site term in the epilogue.
//
// The hopping sum acts on each flavour alike (eq. eo0), so one thread takes both flavours of an
// output site: per hop the link is loaded and reconstructed once and multiplies the projected
// neighbour spinors of the two flavours (projection, adjoint for the backward hop and the
// antiperiodic sign exactly as in the one-flavour kernel).  The epilogue forms
//   out_f = [gamma5 tau1] ( sum_g P_fg y_g + Q_fg (H in)_g )
// per chirality, which covers D^-1 H, gamma5 tau1 (D y - kappa^2 H in) of the Schur operator and
// D y - kappa H in of the full operator, with the fused FP64 CG reductions.
#include <cstdlib>

#include "tm_doublet.cuh"
#include "tm_dslash.cuh"

namespace tmq {

// Both hops of direction mu for both flavours: the one-flavour direction-pair arithmetic
// (tm_dslash.cuh) per flavour, with the pair's two links loaded once for the two flavours.
template <int PREC, int NREAL, int MU, bool FIRST>
__device__ __forceinline__ void dhop_pair(cpx<typename SpinorFmt<PREC>::real> acc[2][12], const char* in,
                                          size_t stride, int h, int nbf, const char* slabf, int lif, bool negf,
                                          int nbb, const char* slabb, int lib, bool negb) {
  typedef typename SpinorFmt<PREC>::real R;
  constexpr int BYTES = NREAL * LinkStore<PREC>::size;
  const RawWords<BYTES> rf = load_raw<BYTES>(slabf, h, lif);
  const RawWords<BYTES> rb = load_raw<BYTES>(slabb, h, lib);
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    cpx<R> p[12];
    R scale;
    SpinorFmt<PREC>::load_unscaled(in + f * stride, h, nbf, p, scale);
    cpx<R> u0[3], u1[3];
    pair_fwd<PREC, NREAL, MU>(u0, u1, rf, p, scale, negf);
    SpinorFmt<PREC>::load_unscaled(in + f * stride, h, nbb, p, scale);
    pair_bwd<PREC, NREAL, MU, FIRST>(acc[f], u0, u1, rb, p, scale, negb);
  }
}

template <int PREC, int NREAL, bool HAS_Y, int MODE>
__global__ void __launch_bounds__(HOP_NT) dhop_kernel(const Geom g, const int out_parity,
                                                      const char* __restrict__ links, const char* in,
                                                      size_t stride, char* out, size_t out_stride, const char* y,
                                                      const DCoef co, const CGState* alpha_src, const Reduce red,
                                                      const int* skip) {
  typedef typename SpinorFmt<PREC>::real R;
  __shared__ double sh[HOP_NT / 32];
  if (skip != nullptr && *skip != 0) return;
  const int cb = blockIdx.x * HOP_NT + threadIdx.x;
  const bool active = cb < g.h;
  typedef typename SiteSum<R>::type SR;
  SR nrm = SR(0);
  if (active) {
    cpx<R> acc[2][12];
#pragma unroll
    for (int f = 0; f < 2; ++f)
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[f][k] = mk<R>(R(0), R(0));
    const SiteCoord c = site_of(g, cb, out_parity);
    int nb[8];
    neighbours(g, cb, c, nb);
    const size_t slab = link_bytes(PREC, NREAL) * (size_t)g.h;
    const char* lf = links + (size_t)(out_parity * 4) * slab;
    const char* lo = links + (size_t)((1 - out_parity) * 4) * slab;
    const bool tfwd = (c.t == g.T - 1), tbwd = (c.t == 0);
    dhop_pair<PREC, NREAL, 0, true>(acc, in, stride, g.h, nb[0], lf + 0 * slab, cb, tfwd, nb[4], lo + 0 * slab, nb[4], tbwd);
    dhop_pair<PREC, NREAL, 1, false>(acc, in, stride, g.h, nb[1], lf + 1 * slab, cb, false, nb[5], lo + 1 * slab, nb[5], false);
    dhop_pair<PREC, NREAL, 2, false>(acc, in, stride, g.h, nb[2], lf + 2 * slab, cb, false, nb[6], lo + 2 * slab, nb[6], false);
    dhop_pair<PREC, NREAL, 3, false>(acc, in, stride, g.h, nb[3], lf + 3 * slab, cb, false, nb[7], lo + 3 * slab, nb[7], false);
    // epilogue, chirality by chirality
    cpx<R> o[2][12];
    if (HAS_Y) {
      cpx<R> y0[12], y1[12];
      SpinorFmt<PREC>::load(y, g.h, cb, y0);
      SpinorFmt<PREC>::load(y + stride, g.h, cb, y1);
#pragma unroll
      for (int f = 0; f < 2; ++f)
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const int ch = k < 6 ? 0 : 1;
          o[f][k] = dco<R>(co.P[ch][f][0], co.fP[ch][f][0]) * y0[k] +
                    dco<R>(co.P[ch][f][1], co.fP[ch][f][1]) * y1[k] +
                    dco<R>(co.Q[ch][f][0], co.fQ[ch][f][0]) * acc[0][k] +
                    dco<R>(co.Q[ch][f][1], co.fQ[ch][f][1]) * acc[1][k];
        }
    } else {
#pragma unroll
      for (int f = 0; f < 2; ++f)
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const int ch = k < 6 ? 0 : 1;
          o[f][k] = dco<R>(co.Q[ch][f][0], co.fQ[ch][f][0]) * acc[0][k] +
                    dco<R>(co.Q[ch][f][1], co.fQ[ch][f][1]) * acc[1][k];
        }
    }
    if (co.swap) {  // gamma5 tau1: swap the flavours, negate the lower spins
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const cpx<R> t = o[0][k];
        o[0][k] = k < 6 ? o[1][k] : mk<R>(-o[1][k].re, -o[1][k].im);
        o[1][k] = k < 6 ? t : mk<R>(-t.re, -t.im);
      }
    }
    if (MODE == 2) {
      constexpr int PR = ResidPrec<PREC>::value;
      typedef typename SpinorFmt<PR>::real RR;
      const RR al = (RR)(alpha_src ? alpha_src->alpha : 1.0);
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        cpx<RR> r[12];
        SpinorFmt<PR>::load(out + f * out_stride, g.h, cb, r);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          r[k] = r[k] - al * mk<RR>((RR)o[f][k].re, (RR)o[f][k].im);
          nrm += (SR)norm2(r[k]);
        }
        SpinorFmt<PR>::store(out + f * out_stride, g.h, cb, r);
      }
    } else {
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        SpinorFmt<PREC>::store(out + f * out_stride, g.h, cb, o[f]);
        if (MODE == 1)
#pragma unroll
          for (int k = 0; k < 12; ++k) nrm += (SR)norm2(o[f][k]);
      }
    }
  }
  if (MODE >= 1) {
    const double bs = block_sum<HOP_NT>(nrm, sh);
    grid_reduce<HOP_NT>(red, 0, gridDim.x, blockIdx.x, bs, sh);
  }
}

// The same operator with two threads per output site, one per flavour (adjacent lanes).  Both
// lanes of a pair load the same link (one memory transaction serves the pair), each applies it
// to its own flavour, and the epilogue takes the partner flavour's sums and site-local input
// through warp shuffles.  Half the registers of the one-thread form and twice the threads.
template <int PREC, int NREAL, bool HAS_Y, int MODE>
__global__ void __launch_bounds__(HOP_NT) dhop2_kernel(const Geom g, const int out_parity,
                                                       const char* __restrict__ links, const char* in,
                                                       size_t stride, char* out, size_t out_stride, const char* y,
                                                       const DCoef co, const CGState* alpha_src, const Reduce red,
                                                       const int* skip) {
  typedef typename SpinorFmt<PREC>::real R;
  __shared__ double sh[HOP_NT / 32];
  if (skip != nullptr && *skip != 0) return;
  const int f = threadIdx.x & 1;
  const int cb = blockIdx.x * (HOP_NT / 2) + (threadIdx.x >> 1);
  const bool active = cb < g.h;
  const char* inf = in + f * stride;
  cpx<R> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = mk<R>(R(0), R(0));
  if (active) {
    const SiteCoord c = site_of(g, cb, out_parity);
    int nb[8];
    neighbours(g, cb, c, nb);
    const size_t slab = link_bytes(PREC, NREAL) * (size_t)g.h;
    const char* lf = links + (size_t)(out_parity * 4) * slab;
    const char* lo = links + (size_t)((1 - out_parity) * 4) * slab;
    const bool tfwd = (c.t == g.T - 1), tbwd = (c.t == 0);
    // the one-flavour direction-pair arithmetic (tm_dslash.cuh) on this lane's flavour
    hop_pair<PREC, NREAL, 0, true>(acc, inf, g.h, nb[0], lf + 0 * slab, cb, tfwd, nb[4], lo + 0 * slab, nb[4], tbwd);
    hop_pair<PREC, NREAL, 1, false>(acc, inf, g.h, nb[1], lf + 1 * slab, cb, false, nb[5], lo + 1 * slab, nb[5], false);
    hop_pair<PREC, NREAL, 2, false>(acc, inf, g.h, nb[2], lf + 2 * slab, cb, false, nb[6], lo + 2 * slab, nb[6], false);
    hop_pair<PREC, NREAL, 3, false>(acc, inf, g.h, nb[3], lf + 3 * slab, cb, false, nb[7], lo + 3 * slab, nb[7], false);
  }
  // epilogue, component by component: the partner lane's sum (and site-local input) of the same
  // component comes through a shuffle (every lane takes part), the result overwrites acc[k].
  // This lane writes flavour f; with the gamma5 tau1 swap its value is gamma5 (row 1 - f).
  cpx<R> yv[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) yv[k] = mk<R>(R(0), R(0));
  if (HAS_Y && active) SpinorFmt<PREC>::load(y + f * stride, g.h, cb, yv);
  const int row = co.swap ? 1 - f : f;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int ch = k < 6 ? 0 : 1;
    const cpx<R> ap = mk<R>(__shfl_xor_sync(0xffffffffu, acc[k].re, 1), __shfl_xor_sync(0xffffffffu, acc[k].im, 1));
    cpx<R> v = dco<R>(co.Q[ch][row][f], co.fQ[ch][row][f]) * acc[k] +
               dco<R>(co.Q[ch][row][1 - f], co.fQ[ch][row][1 - f]) * ap;
    if (HAS_Y) {
      const cpx<R> yp = mk<R>(__shfl_xor_sync(0xffffffffu, yv[k].re, 1), __shfl_xor_sync(0xffffffffu, yv[k].im, 1));
      v = v + dco<R>(co.P[ch][row][f], co.fP[ch][row][f]) * yv[k] +
          dco<R>(co.P[ch][row][1 - f], co.fP[ch][row][1 - f]) * yp;
    }
    acc[k] = (co.swap && k >= 6) ? mk<R>(-v.re, -v.im) : v;
  }
  typedef typename SiteSum<R>::type SR;
  SR nrm = SR(0);
  if (active) {
    const cpx<R>* o = acc;
    char* outf = out + f * out_stride;
    if (MODE == 2) {
      constexpr int PR = ResidPrec<PREC>::value;
      typedef typename SpinorFmt<PR>::real RR;
      const RR al = (RR)(alpha_src ? alpha_src->alpha : 1.0);
      cpx<RR> r[12];
      SpinorFmt<PR>::load(outf, g.h, cb, r);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        r[k] = r[k] - al * mk<RR>((RR)o[k].re, (RR)o[k].im);
        nrm += (SR)norm2(r[k]);
      }
      SpinorFmt<PR>::store(outf, g.h, cb, r);
    } else {
      SpinorFmt<PREC>::store(outf, g.h, cb, o);
      if (MODE == 1)
#pragma unroll
        for (int k = 0; k < 12; ++k) nrm += (SR)norm2(o[k]);
    }
  }
  if (MODE >= 1) {
    const double bs = block_sum<HOP_NT>(nrm, sh);
    grid_reduce<HOP_NT>(red, 0, gridDim.x, blockIdx.x, bs, sh);
  }
}

static int dhop_threads_per_site() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("TM_DHOP_TPS");
    v = (e && *e == '1') ? 1 : 2;
  }
  return v;
}

template <int PREC, int NREAL>
static tm_status dhop_launch_t(tm_lattice lat, const DHopArgs& a, cudaStream_t s) {
  const Geom& g = lat->geom;
  const char* links = static_cast<const char*>(lat->links[PREC][link_index(NREAL)]);
  const char* in = static_cast<const char*>(a.in);
  const char* y = static_cast<const char*>(a.y);
  char* out = static_cast<char*>(a.out);
  const bool two = dhop_threads_per_site() == 2;
  const unsigned grid = (unsigned)((g.h + (two ? HOP_NT / 2 : HOP_NT) - 1) / (two ? HOP_NT / 2 : HOP_NT));
  const DCoef co = dcoef_finish(a.co);
#define TM_DHOP_ARGS g, a.out_parity, links, in, a.stride, out, a.out_stride, y, co, a.alpha_src, a.red, a.skip
#define TM_DHOP_LAUNCH(HY, MM)                                                       \
  do {                                                                               \
    if (two)                                                                         \
      dhop2_kernel<PREC, NREAL, HY, MM><<<grid, HOP_NT, 0, s>>>(TM_DHOP_ARGS);       \
    else                                                                             \
      dhop_kernel<PREC, NREAL, HY, MM><<<grid, HOP_NT, 0, s>>>(TM_DHOP_ARGS);        \
  } while (0)
  if (!a.y && a.mode == 0)
    TM_DHOP_LAUNCH(false, 0);
  else if (a.y && a.mode == 0)
    TM_DHOP_LAUNCH(true, 0);
  else if (a.y && a.mode == 1)
    TM_DHOP_LAUNCH(true, 1);
  else if (a.y && a.mode == 2)
    TM_DHOP_LAUNCH(true, 2);
  else
    return set_error(TM_ERR_ARG, "doublet hopping: unsupported epilogue combination");
#undef TM_DHOP_LAUNCH
#undef TM_DHOP_ARGS
  count_launch();
  return cuda_check(cudaGetLastError(), "doublet hopping kernel launch");
}

tm_status dhop_launch(tm_lattice lat, const DHopArgs& a, cudaStream_t s) {
  tm_status st = ensure_links(lat, a.prec, a.nreal, s);
  if (st != TM_OK) return st;
  if (a.prec == TM_F64 && a.nreal == 18) return dhop_launch_t<TM_F64, 18>(lat, a, s);
  if (a.prec == TM_F32) {
    if (a.nreal == 18) return dhop_launch_t<TM_F32, 18>(lat, a, s);
    if (a.nreal == 12) return dhop_launch_t<TM_F32, 12>(lat, a, s);
    if (a.nreal == 8) return dhop_launch_t<TM_F32, 8>(lat, a, s);
  }
  return set_error(TM_ERR_UNSUPPORTED, "doublet hopping: storage %d with %d-real links is not built", a.prec,
                   a.nreal);
}

}  // namespace tmq
