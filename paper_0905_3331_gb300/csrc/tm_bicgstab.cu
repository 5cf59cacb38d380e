// tm_bicgstab.cu -- BiCGstab on the even/odd Schur operator (Sec. 4.4, eq. eo4) on the device.
//
// System:  M^f x = b.  Source preparation as for CG (App. B.2), varphi_o = b_o - M_oe (M_ee^f)^-1
// b_e, then BiCGstab (van der Vorst 1992) directly on the non-hermitian Schur system
//   Mhat^f x_o = varphi_o,   Mhat^f = (1 + i f mu~ gamma5) - kappa^2 H_oe (M_ee^f)^-1 H_eo,
// and x_e = (M_ee^f)^-1 (b_e + kappa H_eo x_o).  One iteration applies Mhat twice (four hopping
// kernels, like one CG iteration on the normal equations) and needs no normal equations, so its
// Krylov space is built from Mhat rather than Mhat^dag Mhat.
//
// One iteration is eight kernels on the caller's stream; every scalar (rho, alpha, omega, beta,
// ||r||^2) lives in a device-side BiState written by the last block of the kernel that
// completes its reduction (deterministic fixed-order sums):
//   K1, K2  v = Mhat p                (T = (M_ee^f)^-1 H_eo p;  v = (1 + i f mu~ g5) p - kappa^2 H_oe T)
//   A       alpha = rho / <r^, v>
//   S       s = r - alpha v
//   K1, K2  t = Mhat s
//   O       omega = <t, s> / <t, t>
//   X       x += alpha p + omega s;  r = s - omega t;  rho' = <r^, r>, ||r||^2, beta, tests
//   P       p = r + beta (p - omega v)   (sets the loop condition inside a graph)
// Mixed precision follows the CG solver: p, s, v, t (and the operator) in the sloppy storage
// (FP32 or FP16 + norm, 18/12/8-real links, FP32 arithmetic); x, r, r^ in FP32; FP64 sums.
// Reliable updates: when ||r|| falls by delta, x is added to the FP64 solution, the FP64
// residual varphi_o - Mhat x_o replaces r and rho is recomputed; p and r^ carry on.  A
// breakdown (<r^, v> = 0, omega = 0, rho = 0), an overflow or a divergence restarts the method
// from the FP64 residual with a new shadow vector; the increment of a diverging stage is kept
// only if it lowered the FP64 residual.
//
// BiCGstab needs the spectrum of Mhat on one side of the origin: where a few eigenvalues
// have crossed into Re < 0 (kappa beyond the critical value of the gauge field, twisted mass
// alone keeping Mhat invertible) it stagnates while CG on the normal equations still converges.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "tm_solver.cuh"

namespace tmq {

struct BiState {
  double rho_re, rho_im;      // <r^, r>
  double alpha_re, alpha_im;  // rho / <r^, v>
  double omega_re, omega_im;  // <t, s> / <t, t>
  double beta_re, beta_im;
  double rr;                  // ||r||^2 of the iterated residual
  double stop2;               // stop when rr < stop2
  double rr_ref;              // ||r||^2 at the last reliable update
  double delta2;              // reliable update when rr < delta2 rr_ref (0: never)
  double rr_min;
  double grow2;               // divergence guard: rr > grow2 rr_min ends the stage (0: off)
  int iter, max_iter, applied;
  int done, converged, nonfinite, want_update, breakdown, diverged;
  int loops, loop_cap;
};

constexpr int CHUNK_BI = 8;  // iterations per host check without graphs

// ------------------------------------------------------- multi-value sums ---
// Every block adds its N values; the last block to arrive sums the per-block partials in
// fixed order and returns true in thread 0 with the totals in tot[].
// T: the per-thread sums' type (FP32 for FP32 data: the warp's shuffle tree in FP32, then FP64 --
// GB300 runs FP64 adds and conversions at ~1/64 of the FP32 rate).
template <int N, typename T>
__device__ __forceinline__ bool grid_sum(T (&v)[N], double* partials, unsigned* counter, double (&tot)[N]) {
  __shared__ double sh[N][BNT / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    T x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k][warp] = (double)x;
  }
  __syncthreads();
  const int nb = gridDim.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double s = 0.0;
      for (int w = 0; w < BNT / 32; ++w) s += sh[k][w];
      partials[(size_t)k * nb + blockIdx.x] = s;
    }
    last = (arrive_acq_rel(counter) == (unsigned)nb - 1);  // see grid_reduce
  }
  __syncthreads();
  if (!last) return false;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    double x = 0.0;  // partials b = t, t + BNT, ... in order, loads of a group of 8 issued together
    for (int base = threadIdx.x; base < nb; base += 8 * BNT) {
      double t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int b = base + u * BNT;
        t[u] = b < nb ? __ldcg(partials + (size_t)k * nb + b) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) x += t[u];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    __syncthreads();
    if (lane == 0) sh[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x != 0) return false;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    double s = 0.0;
    for (int w = 0; w < BNT / 32; ++w) s += sh[k][w];
    tot[k] = s;
  }
  *counter = 0u;
  return true;
}

__device__ __forceinline__ bool finite2(double a, double b) { return isfinite(a) && isfinite(b); }

// ---------------------------------------------------------------- kernels ---
// alpha = rho / <r^, v>
template <int PR, int PP>
__global__ void __launch_bounds__(BNT) bi_alpha_kernel(int h, const char* rh, const char* v, BiState* st,
                                                       double* partials, unsigned* counter) {
  if (st->done) return;
  typedef typename SpinorFmt<PR>::real RR;
  typedef typename SpinorFmt<PP>::real RP;
  typedef typename SiteSum<RR>::type SR;
  SR acc[2] = {};  // FP32 for FP32 data (the warp tree too), FP64 from the warps on
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    cpx<RR> a[12];
    cpx<RP> b[12];
    SpinorFmt<PR>::load(rh, h, i, a);
    SpinorFmt<PP>::load(v, h, i, b);
    SR l0 = SR(0), l1 = SR(0);
#pragma unroll
    for (int k = 0; k < 12; ++k) {  // conj(a) b
      const SR ar = (SR)a[k].re, ai = (SR)a[k].im, br = (SR)b[k].re, bi = (SR)b[k].im;
      l0 += ar * br + ai * bi;
      l1 += ar * bi - ai * br;
    }
    acc[0] += l0;
    acc[1] += l1;
  }
  double tot[2];
  if (!grid_sum<2>(acc, partials, counter, tot)) return;
  BiState& S = *st;
  const double d = tot[0] * tot[0] + tot[1] * tot[1];
  if (!finite2(tot[0], tot[1])) {
    S.nonfinite = 1;
    S.done = 1;
  } else if (!(d > 0.0)) {
    S.breakdown = 1;
    S.done = 1;
  } else {  // rho / rv
    S.alpha_re = (S.rho_re * tot[0] + S.rho_im * tot[1]) / d;
    S.alpha_im = (S.rho_im * tot[0] - S.rho_re * tot[1]) / d;
  }
}

// s = r - alpha v
template <int PR, int PP>
__global__ void __launch_bounds__(BNT) bi_s_kernel(int h, const char* r, const char* v, char* s, const BiState* st) {
  if (st->done) return;
  typedef typename SpinorFmt<PR>::real RR;
  typedef typename SpinorFmt<PP>::real RP;
  const cpx<RP> al = mk<RP>((RP)st->alpha_re, (RP)st->alpha_im);
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    cpx<RR> a[12];
    cpx<RP> b[12], o[12];
    SpinorFmt<PR>::load(r, h, i, a);
    SpinorFmt<PP>::load(v, h, i, b);
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = mk<RP>((RP)a[k].re, (RP)a[k].im) - al * b[k];
    SpinorFmt<PP>::store(s, h, i, o);
  }
}

// omega = <t, s> / <t, t>
template <int PP>
__global__ void __launch_bounds__(BNT) bi_omega_kernel(int h, const char* s, const char* t, BiState* st,
                                                       double* partials, unsigned* counter) {
  if (st->done) return;
  typedef typename SpinorFmt<PP>::real RP;
  typedef typename SiteSum<RP>::type SR;
  SR acc[3] = {};  // FP32 for FP32 data (the warp tree too), FP64 from the warps on
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    cpx<RP> a[12], b[12];
    SpinorFmt<PP>::load(t, h, i, a);
    SpinorFmt<PP>::load(s, h, i, b);
    SR l[3] = {SR(0), SR(0), SR(0)};
#pragma unroll
    for (int k = 0; k < 12; ++k) {  // conj(t) s, |t|^2
      const SR tr = a[k].re, ti = a[k].im, sr = b[k].re, si = b[k].im;
      l[0] += tr * sr + ti * si;
      l[1] += tr * si - ti * sr;
      l[2] += tr * tr + ti * ti;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) acc[j] += l[j];
  }
  double tot[3];
  if (!grid_sum<3>(acc, partials, counter, tot)) return;
  BiState& S = *st;
  if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
    S.nonfinite = 1;
    S.done = 1;
  } else if (tot[2] > 0.0) {
    S.omega_re = tot[0] / tot[2];
    S.omega_im = tot[1] / tot[2];
  } else {
    S.omega_re = S.omega_im = 0.0;
  }
}

// x += alpha p + omega s;  r = s - omega t;  rho' = <r^, r>, ||r||^2;  beta and the tests
template <int PR, int PP>
__global__ void __launch_bounds__(BNT) bi_xr_kernel(int h, char* x, char* r, const char* rh, const char* p,
                                                    const char* s, const char* t, BiState* st, double* partials,
                                                    unsigned* counter) {
  if (st->done) return;
  typedef typename SpinorFmt<PR>::real RR;
  typedef typename SpinorFmt<PP>::real RP;
  const cpx<RR> al = mk<RR>((RR)st->alpha_re, (RR)st->alpha_im);
  const cpx<RR> om = mk<RR>((RR)st->omega_re, (RR)st->omega_im);
  typedef typename SiteSum<RR>::type SR;
  SR acc[3] = {};  // FP32 for FP32 data (the warp tree too), FP64 from the warps on
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    SR l[3] = {SR(0), SR(0), SR(0)};
    cpx<RR> xv[12], rv[12], hv[12];
    cpx<RP> pv[12], sv[12], tv[12];
    SpinorFmt<PR>::load(x, h, i, xv);
    SpinorFmt<PR>::load(rh, h, i, hv);
    SpinorFmt<PP>::load(p, h, i, pv);
    SpinorFmt<PP>::load(s, h, i, sv);
    SpinorFmt<PP>::load(t, h, i, tv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const cpx<RR> pk = mk<RR>((RR)pv[k].re, (RR)pv[k].im);
      const cpx<RR> sk = mk<RR>((RR)sv[k].re, (RR)sv[k].im);
      const cpx<RR> tk = mk<RR>((RR)tv[k].re, (RR)tv[k].im);
      xv[k] = xv[k] + al * pk + om * sk;
      rv[k] = sk - om * tk;
      const SR rr_ = rv[k].re, ri = rv[k].im, hr = hv[k].re, hi = hv[k].im;
      l[0] += hr * rr_ + hi * ri;
      l[1] += hr * ri - hi * rr_;
      l[2] += rr_ * rr_ + ri * ri;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) acc[j] += l[j];
    SpinorFmt<PR>::store(x, h, i, xv);
    SpinorFmt<PR>::store(r, h, i, rv);
  }
  double tot[3];
  if (!grid_sum<3>(acc, partials, counter, tot)) return;
  BiState& S = *st;
  S.iter += 1;
  if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
    S.nonfinite = 1;
    S.done = 1;
    S.beta_re = S.beta_im = 0.0;
    return;
  }
  const double rr = tot[2];
  S.rr = rr;
  if (rr < S.rr_min) S.rr_min = rr;
  if (rr < S.stop2) {
    S.converged = 1;
    S.done = 1;
  } else if (S.iter >= S.max_iter) {
    S.done = 1;
  } else if (S.delta2 > 0.0 && rr < S.delta2 * S.rr_ref) {
    S.want_update = 1;
    S.done = 1;
  } else if (S.grow2 > 0.0 && rr > S.grow2 * S.rr_min) {
    S.diverged = 1;
    S.done = 1;
  }
  // beta = (rho' / rho) (alpha / omega)
  const double rho2 = S.rho_re * S.rho_re + S.rho_im * S.rho_im;
  const double om2 = S.omega_re * S.omega_re + S.omega_im * S.omega_im;
  const double nr = tot[0] * tot[0] + tot[1] * tot[1];
  if (!(rho2 > 0.0) || !(om2 > 0.0) || !(nr > 0.0)) {
    if (!S.converged) {
      S.breakdown = 1;
      S.done = 1;
    }
    S.beta_re = S.beta_im = 0.0;
  } else {
    // q1 = rho' / rho, q2 = alpha / omega
    const double q1r = (tot[0] * S.rho_re + tot[1] * S.rho_im) / rho2;
    const double q1i = (tot[1] * S.rho_re - tot[0] * S.rho_im) / rho2;
    const double q2r = (S.alpha_re * S.omega_re + S.alpha_im * S.omega_im) / om2;
    const double q2i = (S.alpha_im * S.omega_re - S.alpha_re * S.omega_im) / om2;
    S.beta_re = q1r * q2r - q1i * q2i;
    S.beta_im = q1r * q2i + q1i * q2r;
  }
  S.rho_re = tot[0];
  S.rho_im = tot[1];
}

// p = r + beta (p - omega v), once per iteration; inside a graph loop also the loop condition
template <int PR, int PP>
__global__ void __launch_bounds__(BNT) bi_p_kernel(int h, char* p, const char* r, const char* v, BiState* st,
                                                   unsigned* counter, cudaGraphConditionalHandle cond, int use_cond) {
  BiState& S = *st;
  const int iter = S.iter;
  if (iter == S.applied) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) {
      S.loops += 1;
      cudaGraphSetConditional(cond, 0u);
    }
    return;
  }
  typedef typename SpinorFmt<PR>::real RR;
  typedef typename SpinorFmt<PP>::real RP;
  const cpx<RP> be = mk<RP>((RP)S.beta_re, (RP)S.beta_im);
  const cpx<RP> om = mk<RP>((RP)S.omega_re, (RP)S.omega_im);
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    cpx<RR> rv[12];
    cpx<RP> pv[12], vv[12];
    SpinorFmt<PR>::load(r, h, i, rv);
    SpinorFmt<PP>::load(p, h, i, pv);
    SpinorFmt<PP>::load(v, h, i, vv);
#pragma unroll
    for (int k = 0; k < 12; ++k) pv[k] = mk<RP>((RP)rv[k].re, (RP)rv[k].im) + be * (pv[k] - om * vv[k]);
    SpinorFmt<PP>::store(p, h, i, pv);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive_acq_rel(counter) == gridDim.x - 1) {
      S.applied = iter;
      *counter = 0u;
      if (use_cond) {
        S.loops += 1;
        const bool again = !S.done && S.loops < S.loop_cap;
        cudaGraphSetConditional(cond, again ? 1u : 0u);
      }
    }
  }
}

// rho = <r^, r>, rr = rr_ref = rr_min = ||r||^2 (start of a stage)
template <int PR>
__global__ void __launch_bounds__(BNT) bi_rho_kernel(int h, const char* rh, const char* r, BiState* st,
                                                     double* partials, unsigned* counter) {
  typedef typename SpinorFmt<PR>::real RR;
  typedef typename SiteSum<RR>::type SR;
  SR acc[3] = {};  // FP32 for FP32 data (the warp tree too), FP64 from the warps on
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    cpx<RR> a[12], b[12];
    SpinorFmt<PR>::load(rh, h, i, a);
    SpinorFmt<PR>::load(r, h, i, b);
    SR l[3] = {SR(0), SR(0), SR(0)};
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const SR ar = a[k].re, ai = a[k].im, br = b[k].re, bi = b[k].im;
      l[0] += ar * br + ai * bi;
      l[1] += ar * bi - ai * br;
      l[2] += br * br + bi * bi;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) acc[j] += l[j];
  }
  double tot[3];
  if (!grid_sum<3>(acc, partials, counter, tot)) return;
  BiState& S = *st;
  S.rho_re = tot[0];
  S.rho_im = tot[1];
  S.rr = S.rr_ref = S.rr_min = tot[2];
  if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
    S.nonfinite = 1;
    S.done = 1;
  } else if (tot[2] < S.stop2) {
    S.converged = 1;
    S.done = 1;
  } else if (!(tot[0] * tot[0] + tot[1] * tot[1] > 0.0)) {
    S.breakdown = 1;
    S.done = 1;
  }
}

// ------------------------------------------------------------ MR kernels ---
// Minimal residual (MR) on Mhat: q = Mhat r (two hopping launches), then
//   A  alpha = <q, r> / <q, q>
//   U  x += alpha r;  r -= alpha q;  ||r||^2 and the tests (sets the loop condition)
// r is the operator's input, so it is stored in the operator's format (FP64 or FP32).
template <int P>
__global__ void __launch_bounds__(BNT) mr_alpha_kernel(int h, const char* q, const char* r, BiState* st,
                                                       double* partials, unsigned* counter) {
  if (st->done) return;
  typedef typename SpinorFmt<P>::real R;
  typedef typename SiteSum<R>::type SR;
  SR acc[3] = {};  // FP32 for FP32 data (the warp tree too), FP64 from the warps on
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    cpx<R> a[12], b[12];
    SpinorFmt<P>::load(q, h, i, a);
    SpinorFmt<P>::load(r, h, i, b);
    SR l[3] = {SR(0), SR(0), SR(0)};
#pragma unroll
    for (int k = 0; k < 12; ++k) {  // conj(q) r, |q|^2
      const SR qr = a[k].re, qi = a[k].im, rr_ = b[k].re, ri = b[k].im;
      l[0] += qr * rr_ + qi * ri;
      l[1] += qr * ri - qi * rr_;
      l[2] += qr * qr + qi * qi;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) acc[j] += l[j];
  }
  double tot[3];
  if (!grid_sum<3>(acc, partials, counter, tot)) return;
  BiState& S = *st;
  if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
    S.nonfinite = 1;
    S.done = 1;
  } else if (!(tot[2] > 0.0)) {
    S.breakdown = 1;
    S.done = 1;
  } else {
    S.alpha_re = tot[0] / tot[2];
    S.alpha_im = tot[1] / tot[2];
  }
}

template <int P>
__global__ void __launch_bounds__(BNT) mr_update_kernel(int h, char* x, char* r, const char* q, BiState* st,
                                                        double* partials, unsigned* counter,
                                                        cudaGraphConditionalHandle cond, int use_cond) {
  BiState& S = *st;
  if (S.done) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) {
      S.loops += 1;
      cudaGraphSetConditional(cond, 0u);
    }
    return;
  }
  typedef typename SpinorFmt<P>::real R;
  const cpx<R> al = mk<R>((R)S.alpha_re, (R)S.alpha_im);
  typedef typename SiteSum<R>::type SR;
  SR acc[1] = {};  // FP32 for FP32 data (the warp tree too), FP64 from the warps on
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    cpx<R> xv[12], rv[12], qv[12];
    SpinorFmt<P>::load(x, h, i, xv);
    SpinorFmt<P>::load(r, h, i, rv);
    SpinorFmt<P>::load(q, h, i, qv);
    SR site = SR(0);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      xv[k] = xv[k] + al * rv[k];
      rv[k] = rv[k] - al * qv[k];
      site += (SR)norm2(rv[k]);
    }
    acc[0] += site;
    SpinorFmt<P>::store(x, h, i, xv);
    SpinorFmt<P>::store(r, h, i, rv);
  }
  double tot[1];
  if (!grid_sum<1>(acc, partials, counter, tot)) return;
  S.iter += 1;
  S.applied = S.iter;
  const double rr = tot[0];
  if (!isfinite(rr)) {
    S.nonfinite = 1;
    S.done = 1;
  } else {
    S.rr = rr;
    if (rr < S.rr_min) S.rr_min = rr;
    if (rr < S.stop2) {
      S.converged = 1;
      S.done = 1;
    } else if (S.iter >= S.max_iter) {
      S.done = 1;
    } else if (S.delta2 > 0.0 && rr < S.delta2 * S.rr_ref) {
      S.want_update = 1;
      S.done = 1;
    } else if (S.grow2 > 0.0 && rr > S.grow2 * S.rr_min) {
      S.diverged = 1;
      S.done = 1;
    }
  }
  if (use_cond) {
    S.loops += 1;
    cudaGraphSetConditional(cond, (!S.done && S.loops < S.loop_cap) ? 1u : 0u);
  }
}

// ------------------------------------------------------------------- host ---
struct BiVecs {
  int mr;     // 0 BiCGstab, 1 MR (then r^ = r and r is in the operator's format)
  int pp;     // operator storage precision (p, s, v, t, T)
  int nreal;  // link format
  int pr;     // precision of x, r, r^
  void *x, *r, *rh, *p, *s, *v, *t, *T;  // MR: v holds q = Mhat r
};

static unsigned* bi_counters(tm_lattice lat) { return lat->counters + 4; }

// Mhat^f in -> out (T scratch), in the iteration form (skipped when the state is done)
static tm_status schur_apply(const Solver& S, int prec, int nreal, const void* in, void* T, void* out,
                             const int* skip) {
  tm_lattice lat = S.lat;
  HopArgs a{};
  a.prec = prec;
  a.nreal = nreal;
  a.nrhs = 1;
  a.skip = skip;
  a.out_parity = 0;
  a.in = in;
  a.out = T;
  a.coef = epi_mdiag_inv_hop(S.mut, S.f);
  a.mode = 0;
  tm_status st = hop_launch(lat, a, S.s);
  if (st != TM_OK) return st;
  a.out_parity = 1;
  a.in = T;
  a.y = in;
  a.out = out;
  a.coef = epi_full_M(lat->kappa * lat->kappa, S.mut, S.f);  // (1 + i f mu~ g5) y - kappa^2 H T
  return hop_launch(lat, a, S.s);
}

template <int PR, int PP>
static void launch_iteration_blas(const Solver& S, const BiVecs& v, BiState* st, int which,
                                  cudaGraphConditionalHandle cond, int use_cond) {
  tm_lattice lat = S.lat;
  const int h = lat->geom.h;
  const unsigned nb = blas_blocks(h);
  unsigned* ctr = bi_counters(lat);
  char *x = (char*)v.x, *r = (char*)v.r, *rh = (char*)v.rh, *p = (char*)v.p, *s = (char*)v.s, *vv = (char*)v.v,
       *t = (char*)v.t;
  switch (which) {
    case 0:
      bi_alpha_kernel<PR, PP><<<nb, BNT, 0, S.s>>>(h, rh, vv, st, lat->partials, ctr);
      break;
    case 1:
      bi_s_kernel<PR, PP><<<nb, BNT, 0, S.s>>>(h, r, vv, s, st);
      break;
    case 2:
      bi_omega_kernel<PP><<<nb, BNT, 0, S.s>>>(h, s, t, st, lat->partials, ctr);
      break;
    case 3:
      bi_xr_kernel<PR, PP><<<nb, BNT, 0, S.s>>>(h, x, r, rh, p, s, t, st, lat->partials, ctr);
      break;
    default:
      bi_p_kernel<PR, PP><<<nb, BNT, 0, S.s>>>(h, p, r, vv, st, ctr + 1, cond, use_cond);
      break;
  }
  count_launch();
}

static void blas_step(const Solver& S, const BiVecs& v, BiState* st, int which, cudaGraphConditionalHandle cond = 0,
                      int use_cond = 0) {
  if (v.pr == TM_F64)
    launch_iteration_blas<TM_F64, TM_F64>(S, v, st, which, cond, use_cond);
  else if (v.pp == TM_F32)
    launch_iteration_blas<TM_F32, TM_F32>(S, v, st, which, cond, use_cond);
  else
    launch_iteration_blas<TM_F32, TM_F16>(S, v, st, which, cond, use_cond);
}

static tm_status enqueue_mr_iteration(const Solver& S, const BiVecs& v, BiState* st,
                                      cudaGraphConditionalHandle cond, int use_cond) {
  tm_lattice lat = S.lat;
  const int h = lat->geom.h;
  const unsigned nb = blas_blocks(h);
  unsigned* ctr = bi_counters(lat);
  tm_status e = schur_apply(S, v.pp, v.nreal, v.r, v.T, v.v, &st->done);
  if (e != TM_OK) return e;
  char *x = (char*)v.x, *r = (char*)v.r, *q = (char*)v.v;
  if (v.pp == TM_F64) {
    mr_alpha_kernel<TM_F64><<<nb, BNT, 0, S.s>>>(h, q, r, st, lat->partials, ctr);
    mr_update_kernel<TM_F64><<<nb, BNT, 0, S.s>>>(h, x, r, q, st, lat->partials, ctr + 1, cond, use_cond);
  } else {
    mr_alpha_kernel<TM_F32><<<nb, BNT, 0, S.s>>>(h, q, r, st, lat->partials, ctr);
    mr_update_kernel<TM_F32><<<nb, BNT, 0, S.s>>>(h, x, r, q, st, lat->partials, ctr + 1, cond, use_cond);
  }
  count_launch(2);
  return cuda_check(cudaGetLastError(), "MR kernels");
}

// One BiCGstab iteration (eight kernels), or one MR iteration (four).
static tm_status enqueue_iteration(const Solver& S, const BiVecs& v, BiState* st, cudaGraphConditionalHandle cond,
                                   int use_cond) {
  if (v.mr) return enqueue_mr_iteration(S, v, st, cond, use_cond);
  tm_status e;
  if ((e = schur_apply(S, v.pp, v.nreal, v.p, v.T, v.v, &st->done)) != TM_OK) return e;
  blas_step(S, v, st, 0);
  blas_step(S, v, st, 1);
  if ((e = schur_apply(S, v.pp, v.nreal, v.s, v.T, v.t, &st->done)) != TM_OK) return e;
  blas_step(S, v, st, 2);
  blas_step(S, v, st, 3);
  blas_step(S, v, st, 4, cond, use_cond);
  return cuda_check(cudaGetLastError(), "BiCGstab kernels");
}

static tm_status bi_graph(const Solver& S, const BiVecs& v, BiState* dst, cudaGraphExec_t* out) {
  tm_lattice lat = S.lat;
  unsigned long long key[16] = {};
  key[0] = v.mr ? 0x3A11ull : 0xB1C6ull;
  key[1] = (unsigned long long)v.pp | ((unsigned long long)v.nreal << 8) | ((unsigned long long)v.pr << 16) |
           ((unsigned long long)(S.f + 1) << 24);
  memcpy(&key[2], &lat->kappa, sizeof(double));
  memcpy(&key[3], &lat->mu, sizeof(double));
  const void* ptrs[10] = {v.x, v.r, v.rh, v.p, v.s, v.v, v.t, v.T, dst, lat->partials};
  for (int k = 0; k < 10; ++k) key[4 + k] = (unsigned long long)(uintptr_t)ptrs[k];
  key[14] = (unsigned long long)(uintptr_t)lat->counters;
  tm_status st = ensure_links(lat, v.pp, v.nreal, S.s);
  if (st != TM_OK) return st;
  return aux_loop_graph(lat, key, S.s, [&](cudaStream_t cs, cudaGraphConditionalHandle cond) {
    Solver C = S;
    C.s = cs;
    return enqueue_iteration(C, v, dst, cond, 1);
  }, out);
}

// Runs one stage: uploads `init`, recomputes rho and ||r||^2 on the device, iterates until the
// state is done, reads the state back.
static tm_status run_bi_stage(const Solver& S, const BiVecs& v, BiState* dst, const BiState& init, BiState* out) {
  tm_lattice lat = S.lat;
  tm_status st;
  BiState hs = init;
  hs.loops = 0;
  hs.loop_cap = (init.max_iter - init.iter) + 2;
  hs.applied = init.iter;
  if ((st = cuda_check(cudaMemcpyAsync(dst, &hs, sizeof(BiState), cudaMemcpyHostToDevice, S.s), "state")) != TM_OK)
    return st;
  const unsigned nb = blas_blocks(lat->geom.h);
  if (v.pr == TM_F64)
    bi_rho_kernel<TM_F64><<<nb, BNT, 0, S.s>>>(lat->geom.h, (const char*)v.rh, (const char*)v.r, dst, lat->partials,
                                                bi_counters(lat));
  else
    bi_rho_kernel<TM_F32><<<nb, BNT, 0, S.s>>>(lat->geom.h, (const char*)v.rh, (const char*)v.r, dst, lat->partials,
                                                bi_counters(lat));
  count_launch();
  if ((st = cuda_check(cudaGetLastError(), "rho kernel")) != TM_OK) return st;
  if (use_graphs()) {
    cudaGraphExec_t ex;
    if ((st = bi_graph(S, v, dst, &ex)) != TM_OK) return st;
    if ((st = cuda_check(cudaGraphLaunch(ex, S.s), "graph launch")) != TM_OK) return st;
    if ((st = cuda_check(cudaMemcpyAsync(&hs, dst, sizeof(BiState), cudaMemcpyDeviceToHost, S.s), "state")) != TM_OK)
      return st;
    if ((st = cuda_check(cudaStreamSynchronize(S.s), "BiCGstab stage")) != TM_OK) return st;
    count_launch((v.mr ? 4u : 8u) * (unsigned)hs.loops);
    if (!hs.done) return set_error(TM_ERR_TIMEOUT, "solver stage loop reached its bound without finishing");
  } else {
    if ((st = ensure_links(lat, v.pp, v.nreal, S.s)) != TM_OK) return st;
    for (;;) {
      for (int k = 0; k < CHUNK_BI; ++k)
        if ((st = enqueue_iteration(S, v, dst, 0, 0)) != TM_OK) return st;
      if ((st = cuda_check(cudaMemcpyAsync(&hs, dst, sizeof(BiState), cudaMemcpyDeviceToHost, S.s), "state")) !=
          TM_OK)
        return st;
      if ((st = cuda_check(cudaStreamSynchronize(S.s), "BiCGstab chunk")) != TM_OK) return st;
      if (hs.done && hs.applied == hs.iter) break;
    }
  }
  *out = hs;
  return TM_OK;
}

// R = B - Mhat X in FP64 (2 FP64 hopping kernels); returns ||R||^2.
static tm_status schur_residual(const Solver& S, void* R, const void* X, const void* B, void* T, double* rr) {
  tm_lattice lat = S.lat;
  tm_status st = cuda_check(cudaMemcpyAsync(R, B, S.hb[TM_F64], cudaMemcpyDeviceToDevice, S.s), "copy");
  if (st != TM_OK) return st;
  HopArgs a{};
  a.prec = TM_F64;
  a.nreal = 18;
  a.nrhs = 1;
  a.out_parity = 0;
  a.in = X;
  a.out = T;
  a.coef = epi_mdiag_inv_hop(S.mut, S.f);
  if ((st = hop_launch(lat, a, S.s)) != TM_OK) return st;
  a.out_parity = 1;
  a.in = T;
  a.y = X;
  a.out = R;  // R -= Mhat X, ||R||^2 into dscalars[0]
  a.coef = epi_full_M(lat->kappa * lat->kappa, S.mut, S.f);
  a.mode = 2;
  a.alpha_src = nullptr;
  a.alpha_sign = 1.0;
  a.red = Reduce{lat->partials, lat->counters, lat->dscalars, nullptr, FIN_STORE};
  if ((st = hop_launch(lat, a, S.s)) != TM_OK) return st;
  if ((st = cuda_check(cudaMemcpyAsync(rr, lat->dscalars, sizeof(double), cudaMemcpyDeviceToHost, S.s), "readback")) !=
      TM_OK)
    return st;
  return cuda_check(cudaStreamSynchronize(S.s), "synchronise");
}

static bool bi_verbose() {
  const char* e = getenv("TM_VERBOSE");
  return e && *e && *e != '0';
}

static tm_status solve_one_krylov(tm_lattice lat, double* x, const double* b, const tm_cg_params& P,
                                  tm_cg_info* info, cudaStream_t s, bool mr);

tm_status solve_one_bicgstab(tm_lattice lat, double* x, const double* b, const tm_cg_params& P, tm_cg_info* info,
                             cudaStream_t s) {
  return solve_one_krylov(lat, x, b, P, info, s, false);
}

tm_status solve_one_mr(tm_lattice lat, double* x, const double* b, const tm_cg_params& P, tm_cg_info* info,
                       cudaStream_t s) {
  return solve_one_krylov(lat, x, b, P, info, s, true);
}

// BiCGstab (mr false) or MR (mr true) on Mhat^f x_o = varphi_o for one canonical full field.
static tm_status solve_one_krylov(tm_lattice lat, double* x, const double* b, const tm_cg_params& P, tm_cg_info* info,
                                  cudaStream_t s, bool mr) {
  const char* nm = mr ? "tm_solve_mr" : "tm_solve_bicgstab";
  Solver S{lat, s, P.flavour, 2.0 * lat->kappa * lat->mu, {0, 0, 0, 0}};
  for (int p = 0; p < 4; ++p) S.hb[p] = spinor_bytes_per_site(p) * lat->h;
  tm_status st = TM_OK;
  // FP64 fields: 0 b_e, 1 b_o, 2 b' (then varphi_o), 3 X, 4 R, 5 T, 6 / 7 scratch of the checks
  void* w[8];
  for (int k = 0; k < 8; ++k) {
    w[k] = workspace(lat, k, S.hb[TM_F64], &st);
    if (st != TM_OK) return st;
  }
  void *be = w[0], *bo = w[1], *B = w[2], *X = w[3], *R = w[4], *T = w[5];
  double bb = 0.0, bfull = 0.0;
  if ((st = prepare_source(S, b, be, bo, B, T, &bb, &bfull)) != TM_OK) return st;
  if (!std::isfinite(bb) || !std::isfinite(bfull))
    return set_error(TM_ERR_NONFINITE, "%s: the source has non-finite entries", nm);
  // prepare_source gives gamma5 varphi_o; the Schur system wants varphi_o itself
  if ((st = diag_apply(lat, TM_F64, B, B, 1, 1.0, 0.0, -1.0, 0.0, s)) != TM_OK) return st;
  info->iters = 0;
  info->reliable_updates = 0;
  if (bfull == 0.0) {
    st = cuda_check(cudaMemsetAsync(x, 0, lat->V * 24 * sizeof(double), s), "memset");
    info->true_rel_residual = info->schur_rel_residual = 0.0;
    info->status = TM_OK;
    return st;
  }
  if ((st = cuda_check(cudaMemsetAsync(X, 0, S.hb[TM_F64], s), "memset")) != TM_OK) return st;
  if ((st = cuda_check(cudaMemcpyAsync(R, B, S.hb[TM_F64], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK) return st;
  const bool fp64 = P.mode == TM_CG_FP64;
  BiVecs v{};
  v.mr = mr ? 1 : 0;
  if (mr) {  // x, r (the operator's input), q = Mhat r, T: all in the operator's format
    v.pp = fp64 ? TM_F64 : TM_F32;
    v.nreal = fp64 ? 18 : P.sloppy_link;
    v.pr = v.pp;
    v.T = T;
    if (fp64) {
      v.x = X;
      v.r = R;
    } else {
      v.x = workspace(lat, 9, S.hb[TM_F32], &st);
      if (st == TM_OK) v.r = workspace(lat, 8, S.hb[TM_F32], &st);
      if (st == TM_OK) v.T = workspace(lat, 11, S.hb[TM_F32], &st);
    }
    if (st == TM_OK) v.v = workspace(lat, 19, S.hb[v.pp], &st);
    v.rh = v.r;
  } else if (fp64) {
    v.pp = TM_F64;
    v.nreal = 18;
    v.pr = TM_F64;
    v.x = X;
    v.r = R;
    v.T = T;
    v.p = workspace(lat, 6, S.hb[TM_F64], &st);
    if (st == TM_OK) v.s = workspace(lat, 7, S.hb[TM_F64], &st);
    if (st == TM_OK) v.rh = workspace(lat, 18, S.hb[TM_F64], &st);
    if (st == TM_OK) v.v = workspace(lat, 19, S.hb[TM_F64], &st);
    if (st == TM_OK) v.t = workspace(lat, 20, S.hb[TM_F64], &st);
  } else {
    const int sp = P.sloppy_prec;
    v.pp = sp;
    v.nreal = P.sloppy_link;
    v.pr = TM_F32;
    v.x = workspace(lat, 9, S.hb[TM_F32], &st);
    if (st == TM_OK) v.r = workspace(lat, 8, S.hb[TM_F32], &st);
    if (st == TM_OK) v.rh = workspace(lat, 18, S.hb[TM_F32], &st);
    if (st == TM_OK) v.p = workspace(lat, 10, S.hb[sp], &st);
    if (st == TM_OK) v.T = workspace(lat, 11, S.hb[sp], &st);
    if (st == TM_OK) v.s = workspace(lat, 12, S.hb[sp], &st);
    if (st == TM_OK) v.v = workspace(lat, 19, S.hb[sp], &st);
    if (st == TM_OK) v.t = workspace(lat, 20, S.hb[sp], &st);
  }
  if (st != TM_OK) return st;
  if ((st = ensure_reduce(lat, 3 * (size_t)blas_blocks(lat->geom.h), 8)) != TM_OK) return st;
  BiState* dst = static_cast<BiState*>(workspace(lat, WS_BISTATE, sizeof(BiState), &st));
  if (st != TM_OK) return st;

  const double stop2 = P.tol * P.tol * bb;
  const double delta2 = fp64 ? 0.0 : P.delta * P.delta;
  double rr_true = bb;
  int iters = 0, updates = 0, bad = 0, stall = 0, dropped = 0;
  bool converged = rr_true < stop2, restart = true, reconstructed = false;
  while (!converged && iters < P.max_iter) {
    // r from the FP64 residual R; on a restart also r^ = r, p = r and a zero increment
    if (mr) {
      if (!fp64) {
        if ((st = convert_half(lat, TM_F32, v.r, TM_F64, R, s)) != TM_OK) return st;
        if ((st = cuda_check(cudaMemsetAsync(v.x, 0, S.hb[TM_F32], s), "memset")) != TM_OK) return st;
      }
    } else if (fp64) {
      if (restart) {
        if ((st = cuda_check(cudaMemcpyAsync(v.rh, R, S.hb[TM_F64], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK)
          return st;
        if ((st = cuda_check(cudaMemcpyAsync(v.p, R, S.hb[TM_F64], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK)
          return st;
      }
    } else {
      if ((st = convert_half(lat, TM_F32, v.r, TM_F64, R, s)) != TM_OK) return st;
      if ((st = cuda_check(cudaMemsetAsync(v.x, 0, S.hb[TM_F32], s), "memset")) != TM_OK) return st;
      if (restart) {
        if ((st = convert_half(lat, TM_F32, v.rh, TM_F64, R, s)) != TM_OK) return st;
        if ((st = convert_half(lat, v.pp, v.p, TM_F64, R, s)) != TM_OK) return st;
      }
    }
    BiState init{};
    init.stop2 = stop2;
    init.delta2 = delta2;
    init.grow2 = fp64 ? 0.0 : SLOPPY_GROWTH;
    init.iter = iters;
    init.max_iter = P.max_iter;
    BiState fin;
    if ((st = run_bi_stage(S, v, dst, init, &fin)) != TM_OK) return st;
    if (bi_verbose())
      fprintf(stderr,
              "[%s] stage: iter %d |r|/|b| %.3e converged %d update %d breakdown %d diverged %d "
              "nonfinite %d\n",
              nm, fin.iter, std::sqrt(fin.rr / bb), fin.converged, fin.want_update, fin.breakdown, fin.diverged,
              fin.nonfinite);
    const bool progress = fin.iter > iters;
    iters = fin.iter;
    if (fin.nonfinite) {
      if (++bad > 3 || fp64) return set_error(TM_ERR_NONFINITE, "%s: non-finite value in the iteration", nm);
      restart = true;  // drop the sloppy increment
      continue;
    }
    bad = 0;
    const double rr_before = rr_true;
    const bool keep_backup = !fp64 && fin.diverged;
    if (keep_backup) {  // a diverging stage may leave a worse iterate: keep the FP64 solution
      if ((st = cuda_check(cudaMemcpyAsync(w[6], X, S.hb[TM_F64], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK)
        return st;
      if ((st = cuda_check(cudaMemcpyAsync(w[7], R, S.hb[TM_F64], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK)
        return st;
    }
    if (!fp64) {
      if ((st = launch_accumulate(S, X, v.x)) != TM_OK) return st;
    }
    if (fin.converged && !keep_backup) {
      // confirm through the reconstruction: the odd part of its FP64 full-system residual is
      // ||varphi_o - Mhat X|| up to the rounding of x_e (2 FP64 hopping launches instead of the
      // Schur residual's 2 followed by the reconstruction's 2)
      double rro = 0.0;
      if ((st = reconstruct_xo(S, X, be, bo, bfull, x, T, w[6], w[7], &info->true_rel_residual, &rro)) != TM_OK)
        return st;
      ++updates;
      if (bi_verbose())
        fprintf(stderr, "[%s] confirmation: FP64 |(b - M x)_o|/|b'| %.3e (%s)\n", nm, std::sqrt(rro / bb),
                rro < stop2 ? "converged" : "not confirmed, continuing");
      if (rro < stop2) {
        rr_true = rro;
        converged = reconstructed = true;
        break;
      }
    }
    if ((st = schur_residual(S, R, X, B, T, &rr_true)) != TM_OK) return st;
    if (keep_backup && !(rr_true < rr_before)) {  // drop the increment, restart from the old solution
      if ((st = cuda_check(cudaMemcpyAsync(X, w[6], S.hb[TM_F64], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK)
        return st;
      if ((st = cuda_check(cudaMemcpyAsync(R, w[7], S.hb[TM_F64], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK)
        return st;
      rr_true = rr_before;
      if (++dropped > 3) break;  // the sloppy iteration keeps diverging: report not converged
    } else {
      dropped = 0;
    }
    ++updates;
    if (bi_verbose()) fprintf(stderr, "[%s] update %d: true |r|/|b| %.3e\n", nm, updates, std::sqrt(rr_true / bb));
    if (!(rr_true < 1e300)) return set_error(TM_ERR_NONFINITE, "%s: residual diverged", nm);
    if (rr_true < stop2) {
      converged = true;
      break;
    }
    if (progress)
      stall = 0;
    else if (++stall > 2)
      break;  // repeated breakdown without progress: report not converged
    // FP64: the iterated residual drifted (or broke down): restart.  Mixed: a reliable update
    // keeps p and r^; breakdown, divergence and a false convergence restart.
    restart = fp64 || fin.breakdown || fin.diverged || fin.converged || !fin.want_update;
  }
  info->iters = iters;
  info->reliable_updates = updates;
  info->schur_rel_residual = std::sqrt(rr_true / bb);
  if (!reconstructed &&
      (st = reconstruct_xo(S, X, be, bo, bfull, x, T, w[6], w[7], &info->true_rel_residual)) != TM_OK)
    return st;
  info->status = converged ? TM_OK : TM_ERR_NOT_CONVERGED;
  if (!converged)
    return set_error(TM_ERR_NOT_CONVERGED, "%s: not converged after %d iterations (||r||/||b|| = %.3e)", nm,
                     iters, info->schur_rel_residual);
  return TM_OK;
}

}  // namespace tmq

using namespace tmq;

extern "C" tm_status tm_solve_bicgstab(tm_lattice lat, double* x, const double* b, int nrhs,
                                       const tm_cg_params* params, tm_cg_info* info, void* stream) {
  return solve_driver(lat, x, b, nrhs, params, info, stream, SOLVER_BICGSTAB);
}

extern "C" tm_status tm_solve_mr(tm_lattice lat, double* x, const double* b, int nrhs, const tm_cg_params* params,
                                 tm_cg_info* info, void* stream) {
  return solve_driver(lat, x, b, nrhs, params, info, stream, SOLVER_MR);
}
