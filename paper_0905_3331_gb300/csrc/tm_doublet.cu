// tm_doublet.cu -- the mass non-degenerate doublet (eq. Dh): operator and even/odd CG solve.
//
// Hopping-parameter form (eq. eo0 with the doublet's site term):
//   M_h = D - kappa H,   D = 1_f + i mb gamma5 tau3 + eb tau1,   mb = 2 kappa mubar, eb = 2 kappa epsbar,
// with H the one-flavour hopping sum acting on both flavours alike.  Per chirality g = +-1 (the
// eigenvalue of gamma5 on spins 0,1 / 2,3) D is the flavour matrix [[1 + i mb g, eb], [eb, 1 - i mb g]]
// with determinant n = 1 + mb^2 - eb^2, so D^-1 = (1 - i mb gamma5 tau3 - eb tau1) / n.
//
// Even/odd (the block elimination of App. B.1, written out for the doublet's site term):
//   Mhat_h = D - kappa^2 H_oe D^-1 H_eo on odd sites, varphi_o = phi_o + kappa H_oe D^-1 phi_e,
//   x_e = D^-1 (phi_e + kappa H_eo x_o).
// Mhat_h^dag = G Mhat_h G with G = gamma5 tau1 (G^2 = 1; the relation D_h^dag = tau1 gamma5 D_h
// gamma5 tau1 of Sec. 2.3 holds block by block), so Qhat_h = G Mhat_h is hermitian and CG runs on
//   Qhat_h^2 y = G varphi_o,   x_o = Qhat_h y,
// whose residual G (varphi_o - Mhat_h x_o) has the norm of the Schur residual.
//
// Fields: a doublet half field is two one-flavour half fields back to back (upper flavour,
// tau3 = +1, first), each in the library's half-field layout.  The hopping term runs in the
// two-flavour kernel of tm_dslash_doublet.cu (both flavours of a site in one thread, each link
// loaded once), whose epilogue applies the flavour-mixing site term, the gamma5 tau1 swap and
// the fused CG reductions; purely site-local steps use the site kernel below.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "tm_doublet.cuh"
#include "tm_solver.cuh"

namespace tmq {

static DCoef dcoef_zero() {
  DCoef c;
  memset(&c, 0, sizeof(c));
  return c;
}
static void set_D(double (&M)[2][2][2][2], double mb, double eb, double scale) {  // scale * D
  for (int c = 0; c < 2; ++c) {
    const double g = c == 0 ? 1.0 : -1.0;
    M[c][0][0][0] = scale;
    M[c][0][0][1] = scale * mb * g;
    M[c][1][1][0] = scale;
    M[c][1][1][1] = -scale * mb * g;
    M[c][0][1][0] = M[c][1][0][0] = scale * eb;
    M[c][0][1][1] = M[c][1][0][1] = 0.0;
  }
}
static void set_Dinv(double (&M)[2][2][2][2], double mb, double eb, double scale) {  // scale * D^-1
  const double n = 1.0 + mb * mb - eb * eb;
  for (int c = 0; c < 2; ++c) {
    const double g = c == 0 ? 1.0 : -1.0;
    M[c][0][0][0] = scale / n;
    M[c][0][0][1] = -scale * mb * g / n;
    M[c][1][1][0] = scale / n;
    M[c][1][1][1] = scale * mb * g / n;
    M[c][0][1][0] = M[c][1][0][0] = -scale * eb / n;
    M[c][0][1][1] = M[c][1][0][1] = 0.0;
  }
}
static void set_I(double (&M)[2][2][2][2], double scale) {
  for (int c = 0; c < 2; ++c) {
    memset(M[c], 0, sizeof(M[c]));
    M[c][0][0][0] = M[c][1][1][0] = scale;
  }
}

// MODE 0: out = ...;  1: out = ..., sum |out|^2;  2: r -= alpha (...), sum |r|^2.
// Reductions finish through grid_reduce (FIN_STORE / FIN_CG_ALPHA / FIN_CG_RR).
template <int P, int MODE>
__global__ void __launch_bounds__(BNT) dsite_kernel(int h, const char* a, const char* b, char* out, size_t stride,
                                                    char* r, size_t rstride, DCoef co, Reduce red,
                                                    const int* skip, const CGState* alpha_src) {
  if (skip && *skip) return;
  typedef typename SpinorFmt<P>::real R;
  constexpr int PR = ResidPrec<P>::value;
  typedef typename SpinorFmt<PR>::real RR;
  __shared__ double sh[BNT / 32];
  typedef typename SiteSum<R>::type SR;
  SR acc = SR(0);  // this thread's sites: FP32 for FP32 data (the warp tree too), FP64 after
  const double al = MODE == 2 ? (alpha_src ? alpha_src->alpha : 1.0) : 0.0;
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    SR site = SR(0);
    cpx<R> va[2][12], vb[2][12], o[2][12];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      if (a) SpinorFmt<P>::load(a + f * stride, h, i, va[f]);
      if (b) SpinorFmt<P>::load(b + f * stride, h, i, vb[f]);
    }
#pragma unroll
    for (int f = 0; f < 2; ++f)
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const int c = k < 6 ? 0 : 1;  // spins 0,1: gamma5 = +1; spins 2,3: -1
        cpx<R> s = mk<R>(R(0), R(0));
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          if (a) s = s + dco<R>(co.P[c][f][g], co.fP[c][f][g]) * va[g][k];
          if (b) s = s + dco<R>(co.Q[c][f][g], co.fQ[c][f][g]) * vb[g][k];
        }
        o[f][k] = s;
      }
    if (co.swap) {  // G = gamma5 tau1: swap the flavours, negate the lower spins
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const cpx<R> t = o[0][k];
        o[0][k] = k < 6 ? o[1][k] : mk<R>(-o[1][k].re, -o[1][k].im);
        o[1][k] = k < 6 ? t : mk<R>(-t.re, -t.im);
      }
    }
    if (MODE == 2) {
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        cpx<RR> rv[12];
        SpinorFmt<PR>::load(r + f * rstride, h, i, rv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          rv[k] = rv[k] - (RR)al * mk<RR>((RR)o[f][k].re, (RR)o[f][k].im);
          site += (SR)norm2(rv[k]);
        }
        SpinorFmt<PR>::store(r + f * rstride, h, i, rv);
      }
    } else {
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        SpinorFmt<P>::store(out + f * stride, h, i, o[f]);
        if (MODE == 1)
#pragma unroll
          for (int k = 0; k < 12; ++k)
            site += (SR)norm2(o[f][k]);
      }
    }
    acc += site;
  }
  if (MODE != 0) {
    const double bs = block_sum<BNT>(acc, sh);
    grid_reduce<BNT>(red, 0, gridDim.x, blockIdx.x, bs, sh);
  }
}

// Doublet solver context: the one-flavour Solver (flavour unused) plus mb, eb.
struct DSolver {
  Solver S;
  double mb, eb;
};

static tm_status dsite(const DSolver& D, int prec, int mode, const void* a, const void* b, void* out, void* r,
                       const DCoef& co, const Reduce& red, const int* skip = nullptr,
                       const CGState* alpha_src = nullptr) {
  tm_lattice lat = D.S.lat;
  const int h = lat->geom.h;
  const unsigned nb = blas_blocks(h);
  const size_t st = D.S.hb[prec];
  const size_t rst = D.S.hb[prec == TM_F64 ? TM_F64 : TM_F32];
  const char* ac = static_cast<const char*>(a);
  const char* bc = static_cast<const char*>(b);
  char* oc = static_cast<char*>(out);
  char* rc = static_cast<char*>(r);
  const DCoef cf = dcoef_finish(co);
#define DSITE_LAUNCH(PP, MM) \
  dsite_kernel<PP, MM><<<nb, BNT, 0, D.S.s>>>(h, ac, bc, oc, st, rc, rst, cf, red, skip, alpha_src)
  if (mode != 0) return set_error(TM_ERR_ARG, "internal: doublet site kernel mode %d", mode);
  if (prec == TM_F64)
    DSITE_LAUNCH(TM_F64, 0);
  else
    DSITE_LAUNCH(TM_F32, 0);
#undef DSITE_LAUNCH
  count_launch();
  return cuda_check(cudaGetLastError(), "doublet site kernel");
}

// Fused two-flavour hopping: out = [G] (P y + Q H_{p,1-p} in), see tm_doublet.cuh.
static tm_status dhop(const DSolver& D, int prec, int nreal, int out_parity, const void* in, const void* y,
                      void* out, const DCoef& co, int mode = 0, const Reduce& red = Reduce{},
                      const int* skip = nullptr, const CGState* alpha_src = nullptr) {
  DHopArgs a{};
  a.prec = prec;
  a.nreal = nreal;
  a.out_parity = out_parity;
  a.in = in;
  a.stride = D.S.hb[prec];
  a.out = out;
  a.out_stride = mode == 2 ? D.S.hb[prec == TM_F64 ? TM_F64 : TM_F32] : D.S.hb[prec];
  a.y = y;
  a.co = co;
  a.mode = mode;
  a.alpha_src = alpha_src;
  a.red = red;
  a.skip = skip;
  return dhop_launch(D.S.lat, a, D.S.s);
}

// the coefficient sets of the operator
static DCoef co_dinv_hop(const DSolver& D) {  // D^-1 H in
  DCoef c = dcoef_zero();
  set_Dinv(c.Q, D.mb, D.eb, 1.0);
  return c;
}
static DCoef co_schur_g(const DSolver& D) {  // G (D y - kappa^2 H in)
  DCoef c = dcoef_zero();
  set_D(c.P, D.mb, D.eb, 1.0);
  set_I(c.Q, -D.S.lat->kappa * D.S.lat->kappa);
  c.swap = 1;
  return c;
}

// r -= alpha Qhat_h^2 p  (Qhat_h = G Mhat_h), iteration form with `state` (alpha from the state,
// <p, A p> = ||Qhat_h p||^2 finalised into alpha, ||r||^2 into beta and the tests); without it
// alpha = 1 and ||r||^2 goes to dscalars[0].  T, W: work fields of format prec.  Four launches.
static tm_status dnormal_apply(const DSolver& D, int prec, int nreal, const void* p, void* T, void* W, void* r,
                               CGState* state) {
  tm_lattice lat = D.S.lat;
  tm_status st = ensure_reduce(lat, (lat->geom.h + 127) / 128, 4);
  if (st != TM_OK) return st;
  const int* skip = state ? &state->done : nullptr;
  const DCoef dinv = co_dinv_hop(D), comb = co_schur_g(D);
  // W = Qhat_h p = G (D p - kappa^2 H_oe D^-1 H_eo p)
  if ((st = dhop(D, prec, nreal, 0, p, nullptr, T, dinv, 0, Reduce{}, skip)) != TM_OK) return st;
  if (state) {
    const Reduce ra{lat->partials, lat->counters, nullptr, state, FIN_CG_ALPHA};
    if ((st = dhop(D, prec, nreal, 1, T, p, W, comb, 1, ra, skip)) != TM_OK) return st;
  } else if ((st = dhop(D, prec, nreal, 1, T, p, W, comb)) != TM_OK) {
    return st;
  }
  // r -= alpha Qhat_h W
  if ((st = dhop(D, prec, nreal, 0, W, nullptr, T, dinv, 0, Reduce{}, skip)) != TM_OK) return st;
  const Reduce rr = state ? Reduce{lat->partials, lat->counters, nullptr, state, FIN_CG_RR}
                          : Reduce{lat->partials, lat->counters, lat->dscalars, nullptr, FIN_STORE};
  return dhop(D, prec, nreal, 1, T, W, r, comb, 2, rr, skip, state);
}

// r = b' - Qhat_h^2 X in FP64; ||r||^2 returned (synchronises)
static tm_status dtrue_residual(const DSolver& D, void* r, const void* X, const void* bp, void* T, void* W,
                                double* rr) {
  tm_status st = cuda_check(cudaMemcpyAsync(r, bp, 2 * D.S.hb[TM_F64], cudaMemcpyDeviceToDevice, D.S.s), "copy");
  if (st != TM_OK) return st;
  if ((st = dnormal_apply(D, TM_F64, 18, X, T, W, r, nullptr)) != TM_OK) return st;
  if ((st = cuda_check(cudaMemcpyAsync(rr, D.S.lat->dscalars, sizeof(double), cudaMemcpyDeviceToHost, D.S.s),
                       "readback")) != TM_OK)
    return st;
  return cuda_check(cudaStreamSynchronize(D.S.s), "synchronise");
}

struct DVecs {
  int prec, nreal;  // operator storage (p, T, W); x and r are FP64 (prec F64) or FP32
  void *x, *r, *p, *T, *W;
};

static tm_status enqueue_diter(const DSolver& D, const DVecs& v, CGState* state, cudaGraphConditionalHandle cond,
                               int use_cond) {
  tm_status st = dnormal_apply(D, v.prec, v.nreal, v.p, v.T, v.W, v.r, state);
  if (st != TM_OK) return st;
  const int px = v.prec == TM_F64 ? TM_F64 : TM_F32;
  return launch_update_n(D.S, 2 * D.S.lat->geom.h, px, v.prec, v.x, v.p, v.r, state, cond, use_cond);
}

// One CG stage from `init` until the device state says done.
static tm_status run_dstage(const DSolver& D, const DVecs& v, const CGState& init, CGState* out) {
  tm_lattice lat = D.S.lat;
  tm_status st = ensure_cgstate(lat, 2);
  if (st != TM_OK) return st;
  if ((st = ensure_links(lat, v.prec, v.nreal, D.S.s)) != TM_OK) return st;
  CGState* dst = lat->cgstate;
  CGState* hst = lat->cgstate_host;
  hst[0] = init;
  hst[0].loops = 0;
  hst[0].loop_cap = (init.max_iter - init.iter) + 2;
  if ((st = cuda_check(cudaMemcpyAsync(dst, &hst[0], sizeof(CGState), cudaMemcpyHostToDevice, D.S.s), "state")) !=
      TM_OK)
    return st;
  if (use_graphs()) {
    unsigned long long key[16] = {};
    key[0] = 0xD0B1ull;
    key[1] = (unsigned long long)v.prec | ((unsigned long long)v.nreal << 8);
    memcpy(&key[2], &lat->kappa, sizeof(double));
    memcpy(&key[3], &D.mb, sizeof(double));
    memcpy(&key[4], &D.eb, sizeof(double));
    const void* ptrs[8] = {v.x, v.r, v.p, v.T, v.W, dst, lat->partials, lat->counters};
    for (int k = 0; k < 8; ++k) key[5 + k] = (unsigned long long)(uintptr_t)ptrs[k];
    cudaGraphExec_t ex;
    st = aux_loop_graph(lat, key, D.S.s, [&](cudaStream_t cs, cudaGraphConditionalHandle cond) {
      DSolver C = D;
      C.S.s = cs;
      return enqueue_diter(C, v, dst, cond, 1);
    }, &ex);
    if (st != TM_OK) return st;
    if ((st = cuda_check(cudaGraphLaunch(ex, D.S.s), "graph launch")) != TM_OK) return st;
    if ((st = cuda_check(cudaMemcpyAsync(&hst[1], dst, sizeof(CGState), cudaMemcpyDeviceToHost, D.S.s), "state")) !=
        TM_OK)
      return st;
    if ((st = cuda_check(cudaStreamSynchronize(D.S.s), "doublet CG stage")) != TM_OK) return st;
    count_launch(5u * (unsigned)hst[1].loops);
    if (!hst[1].done) return set_error(TM_ERR_TIMEOUT, "tm_solve_doublet: stage loop reached its bound");
    *out = hst[1];
    return TM_OK;
  }
  for (;;) {
    for (int k = 0; k < 8; ++k)
      if ((st = enqueue_diter(D, v, dst, 0, 0)) != TM_OK) return st;
    if ((st = cuda_check(cudaMemcpyAsync(&hst[1], dst, sizeof(CGState), cudaMemcpyDeviceToHost, D.S.s), "state")) !=
        TM_OK)
      return st;
    if ((st = cuda_check(cudaStreamSynchronize(D.S.s), "doublet CG chunk")) != TM_OK) return st;
    if (hst[1].done && hst[1].applied == hst[1].iter) break;
  }
  *out = hst[1];
  return TM_OK;
}

// both flavours of a doublet half field: precision conversion / FP64 accumulation per flavour
static tm_status dconvert(const DSolver& D, int pout, void* dst, int pin, const void* src) {
  for (int f = 0; f < 2; ++f) {
    tm_status st = convert_half(D.S.lat, pout, static_cast<char*>(dst) + f * D.S.hb[pout], pin,
                                static_cast<const char*>(src) + f * D.S.hb[pin], D.S.s);
    if (st != TM_OK) return st;
  }
  return TM_OK;
}
static tm_status daccumulate(const DSolver& D, void* X, void* xs) {
  for (int f = 0; f < 2; ++f) {
    tm_status st = launch_accumulate(D.S, static_cast<char*>(X) + f * D.S.hb[TM_F64],
                                     static_cast<char*>(xs) + f * D.S.hb[TM_F32]);
    if (st != TM_OK) return st;
  }
  return TM_OK;
}

static bool dverbose() {
  const char* e = getenv("TM_VERBOSE");
  return e && *e && *e != '0';
}

// CG on Qhat_h^2 y = bp (FP64 or reliable-update mixed precision); y starts at 0.
// On return *xo_in_W says whether W holds Qhat_h Y of the final Y (left by the last FP64
// residual, which forms it first): then it is x_o and the caller need not recompute it.
// With `guess` Y holds a starting point (its FP64 residual is computed first).  With `defer`
// (mixed mode) a sloppy stage that reaches the tolerance ends the call with *pending set and Y
// accumulated but not confirmed in FP64: the caller confirms it through the reconstruction.
static tm_status dcg(const DSolver& D, const tm_cg_params& P, const void* bp, double bb, void* Y, void* R, void* Pv,
                     void* T, void* W, int* iters_out, int* updates_out, bool* conv_out, double* rr_out,
                     bool* xo_in_W, bool guess = false, bool defer = false, bool* pending = nullptr) {
  tm_lattice lat = D.S.lat;
  cudaStream_t s = D.S.s;
  const size_t hb64 = 2 * D.S.hb[TM_F64];
  tm_status st;
  const double stop2 = P.tol * P.tol * bb;
  int iters = 0, updates = 0, bad = 0;
  bool converged = false, w_valid = false;
  double rr_true = bb;
  if (pending) *pending = false;
  if (guess) {
    if ((st = dtrue_residual(D, R, Y, bp, T, W, &rr_true)) != TM_OK) return st;
    w_valid = true;
    ++updates;
    converged = rr_true < stop2;
    if (converged || !(rr_true < 1e300)) {
      *iters_out = 0;
      *updates_out = updates;
      *conv_out = converged;
      *rr_out = rr_true;
      *xo_in_W = true;
      return converged ? TM_OK : set_error(TM_ERR_NONFINITE, "tm_solve_doublet: residual diverged");
    }
  } else {
    if ((st = cuda_check(cudaMemsetAsync(Y, 0, hb64, s), "memset")) != TM_OK) return st;
    if ((st = cuda_check(cudaMemcpyAsync(R, bp, hb64, cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK) return st;
  }
  if (P.mode == TM_CG_FP64) {
    if ((st = cuda_check(cudaMemcpyAsync(Pv, R, hb64, cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK) return st;
    DVecs v{TM_F64, 18, Y, R, Pv, T, W};
    double rr = rr_true;
    while (!converged) {
      CGState fin;
      if ((st = run_dstage(D, v, fresh_state(rr, stop2, P.max_iter, iters, 0.0), &fin)) != TM_OK) return st;
      w_valid = false;  // the stage updates Y in place
      if (fin.nonfinite) return set_error(TM_ERR_NONFINITE, "tm_solve_doublet: non-finite value in the iteration");
      const bool progress = fin.iter > iters;
      iters = fin.iter;
      if ((st = dtrue_residual(D, R, Y, bp, T, W, &rr_true)) != TM_OK) return st;
      w_valid = true;
      ++updates;
      if (dverbose())
        fprintf(stderr, "[tm_solve_doublet] fp64 stage: iter %d true |r|/|b| %.3e\n", iters, std::sqrt(rr_true / bb));
      if (rr_true < stop2) {
        converged = true;
        break;
      }
      if (iters >= P.max_iter || !fin.converged || !progress) break;
      if ((st = cuda_check(cudaMemcpyAsync(Pv, R, hb64, cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK) return st;
      rr = rr_true;
    }
  } else {
    const int sp = P.sloppy_prec;  // TM_F32 (checked by the caller)
    const size_t hs = 2 * D.S.hb[sp], h32 = 2 * D.S.hb[TM_F32];
    void *rs = workspace(lat, 8, h32, &st), *xs = nullptr, *ps = nullptr, *Ts = nullptr, *Ws = nullptr;
    if (st == TM_OK) xs = workspace(lat, 9, h32, &st);
    if (st == TM_OK) ps = workspace(lat, 10, hs, &st);
    if (st == TM_OK) Ts = workspace(lat, 11, hs, &st);
    if (st == TM_OK) Ws = workspace(lat, 12, hs, &st);
    if (st != TM_OK) return st;
    DVecs v{sp, P.sloppy_link, xs, rs, ps, Ts, Ws};
    if ((st = cuda_check(cudaMemsetAsync(xs, 0, h32, s), "memset")) != TM_OK) return st;
    if ((st = dconvert(D, TM_F32, rs, TM_F64, R)) != TM_OK) return st;
    if ((st = dconvert(D, sp, ps, TM_F64, R)) != TM_OK) return st;
    const double delta2 = P.delta * P.delta;
    double rr = rr_true;
    while (!converged && iters < P.max_iter) {
      CGState fin;
      if ((st = run_dstage(D, v, fresh_state(rr, stop2, P.max_iter, iters, delta2, SLOPPY_GROWTH), &fin)) != TM_OK)
        return st;
      if (fin.nonfinite) {
        if (++bad > 3) return set_error(TM_ERR_NONFINITE, "tm_solve_doublet: non-finite value in the iteration");
        iters = fin.iter;
        if ((st = cuda_check(cudaMemsetAsync(xs, 0, h32, s), "memset")) != TM_OK) return st;
        fin.diverged = 1;
      } else {
        bad = 0;
        if (fin.iter == iters) break;
        iters = fin.iter;
        if ((st = daccumulate(D, Y, xs)) != TM_OK) return st;
        w_valid = false;
        if (defer && pending && fin.converged) {
          *iters_out = iters;
          *updates_out = updates;
          *conv_out = false;
          *rr_out = fin.rr;
          *xo_in_W = false;
          *pending = true;
          return TM_OK;
        }
      }
      if ((st = dtrue_residual(D, R, Y, bp, T, W, &rr_true)) != TM_OK) return st;
      w_valid = true;
      ++updates;
      if (dverbose())
        fprintf(stderr, "[tm_solve_doublet] sloppy stage: iter %d true |r|/|b| %.3e diverged %d\n", iters,
                std::sqrt(rr_true / bb), fin.diverged);
      if (rr_true < stop2) {
        converged = true;
        break;
      }
      if (!(rr_true < 1e300)) return set_error(TM_ERR_NONFINITE, "tm_solve_doublet: residual diverged");
      if ((st = dconvert(D, TM_F32, rs, TM_F64, R)) != TM_OK) return st;
      if (fin.diverged && (st = dconvert(D, sp, ps, TM_F64, R)) != TM_OK) return st;
      rr = rr_true;
    }
  }
  *iters_out = iters;
  *updates_out = updates;
  *conv_out = converged;
  *rr_out = rr_true;
  *xo_in_W = w_valid;
  return TM_OK;
}

// canonical doublet field (2 x 24 V doubles) <-> per-parity doublet half fields (FP64)
static tm_status dpack(const DSolver& D, void* dst, const double* src, int parity) {
  for (int f = 0; f < 2; ++f) {
    tm_status st = pack_full_parity(D.S.lat, TM_F64, static_cast<char*>(dst) + f * D.S.hb[TM_F64],
                                    src + (size_t)f * D.S.lat->V * 24, parity, 0, D.S.s);
    if (st != TM_OK) return st;
  }
  return TM_OK;
}
static tm_status dunpack(const DSolver& D, double* dst, const void* src, int parity) {
  for (int f = 0; f < 2; ++f) {
    tm_status st = unpack_full_parity(D.S.lat, TM_F64, dst + (size_t)f * D.S.lat->V * 24,
                                      static_cast<const char*>(src) + f * D.S.hb[TM_F64], parity, 0, D.S.s);
    if (st != TM_OK) return st;
  }
  return TM_OK;
}

// (M_h in) on both parities from the half fields ie, io into oe, oo (FP64)
static tm_status dapply_M(const DSolver& D, void* oe, void* oo, const void* ie, const void* io) {
  DCoef m = dcoef_zero();  // D y - kappa H in
  set_D(m.P, D.mb, D.eb, 1.0);
  set_I(m.Q, -D.S.lat->kappa);
  tm_status st = dhop(D, TM_F64, 18, 0, io, ie, oe, m);
  if (st != TM_OK) return st;
  return dhop(D, TM_F64, 18, 1, ie, io, oo, m);
}

static DSolver make_dsolver(tm_lattice lat, double mubar, double epsbar, cudaStream_t s) {
  DSolver D;
  D.S = Solver{lat, s, 1, 0.0, {0, 0, 0, 0}};
  for (int p = 0; p < 4; ++p) D.S.hb[p] = spinor_bytes_per_site(p) * lat->h;
  D.mb = 2.0 * lat->kappa * mubar;
  D.eb = 2.0 * lat->kappa * epsbar;
  return D;
}

static tm_status full_norm2_host(const DSolver& D, const void* half_e, const void* half_o, double* out) {
  double a = 0.0, b = 0.0;
  tm_status st = norm2_n(D.S, TM_F64, 2 * D.S.lat->geom.h, half_e, &a);
  if (st == TM_OK) st = norm2_n(D.S, TM_F64, 2 * D.S.lat->geom.h, half_o, &b);
  *out = a + b;
  return st;
}

// Solves M_h x = b for one canonical doublet field (device pointers).
static tm_status dsolve_one(const DSolver& D, double* x, const double* b, const tm_cg_params& P, tm_cg_info* info) {
  tm_lattice lat = D.S.lat;
  const size_t hb2 = 2 * D.S.hb[TM_F64];
  tm_status st = TM_OK;
  // doublet FP64 half fields: 0 b_e, 1 b_o, 2 b', 3 Y, 4 R, 5 P, 6 T, 7 W, 14 Z
  void* w[9];
  const int slots[9] = {0, 1, 2, 3, 4, 5, 6, 7, 14};
  for (int k = 0; k < 9; ++k) {
    w[k] = workspace(lat, slots[k], hb2, &st);
    if (st != TM_OK) return st;
  }
  void *be = w[0], *bo = w[1], *bp = w[2], *Y = w[3], *R = w[4], *Pv = w[5], *T = w[6], *W = w[7], *Z = w[8];
  const Reduce none{};
  if ((st = dpack(D, be, b, 0)) != TM_OK) return st;
  if ((st = dpack(D, bo, b, 1)) != TM_OK) return st;
  double bfull = 0.0;
  if ((st = full_norm2_host(D, be, bo, &bfull)) != TM_OK) return st;
  if (!std::isfinite(bfull)) return set_error(TM_ERR_NONFINITE, "tm_solve_doublet: the source has non-finite entries");
  info->iters = info->reliable_updates = 0;
  if (bfull == 0.0) {
    info->true_rel_residual = info->schur_rel_residual = 0.0;
    info->status = TM_OK;
    return cuda_check(cudaMemsetAsync(x, 0, 2 * lat->V * 24 * sizeof(double), D.S.s), "memset");
  }
  // b' = G (b_o + kappa H_oe D^-1 b_e)
  DCoef dinv = dcoef_zero();
  set_Dinv(dinv.P, D.mb, D.eb, 1.0);
  if ((st = dsite(D, TM_F64, 0, be, nullptr, T, nullptr, dinv, none)) != TM_OK) return st;
  DCoef prep = dcoef_zero();
  set_I(prep.P, 1.0);
  set_I(prep.Q, lat->kappa);
  prep.swap = 1;
  if ((st = dhop(D, TM_F64, 18, 1, T, bo, bp, prep)) != TM_OK) return st;
  double bb = 0.0;
  if ((st = norm2_n(D.S, TM_F64, 2 * lat->geom.h, bp, &bb)) != TM_OK) return st;
  int iters = 0, updates = 0;
  bool converged = bb == 0.0, xo_in_W = false, pending = false;
  double rr_true = 0.0;
  const double stop2 = P.tol * P.tol * bb;
  const bool defer = P.mode != TM_CG_FP64;
  if (!converged) {
    if ((st = dcg(D, P, bp, bb, Y, R, Pv, T, W, &iters, &updates, &converged, &rr_true, &xo_in_W, false, defer,
                  &pending)) != TM_OK)
      return st;
  } else if ((st = cuda_check(cudaMemsetAsync(Y, 0, hb2, D.S.s), "memset")) != TM_OK) {
    return st;
  }
  // x_o = Qhat_h Y (-> W), x_e = D^-1 (b_e + kappa H_eo x_o) (-> Pv) and the FP64 residual of the
  // full system: its odd part ||(b - M x)_o|| = ||varphi_o - Mhat_h x_o|| = ||b' - Qhat_h^2 Y|| up
  // to the rounding of x_e (G is unitary), so it also confirms a pending sloppy convergence.
  double rfull = 0.0, rodd = 0.0;
  for (;;) {
    if (!xo_in_W) {
      if ((st = dhop(D, TM_F64, 18, 0, Y, nullptr, T, co_dinv_hop(D))) != TM_OK) return st;
      if ((st = dhop(D, TM_F64, 18, 1, T, Y, W, co_schur_g(D))) != TM_OK) return st;
    }
    DCoef rec = dcoef_zero();
    set_Dinv(rec.P, D.mb, D.eb, 1.0);
    set_Dinv(rec.Q, D.mb, D.eb, lat->kappa);
    if ((st = dhop(D, TM_F64, 18, 0, W, be, Pv, rec)) != TM_OK) return st;
    if ((st = dapply_M(D, R, Z, Pv, W)) != TM_OK) return st;  // (M x)_e -> R, (M x)_o -> Z
    DCoef diff = dcoef_zero();  // b - M x
    set_I(diff.P, 1.0);
    set_I(diff.Q, -1.0);
    if ((st = dsite(D, TM_F64, 0, be, R, R, nullptr, diff, none)) != TM_OK) return st;
    if ((st = dsite(D, TM_F64, 0, bo, Z, Z, nullptr, diff, none)) != TM_OK) return st;
    double reven = 0.0;
    if ((st = norm2_n(D.S, TM_F64, 2 * lat->geom.h, R, &reven)) != TM_OK) return st;
    if ((st = norm2_n(D.S, TM_F64, 2 * lat->geom.h, Z, &rodd)) != TM_OK) return st;
    rfull = reven + rodd;
    if (!pending) break;
    ++updates;  // an FP64 residual recomputation
    if (dverbose())
      fprintf(stderr, "[tm_solve_doublet] confirmation: FP64 |(b - M x)_o|/|b'| %.3e (%s)\n", std::sqrt(rodd / bb),
              rodd < stop2 ? "converged" : "not confirmed, continuing");
    if (rodd < stop2) {
      converged = true;
      rr_true = rodd;
      break;
    }
    if (iters >= P.max_iter) {  // report not converged with this residual
      rr_true = rodd;
      break;
    }
    // not confirmed: continue from Y (its FP64 residual first)
    tm_cg_params Q = P;
    Q.max_iter = P.max_iter - iters;
    int it2 = 0, up2 = 0;
    if ((st = dcg(D, Q, bp, bb, Y, R, Pv, T, W, &it2, &up2, &converged, &rr_true, &xo_in_W, true, defer,
                  &pending)) != TM_OK)
      return st;
    iters += it2;
    updates += up2;
  }
  info->iters = iters;
  info->reliable_updates = updates;
  info->schur_rel_residual = bb > 0.0 ? std::sqrt(rr_true / bb) : 0.0;
  info->true_rel_residual = std::sqrt(rfull / bfull);
  if ((st = dunpack(D, x, Pv, 0)) != TM_OK) return st;
  if ((st = dunpack(D, x, W, 1)) != TM_OK) return st;
  info->status = converged ? TM_OK : TM_ERR_NOT_CONVERGED;
  if (!converged)
    return set_error(TM_ERR_NOT_CONVERGED, "tm_solve_doublet: not converged after %d iterations (%.3e)", iters,
                     info->schur_rel_residual);
  return TM_OK;
}

static tm_status check_doublet_params(tm_lattice lat, double mubar, double epsbar, const char* nm) {
  if (!std::isfinite(mubar) || !std::isfinite(epsbar)) return set_error(TM_ERR_ARG, "%s: mubar, epsbar must be finite", nm);
  const double mb = 2.0 * lat->kappa * mubar, eb = 2.0 * lat->kappa * epsbar;
  if (!(1.0 + mb * mb - eb * eb > 0.0))
    return set_error(TM_ERR_ARG, "%s: the site term is singular (1 + (2 kappa mubar)^2 - (2 kappa epsbar)^2 <= 0)", nm);
  return TM_OK;
}

}  // namespace tmq

using namespace tmq;

extern "C" tm_status tm_apply_Dh(tm_lattice lat, double* out, const double* in, double mubar, double epsbar,
                                 int nrhs, void* stream) {
  if (!lat || !out || !in || nrhs < 1) return set_error(TM_ERR_ARG, "tm_apply_Dh: bad argument");
  if (!lat->has_gauge) return set_error(TM_ERR_NO_GAUGE, "tm_apply_Dh: no gauge field");
  if (out == in) return set_error(TM_ERR_ARG, "tm_apply_Dh: out and in must differ");
  tm_status st = check_doublet_params(lat, mubar, epsbar, "tm_apply_Dh");
  if (st != TM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t fbytes = 2 * lat->V * 24 * sizeof(double);
  const double* din = static_cast<const double*>(stage_in(lat, WS_STAGE_IN, in, fbytes * nrhs, s, &st));
  if (st != TM_OK) return st;
  double* dout = static_cast<double*>(stage_out(lat, WS_STAGE_OUT, out, fbytes * nrhs, &st));
  if (st != TM_OK) return st;
  const DSolver D = make_dsolver(lat, mubar, epsbar, s);
  const size_t hb2 = 2 * D.S.hb[TM_F64];
  void* w[4];
  for (int k = 0; k < 4; ++k) {
    w[k] = workspace(lat, WS_APPLY_D + k, hb2, &st);
    if (st != TM_OK) return st;
  }
  for (int r = 0; r < nrhs; ++r) {
    const double* ir = din + (size_t)r * 2 * lat->V * 24;
    double* orr = dout + (size_t)r * 2 * lat->V * 24;
    if ((st = dpack(D, w[0], ir, 0)) != TM_OK) return st;
    if ((st = dpack(D, w[1], ir, 1)) != TM_OK) return st;
    if ((st = dapply_M(D, w[2], w[3], w[0], w[1])) != TM_OK) return st;
    if ((st = dunpack(D, orr, w[2], 0)) != TM_OK) return st;
    if ((st = dunpack(D, orr, w[3], 1)) != TM_OK) return st;
  }
  if (dout != out) return stage_out_finish(out, dout, fbytes * nrhs, s);
  return TM_OK;
}

extern "C" tm_status tm_solve_doublet(tm_lattice lat, double* x, const double* b, double mubar, double epsbar,
                                      const tm_cg_params* params, tm_cg_info* info, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!lat || !x || !b) return set_error(TM_ERR_ARG, "tm_solve_doublet: bad argument");
  if (!lat->has_gauge) return set_error(TM_ERR_NO_GAUGE, "tm_solve_doublet: no gauge field");
  if (x == b) return set_error(TM_ERR_ARG, "tm_solve_doublet: x and b must differ");
  tm_status st = check_doublet_params(lat, mubar, epsbar, "tm_solve_doublet");
  if (st != TM_OK) return st;
  tm_cg_params P;
  if (params)
    P = *params;
  else
    tm_cg_params_default(&P);
  if (!(P.tol > 0.0) || P.max_iter < 1) return set_error(TM_ERR_ARG, "tm_solve_doublet: tol > 0 and max_iter >= 1");
  if (P.mode != TM_CG_FP64 && P.mode != TM_CG_RELIABLE)
    return set_error(TM_ERR_UNSUPPORTED, "tm_solve_doublet: modes TM_CG_FP64 and TM_CG_RELIABLE only");
  if (P.mode == TM_CG_RELIABLE) {
    if (P.sloppy_prec != TM_F32)
      return set_error(TM_ERR_UNSUPPORTED, "tm_solve_doublet: sloppy storage TM_F32 only");
    if (P.sloppy_link != 18 && P.sloppy_link != 12 && P.sloppy_link != 8)
      return set_error(TM_ERR_ARG, "tm_solve_doublet: sloppy link format %d", P.sloppy_link);
    if (!(P.delta > 0.0 && P.delta < 1.0)) return set_error(TM_ERR_ARG, "tm_solve_doublet: delta must be in (0, 1)");
  }
  if (P.use_x0) return set_error(TM_ERR_UNSUPPORTED, "tm_solve_doublet: no initial guess");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t fbytes = 2 * lat->V * 24 * sizeof(double);
  const double* db = static_cast<const double*>(stage_in(lat, WS_STAGE_IN, b, fbytes, s, &st));
  if (st != TM_OK) return st;
  double* dx = static_cast<double*>(stage_out(lat, WS_STAGE_OUT, x, fbytes, &st));
  if (st != TM_OK) return st;
  const DSolver D = make_dsolver(lat, mubar, epsbar, s);
  tm_cg_info one{};
  st = dsolve_one(D, dx, db, P, &one);
  if (st != TM_OK && st != TM_ERR_NOT_CONVERGED) return st;
  tm_status result = st;
  if (dx != x && (st = stage_out_finish(x, dx, fbytes, s)) != TM_OK) return st;
  if ((st = cuda_check(cudaStreamSynchronize(s), "tm_solve_doublet: synchronise")) != TM_OK) return st;
  one.status = result;
  one.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = one;
  return result;
}
