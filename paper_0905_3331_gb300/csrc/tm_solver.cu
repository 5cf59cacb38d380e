// tm_solver.cu -- even/odd-preconditioned CG (App. B.2, eq. eo6) on the device.
//
// System:  M^f x = b.  Source preparation varphi_o = b_o - M_oe (M_ee^f)^{-1} b_e, then CG on
// the Hermitian positive-definite normal operator A = Qhat^f Qhat^{-f} (eq. eo6) with right-
// hand side b' = gamma5 varphi_o; x_o = Qhat^{-f} X, x_e = (M_ee^f)^{-1}(b_e - M_eo x_o).
//
// One CG iteration is five kernels, all on the caller's stream, none of them waiting for the
// host: the scalars alpha, beta and ||r||^2 live in a device-side CGState written by the last
// block of the kernel that completes each reduction (deterministic, fixed summation order):
//   K1  T = (M_ee^{-f})^{-1} H_eo p
//   K2  W = Qhat^{-f} p = gamma5 [(1 - i f mu~ gamma5) p - kappa^2 H_oe T],  sum ||W||^2 = <p, A p>,
//       alpha = ||r||^2 / <p, A p>
//   K3  T = (M_ee^{f})^{-1} H_eo W
//   K4  r -= alpha Qhat^f W  (= alpha A p, never stored),  sum ||r||^2, beta, convergence test
//   U   x += alpha p,  p = r + beta p
// Kernels K1..K4 return at once when the state says "done"; U applies each iteration once.
// The host enqueues chunks of iterations and checks the state of the previous chunk while the
// next one runs, so the device does not wait for the host between chunks.
//
// Mixed precision: the sloppy operator stores p, T, W in FP32 or FP16 (+ per-site norm) with
// 12- or 8-real links and FP32 arithmetic; r and the solution increment are FP32; every
// reduction is FP64.  Reliable updates (TM_CG_RELIABLE): whenever the iterated ||r|| falls by
// the factor delta since the last update, the increment is added to the FP64 solution X and
// the FP64 residual b' - A X is recomputed with the FP64 operator and replaces r.  The
// TM_CG_SQRT_EPS mode follows Sec. 4.4: FP64 until ||r|| / ||b'|| < sqrt(tol), then the sloppy
// operator; the FP64 recomputation at the end (and further reliable updates if needed)
// guarantees the requested true residual.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "tm_internal.cuh"
#include "tm_solver.cuh"

namespace tmq {

constexpr int CHUNK = 8;  // CG iterations enqueued per host check

unsigned blas_blocks(int h) {
  int nb = (h + BNT - 1) / BNT;
  return (unsigned)(nb < 152 * 8 ? nb : 152 * 8);
}

// ------------------------------------------------------------- BLAS kernels ---
// x += alpha p ; p = r + beta p, once per CG iteration (see `applied`).
// Inside a graph loop (use_cond) the kernel also decides whether the loop runs again: the
// last block continues it only while the state is not done and the loop count is below its
// cap; when there is nothing to apply the state is done and block 0 ends the loop.
template <int PX, int PP, int PR>
__global__ void __launch_bounds__(BNT) cg_update_kernel(int h, char* x, char* p, const char* r, CGState* st,
                                                        unsigned* counter, cudaGraphConditionalHandle cond,
                                                        int use_cond) {
  pdl_wait();
  pdl_allow();
  CGState& S = st[0];
  const int iter = S.iter;
  if (iter == S.applied) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) {
      S.loops += 1;
      cudaGraphSetConditional(cond, 0u);
    }
    return;
  }
  const double alpha = S.alpha, beta = S.beta;
  typedef typename SpinorFmt<PX>::real RX;
  typedef typename SpinorFmt<PP>::real RP;
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    cpx<RX> xv[12];
    cpx<RP> pv[12], rv[12];
    SpinorFmt<PX>::load(x, h, i, xv);
    SpinorFmt<PP>::load(p, h, i, pv);
    SpinorFmt<PR>::load(r, h, i, rv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      xv[k] = xv[k] + (RX)alpha * mk<RX>((RX)pv[k].re, (RX)pv[k].im);
      pv[k] = rv[k] + (RP)beta * pv[k];
    }
    SpinorFmt<PX>::store(x, h, i, xv);
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

template <int P>
__global__ void __launch_bounds__(BNT) norm2_kernel(int h, const char* x, Reduce red) {
  __shared__ double sh[BNT / 32];
  typedef typename SpinorFmt<P>::real R;
  typedef typename SiteSum<R>::type SR;
  double v = 0.0;
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    cpx<R> s[12];
    SpinorFmt<P>::load(x, h, i, s);
    SR site = SR(0);
#pragma unroll
    for (int k = 0; k < 12; ++k) site += (SR)norm2(s[k]);
    v += (double)site;
  }
  const double bs = block_sum<BNT>(v, sh);
  grid_reduce<BNT>(red, 0, gridDim.x, blockIdx.x, bs, sh);
}

// X (FP64) += xs (precision PL); xs = 0
template <int PL>
__global__ void __launch_bounds__(BNT) accumulate_kernel(int h, char* X, char* xs) {
  typedef typename SpinorFmt<PL>::real RL;
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    cpx<double> a[12];
    cpx<RL> b[12];
    SpinorFmt<TM_F64>::load(X, h, i, a);
    SpinorFmt<PL>::load(xs, h, i, b);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      a[k] = a[k] + mk<double>((double)b[k].re, (double)b[k].im);
      b[k] = mk<RL>(RL(0), RL(0));
    }
    SpinorFmt<TM_F64>::store(X, h, i, a);
    SpinorFmt<PL>::store(xs, h, i, b);
  }
}

// y = a x + b y on canonical full fields (n doubles)
__global__ void axpby_kernel(size_t n, double a, const double* x, double b, double* y) {
  for (size_t i = (size_t)blockIdx.x * BNT + threadIdx.x; i < n; i += (size_t)gridDim.x * BNT) y[i] = a * x[i] + b * y[i];
}

// sum of squares of n doubles
__global__ void __launch_bounds__(BNT) full_norm2_kernel(size_t n, const double* x, Reduce red) {
  __shared__ double sh[BNT / 32];
  double v = 0.0;
  for (size_t i = (size_t)blockIdx.x * BNT + threadIdx.x; i < n; i += (size_t)gridDim.x * BNT) v += x[i] * x[i];
  const double bs = block_sum<BNT>(v, sh);
  grid_reduce<BNT>(red, 0, gridDim.x, blockIdx.x, bs, sh);
}

// ------------------------------------------------------------ host helpers ---
static tm_status full_norm2(tm_lattice lat, const double* x, double* out, cudaStream_t s) {
  const size_t n = lat->V * 24;
  const unsigned nb = (unsigned)std::min<size_t>((n + BNT - 1) / BNT, 152 * 8);
  tm_status st = ensure_reduce(lat, nb, 4);
  if (st != TM_OK) return st;
  Reduce red{lat->partials, lat->counters, lat->dscalars, nullptr, FIN_STORE};
  full_norm2_kernel<<<nb, BNT, 0, s>>>(n, x, red);
  count_launch();
  if ((st = cuda_check(cudaMemcpyAsync(out, lat->dscalars, sizeof(double), cudaMemcpyDeviceToHost, s), "readback")) !=
      TM_OK)
    return st;
  return cuda_check(cudaStreamSynchronize(s), "synchronise");
}


tm_status norm2_half(const Solver& S, int prec, const void* x, double* out_host) {
  return norm2_n(S, prec, S.lat->geom.h, x, out_host);
}

tm_status norm2_n(const Solver& S, int prec, int n, const void* x, double* out_host) {
  tm_lattice lat = S.lat;
  const unsigned nb = blas_blocks(n);
  tm_status st = ensure_reduce(lat, nb, 4);
  if (st != TM_OK) return st;
  Reduce red{lat->partials, lat->counters, lat->dscalars, nullptr, FIN_STORE};
  const char* xp = static_cast<const char*>(x);
  if (prec == TM_F64)
    norm2_kernel<TM_F64><<<nb, BNT, 0, S.s>>>(n, xp, red);
  else if (prec == TM_F32)
    norm2_kernel<TM_F32><<<nb, BNT, 0, S.s>>>(n, xp, red);
  else if (prec == TM_DF64)
    norm2_kernel<TM_DF64><<<nb, BNT, 0, S.s>>>(n, xp, red);
  else
    norm2_kernel<TM_F16><<<nb, BNT, 0, S.s>>>(n, xp, red);
  count_launch();
  if ((st = cuda_check(cudaGetLastError(), "norm kernel")) != TM_OK) return st;
  if ((st = cuda_check(cudaMemcpyAsync(out_host, lat->dscalars, sizeof(double), cudaMemcpyDeviceToHost, S.s),
                       "readback")) != TM_OK)
    return st;
  return cuda_check(cudaStreamSynchronize(S.s), "synchronise");
}

// A = Qhat^f Qhat^{-f} applied to `in` (precision prec, links nreal), result folded into
// `r` as r -= alpha A in.  With `state` the iteration form is used (skip when done, alpha from
// the state, FIN_CG_ALPHA / FIN_CG_RR); without it alpha = 1 and ||r||^2 goes to dscalars[0].
tm_status normal_apply(const Solver& S, int prec, int nreal, const void* in, void* T, void* W, void* r,
                       CGState* state) {
  tm_lattice lat = S.lat;
  const unsigned nb = hop_grid_blocks(lat->h, 4);  // enough for every threads-per-site choice
  tm_status st = ensure_reduce(lat, nb, 4);
  if (st != TM_OK) return st;
  HopArgs a{};
  a.prec = prec;
  a.nreal = nreal;
  a.nrhs = 1;
  a.skip = state ? &state->done : nullptr;
  // K1: T = (M_ee^{-f})^-1 H_eo in
  a.out_parity = 0;
  a.in = in;
  a.out = T;
  a.coef = epi_mdiag_inv_hop(S.mut, -S.f);
  a.mode = 0;
  if ((st = hop_launch(lat, a, S.s)) != TM_OK) return st;
  // K2: W = Qhat^{-f} in, <in, A in> = ||W||^2
  a.out_parity = 1;
  a.in = T;
  a.y = in;
  a.out = W;
  a.coef = epi_schur_q(lat->kappa, S.mut, -S.f);
  if (state) {
    a.mode = 1;
    a.red = Reduce{lat->partials, lat->counters, nullptr, state, FIN_CG_ALPHA, lat->gcounters};
  } else {
    a.mode = 0;
  }
  if ((st = hop_launch(lat, a, S.s)) != TM_OK) return st;
  // K3: T = (M_ee^{f})^-1 H_eo W
  a.out_parity = 0;
  a.in = W;
  a.y = nullptr;
  a.out = T;
  a.coef = epi_mdiag_inv_hop(S.mut, S.f);
  a.mode = 0;
  if ((st = hop_launch(lat, a, S.s)) != TM_OK) return st;
  // K4: r -= alpha Qhat^f W
  a.out_parity = 1;
  a.in = T;
  a.y = W;
  a.out = r;
  a.coef = epi_schur_q(lat->kappa, S.mut, S.f);
  a.mode = 2;
  if (state) {
    a.alpha_src = state;
    a.alpha_sign = 1.0;
    a.red = Reduce{lat->partials, lat->counters, nullptr, state, FIN_CG_RR, lat->gcounters};
  } else {
    a.alpha_src = nullptr;
    a.alpha_sign = 1.0;
    a.red = Reduce{lat->partials, lat->counters, lat->dscalars, nullptr, FIN_STORE, lat->gcounters};
  }
  return hop_launch(lat, a, S.s);
}

tm_status launch_update_n(const Solver& S, int n, int px, int pp, void* x, void* p, const void* r, CGState* state,
                          cudaGraphConditionalHandle cond, int use_cond) {
  tm_lattice lat = S.lat;
  const unsigned nb = blas_blocks(n);
  char* xc = static_cast<char*>(x);
  char* pc = static_cast<char*>(p);
  const char* rc = static_cast<const char*>(r);
  unsigned* ctr = lat->counters + 2;
  if (px == TM_F64)
    launch_pdl(cg_update_kernel<TM_F64, TM_F64, TM_F64>, dim3(nb), dim3(BNT), S.s, n, xc, pc, rc, state, ctr, cond, use_cond);
  else if (pp == TM_F32)
    launch_pdl(cg_update_kernel<TM_F32, TM_F32, TM_F32>, dim3(nb), dim3(BNT), S.s, n, xc, pc, rc, state, ctr, cond, use_cond);
  else
    launch_pdl(cg_update_kernel<TM_F32, TM_F16, TM_F32>, dim3(nb), dim3(BNT), S.s, n, xc, pc, rc, state, ctr, cond, use_cond);
  count_launch();
  return cuda_check(cudaGetLastError(), "CG update kernel");
}

static tm_status launch_update(const Solver& S, int px, int pp, void* x, void* p, const void* r, CGState* state,
                               cudaGraphConditionalHandle cond = 0, int use_cond = 0) {
  return launch_update_n(S, S.lat->geom.h, px, pp, x, p, r, state, cond, use_cond);
}

// The vectors of one CG stage: x (PX), r (ResidPrec of op), p / T / W (op precision).
struct Stage {
  int prec;   // operator storage precision
  int nreal;  // link format
  int px;     // precision of x
  void *x, *r, *p, *T, *W;
};

static tm_status enqueue_iterations(const Solver& S, const Stage& v, CGState* dst, int n) {
  tm_status st = TM_OK;
  for (int k = 0; k < n && st == TM_OK; ++k) {
    st = normal_apply(S, v.prec, v.nreal, v.p, v.T, v.W, v.r, dst);
    if (st == TM_OK) st = launch_update(S, v.px, v.prec, v.x, v.p, v.r, dst);
  }
  return st;
}

bool use_graphs() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("TM_NO_GRAPH");
    v = (e && *e && *e != '0') ? 0 : 1;
  }
  return v == 1;
}

// Iterations per body of a solver graph's WHILE loop (TM_CG_UNROLL, 1..8, default 4).
// Iterations after the stage is done within a body cost only empty launches (every kernel
// skips on `done`, the update on iter == applied).  Measured on the 16^3 x 32 mixed CG solve:
// each relaunch of the loop body costs ~4 us; 4 iterations per body gave 143 solves/s
// against 138 with one.
int cg_unroll() {
  static int v = 0;
  if (v == 0) {
    const char* e = getenv("TM_CG_UNROLL");
    int u = e && *e ? atoi(e) : 0;
    v = u < 0 ? 0 : (u > 8 ? 8 : u);
    if (v == 0) v = -1;  // not set: by lattice size (cg_unroll_for)
  }
  return v > 0 ? v : 4;
}

// The same for one lattice: without TM_CG_UNROLL, one iteration per body from a million sites
// per parity on.  There an empty launch still schedules every block (~80 us for the 83 000 blocks
// of 48^3 x 96 against ~4 us per relaunch of the body), and up to three per stage would be lost
// to the four-iteration body.
int cg_unroll_for(size_t h) {
  const char* e = getenv("TM_CG_UNROLL");
  if (e && *e) return cg_unroll();
  return h >= ((size_t)1 << 20) ? 1 : 4;
}

// The CUDA graph of one CG stage: a WHILE conditional node whose body is cg_unroll()
// iterations (K1..K4 and the update, which sets the loop condition from the device-side
// state).  Graphs are cached per lattice and stage (vectors, precision, flavour, kappa, mu).
static tm_status stage_graph(const Solver& S, const Stage& v, cudaGraphExec_t* out) {
  tm_lattice lat = S.lat;
  for (int k = 0; k < 8; ++k) {
    const auto& e = lat->graphs[k];
    if (e.valid && e.prec == v.prec && e.nreal == v.nreal && e.px == v.px && e.f == S.f && e.x == v.x &&
        e.r == v.r && e.p == v.p && e.T == v.T && e.W == v.W && e.kappa == lat->kappa && e.mu == lat->mu) {
      *out = e.exec;
      return TM_OK;
    }
  }
  tm_status st = ensure_links(lat, v.prec, v.nreal, S.s);
  if (st != TM_OK) return st;
  if ((st = cuda_check(cudaStreamSynchronize(S.s), "synchronise")) != TM_OK) return st;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaStream_t cs = nullptr;
  cudaGraphConditionalHandle cond;
  cudaGraphNode_t node;
  cudaGraphNodeParams cp = {};
  const unsigned long long before = tm_launch_count();
  if ((st = cuda_check(cudaGraphCreate(&g, 0), "cudaGraphCreate")) != TM_OK) return st;
  st = cuda_check(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault), "conditional handle");
  if (st == TM_OK) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    st = cuda_check(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp), "conditional node");
  }
  if (st == TM_OK) st = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
  if (st == TM_OK) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    st = cuda_check(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                    "begin capture");
    if (st == TM_OK) {
      Solver C = S;
      C.s = cs;
      tm_status st1 = TM_OK;
      for (int u = 0; u < cg_unroll_for(lat->h) && st1 == TM_OK; ++u) {
        st1 = normal_apply(C, v.prec, v.nreal, v.p, v.T, v.W, v.r, lat->cgstate);
        if (st1 == TM_OK) st1 = launch_update(C, v.px, v.prec, v.x, v.p, v.r, lat->cgstate, cond, 1);
      }
      cudaGraph_t captured = nullptr;
      tm_status st2 = cuda_check(cudaStreamEndCapture(cs, &captured), "end capture");
      st = st1 != TM_OK ? st1 : st2;
    }
  }
  if (st == TM_OK) st = cuda_check(cudaGraphInstantiate(&ex, g, 0), "graph instantiate");
  if (cs) cudaStreamDestroy(cs);
  tm_reset_launch_count();
  count_launch((unsigned)before);  // capture enqueues nothing; keep the launch count unchanged
  if (st != TM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  auto& e = lat->graphs[lat->graph_next];
  if (e.valid) {
    cudaGraphExecDestroy(e.exec);
    cudaGraphDestroy(e.graph);
  }
  e.valid = true;
  e.prec = v.prec;
  e.nreal = v.nreal;
  e.px = v.px;
  e.f = S.f;
  e.x = v.x;
  e.r = v.r;
  e.p = v.p;
  e.T = v.T;
  e.W = v.W;
  e.kappa = lat->kappa;
  e.mu = lat->mu;
  e.graph = g;
  e.exec = ex;
  lat->graph_next = (lat->graph_next + 1) % 8;
  *out = ex;
  return TM_OK;
}

tm_status aux_loop_graph(tm_lattice lat, const unsigned long long key[16], cudaStream_t s, const LoopBody& body,
                         cudaGraphExec_t* out) {
  for (int k = 0; k < 8; ++k) {
    const auto& e = lat->aux_graphs[k];
    if (e.valid && memcmp(e.key, key, 16 * sizeof(unsigned long long)) == 0) {
      *out = e.exec;
      return TM_OK;
    }
  }
  tm_status st = cuda_check(cudaStreamSynchronize(s), "synchronise");
  if (st != TM_OK) return st;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaStream_t cs = nullptr;
  cudaGraphConditionalHandle cond;
  cudaGraphNode_t node;
  cudaGraphNodeParams cp = {};
  const unsigned long long before = tm_launch_count();
  if ((st = cuda_check(cudaGraphCreate(&g, 0), "cudaGraphCreate")) != TM_OK) return st;
  st = cuda_check(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault), "conditional handle");
  if (st == TM_OK) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    st = cuda_check(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp), "conditional node");
  }
  if (st == TM_OK) st = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
  if (st == TM_OK) {
    cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
    st = cuda_check(cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                    "begin capture");
    if (st == TM_OK) {
      tm_status st1 = TM_OK;
      for (int u = 0; u < cg_unroll() && st1 == TM_OK; ++u) st1 = body(cs, cond);
      cudaGraph_t captured = nullptr;
      tm_status st2 = cuda_check(cudaStreamEndCapture(cs, &captured), "end capture");
      st = st1 != TM_OK ? st1 : st2;
    }
  }
  if (st == TM_OK) st = cuda_check(cudaGraphInstantiate(&ex, g, 0), "graph instantiate");
  if (cs) cudaStreamDestroy(cs);
  tm_reset_launch_count();
  count_launch((unsigned)before);  // capture enqueues nothing; keep the launch count unchanged
  if (st != TM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  auto& e = lat->aux_graphs[lat->aux_next];
  if (e.valid) {
    cudaGraphExecDestroy(e.exec);
    cudaGraphDestroy(e.graph);
  }
  e.valid = true;
  memcpy(e.key, key, 16 * sizeof(unsigned long long));
  e.graph = g;
  e.exec = ex;
  lat->aux_next = (lat->aux_next + 1) % 8;
  *out = ex;
  return TM_OK;
}

// Graph form of a stage: upload the state, launch the loop graph once, read the state back.
static tm_status run_stage_graph(const Solver& S, const Stage& v, const CGState& init, CGState* out) {
  tm_lattice lat = S.lat;
  tm_status st = ensure_cgstate(lat, 2);
  if (st != TM_OK) return st;
  cudaGraphExec_t ex;
  if ((st = stage_graph(S, v, &ex)) != TM_OK) return st;
  CGState* hst = lat->cgstate_host;
  hst[0] = init;
  hst[0].loops = 0;
  hst[0].loop_cap = (init.max_iter - init.iter) + 2;
  if ((st = cuda_check(cudaMemcpyAsync(lat->cgstate, &hst[0], sizeof(CGState), cudaMemcpyHostToDevice, S.s),
                       "state")) != TM_OK)
    return st;
  if ((st = cuda_check(cudaGraphLaunch(ex, S.s), "graph launch")) != TM_OK) return st;
  if ((st = cuda_check(cudaMemcpyAsync(&hst[1], lat->cgstate, sizeof(CGState), cudaMemcpyDeviceToHost, S.s),
                       "state")) != TM_OK)
    return st;
  if ((st = cuda_check(cudaStreamSynchronize(S.s), "CG stage")) != TM_OK) return st;
  *out = hst[1];
  count_launch(5u * (unsigned)hst[1].loops);
  if (!(hst[1].done)) return set_error(TM_ERR_TIMEOUT, "tm_solve_cg: stage loop reached its bound without finishing");
  return TM_OK;
}

// Runs CG iterations from `init` until the device state says done (and the last update has
// been applied).  Graph form by default (TM_NO_GRAPH=1 selects the host loop below).  Host
// loop: two chunks are in flight, the host reads the state after chunk k while chunk k + 1
// runs; chunks after the end cost only empty launches.
static tm_status run_stage(const Solver& S, const Stage& v, const CGState& init, CGState* out) {
  if (use_graphs()) return run_stage_graph(S, v, init, out);
  tm_lattice lat = S.lat;
  tm_status st = ensure_cgstate(lat, 2);
  if (st != TM_OK) return st;
  CGState* dst = lat->cgstate;
  CGState* hst = lat->cgstate_host;
  hst[0] = init;
  if ((st = cuda_check(cudaMemcpyAsync(dst, &hst[0], sizeof(CGState), cudaMemcpyHostToDevice, S.s), "state"))
      != TM_OK)
    return st;
  if ((st = cuda_check(cudaStreamSynchronize(S.s), "state upload")) != TM_OK) return st;
  cudaEvent_t ev[2];
  cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
  int cur = 0;
  st = enqueue_iterations(S, v, dst, CHUNK);
  if (st == TM_OK) st = cuda_check(cudaMemcpyAsync(&hst[cur], dst, sizeof(CGState), cudaMemcpyDeviceToHost, S.s), "state");
  if (st == TM_OK) st = cuda_check(cudaEventRecord(ev[cur], S.s), "event");
  while (st == TM_OK) {
    const int nxt = cur ^ 1;
    st = enqueue_iterations(S, v, dst, CHUNK);
    if (st == TM_OK)
      st = cuda_check(cudaMemcpyAsync(&hst[nxt], dst, sizeof(CGState), cudaMemcpyDeviceToHost, S.s), "state");
    if (st == TM_OK) st = cuda_check(cudaEventRecord(ev[nxt], S.s), "event");
    if (st == TM_OK) st = cuda_check(cudaEventSynchronize(ev[cur]), "CG chunk");
    if (st != TM_OK) break;
    const CGState c = hst[cur];
    if (c.done && c.applied == c.iter) {
      st = cuda_check(cudaEventSynchronize(ev[nxt]), "CG chunk");
      *out = hst[nxt];
      break;
    }
    cur = nxt;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  return st;
}

// r = b' - A X in FP64 (r, X, b' FP64 odd fields; T, W FP64 temporaries); returns ||r||^2.
tm_status true_residual(const Solver& S, void* r, const void* X, const void* bp, void* T, void* W,
                               double* rr) {
  tm_status st = cuda_check(cudaMemcpyAsync(r, bp, S.hb[TM_F64], cudaMemcpyDeviceToDevice, S.s), "copy");
  if (st != TM_OK) return st;
  if ((st = normal_apply(S, TM_F64, 18, X, T, W, r, nullptr)) != TM_OK) return st;
  if ((st = cuda_check(cudaMemcpyAsync(rr, S.lat->dscalars, sizeof(double), cudaMemcpyDeviceToHost, S.s),
                       "readback")) != TM_OK)
    return st;
  return cuda_check(cudaStreamSynchronize(S.s), "synchronise");
}


// The same in double-float: X (FP64) is converted to Xd, r = b' - A Xd with the double-float
// operator (all fields TM_DF64); returns ||r||^2.
static tm_status true_residual_dd(const Solver& S, void* rd, const void* X, const void* bpd, void* Td, void* Wd,
                                  void* Xd, double* rr) {
  tm_status st = convert_half(S.lat, TM_DF64, Xd, TM_F64, X, S.s);
  if (st != TM_OK) return st;
  if ((st = cuda_check(cudaMemcpyAsync(rd, bpd, S.hb[TM_DF64], cudaMemcpyDeviceToDevice, S.s), "copy")) != TM_OK)
    return st;
  if ((st = normal_apply(S, TM_DF64, 18, Xd, Td, Wd, rd, nullptr)) != TM_OK) return st;
  if ((st = cuda_check(cudaMemcpyAsync(rr, S.lat->dscalars, sizeof(double), cudaMemcpyDeviceToHost, S.s),
                       "readback")) != TM_OK)
    return st;
  return cuda_check(cudaStreamSynchronize(S.s), "synchronise");
}

CGState fresh_state(double rr, double stop2, int max_iter, int iter0, double delta2, double growth) {
  CGState c;
  memset(&c, 0, sizeof(c));
  c.rr = rr;
  c.rr_ref = rr;
  c.rr_min = rr;
  c.stop2 = stop2;
  c.max_iter = max_iter;
  c.iter = iter0;
  c.applied = iter0;
  c.delta2 = delta2;
  c.grow2 = growth * growth;
  return c;
}

static bool verbose() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("TM_VERBOSE");
    v = (e && *e && *e != '0') ? 1 : 0;
  }
  return v == 1;
}

static void trace_stage(const char* what, const CGState& c, double bb) {
  if (!verbose()) return;
  fprintf(stderr, "[tm_solve_cg] %s: iter %d  |r|/|b| %.3e  converged %d  update %d  diverged %d  nonfinite %d\n",
          what, c.iter, std::sqrt(c.rr / bb), c.converged, c.want_update, c.diverged, c.nonfinite);
}

static void trace_update(int k, double rr_true, double bb) {
  if (!verbose()) return;
  fprintf(stderr, "[tm_solve_cg] reliable update %d: true |r|/|b| %.3e\n", k, std::sqrt(rr_true / bb));
}

// b' = gamma5 (b_o + kappa H_oe (M_ee^f)^-1 b_e) (App. B.2), with ||b'||^2 and ||b||^2.
tm_status prepare_source(const Solver& S, const double* b, void* be, void* bo, void* bp, void* T, double* bb,
                         double* bfull) {
  tm_lattice lat = S.lat;
  cudaStream_t s = S.s;
  tm_status st;
  if ((st = pack_full_parity(lat, TM_F64, be, b, 0, 0, s)) != TM_OK) return st;
  if ((st = pack_full_parity(lat, TM_F64, bo, b, 1, 0, s)) != TM_OK) return st;
  const double n = 1.0 / (1.0 + S.mut * S.mut);
  if ((st = diag_apply(lat, TM_F64, T, be, 1, n, -S.f * S.mut * n, n, S.f * S.mut * n, s)) != TM_OK) return st;
  // ||b'||^2, ||b_e||^2, ||b_o||^2 into dscalars[0..2], read back with one synchronisation
  const unsigned nb = blas_blocks(lat->geom.h);
  if ((st = ensure_reduce(lat, std::max<size_t>(hop_grid_blocks(lat->h, 4), nb), 4)) != TM_OK) return st;
  HopArgs a{};
  a.prec = TM_F64;
  a.nreal = 18;
  a.nrhs = 1;
  a.out_parity = 1;
  a.in = T;
  a.y = bo;
  a.out = bp;
  a.coef = epi_g5_y_plus(lat->kappa);
  a.mode = 1;
  a.red = Reduce{lat->partials, lat->counters, lat->dscalars, nullptr, FIN_STORE};
  if ((st = hop_launch(lat, a, s)) != TM_OK) return st;
  for (int k = 0; k < 2; ++k) {
    const Reduce red{lat->partials, lat->counters, lat->dscalars + 1 + k, nullptr, FIN_STORE};
    norm2_kernel<TM_F64><<<nb, BNT, 0, s>>>(lat->geom.h, static_cast<const char*>(k ? bo : be), red);
    count_launch();
  }
  if ((st = cuda_check(cudaGetLastError(), "norm kernel")) != TM_OK) return st;
  double* nn = reinterpret_cast<double*>(lat->flag_host);
  if ((st = cuda_check(cudaMemcpyAsync(nn, lat->dscalars, 3 * sizeof(double), cudaMemcpyDeviceToHost, s),
                       "readback")) != TM_OK)
    return st;
  if ((st = cuda_check(cudaStreamSynchronize(s), "synchronise")) != TM_OK) return st;
  *bb = nn[0];
  *bfull = nn[1] + nn[2];
  return TM_OK;
}

// x_o = Qhat^{-f} X, x_e = (M_ee^f)^-1 (b_e + kappa H_eo x_o) (eq. eo6, App. B.2), written to
// the canonical field x; then ||b - M x|| / ||b|| in FP64 (R, Pv, T, W are FP64 scratch).
tm_status reconstruct_check(const Solver& S, const void* X, const void* be, const void* bo, double bfull, double* x,
                            void* T, void* W, void* R, void* Pv, double* true_rel, double* rr_odd) {
  tm_lattice lat = S.lat;
  tm_status st;
  HopArgs a{};
  a.prec = TM_F64;
  a.nreal = 18;
  a.nrhs = 1;
  a.out_parity = 0;
  a.in = X;
  a.out = T;
  a.coef = epi_mdiag_inv_hop(S.mut, -S.f);
  if ((st = hop_launch(lat, a, S.s)) != TM_OK) return st;
  a.out_parity = 1;
  a.in = T;
  a.y = X;
  a.out = W;  // x_o
  a.coef = epi_schur_q(lat->kappa, S.mut, -S.f);
  if ((st = hop_launch(lat, a, S.s)) != TM_OK) return st;
  return reconstruct_xo(S, W, be, bo, bfull, x, T, R, Pv, true_rel, rr_odd);
}

// x_e = (M_ee^f)^-1 (b_e + kappa H_eo x_o) from the odd solution xo, written with xo to the
// canonical field x; then ||b - M x|| / ||b|| in FP64 (T, R, Pv are FP64 scratch).  Two FP64
// hopping launches: the first stores x_e and sums the even residual
// ||b_e + kappa H_eo x_o - M_ee x_e||^2 from the same hopping sum; the second forms
// (b - M x)_o = b_o - (M_oo x_o - kappa H_oe x_e) and its norm.  R is unused.
tm_status reconstruct_xo(const Solver& S, const void* xo, const void* be, const void* bo, double bfull, double* x,
                         void* T, void* R, void* Pv, double* true_rel, double* rr_odd) {
  (void)R;
  tm_lattice lat = S.lat;
  cudaStream_t s = S.s;
  tm_status st = ensure_reduce(lat, hop_grid_blocks(lat->h, 4), 4);
  if (st != TM_OK) return st;
  void* W = const_cast<void*>(xo);
  HopArgs a{};
  a.prec = TM_F64;
  a.nreal = 18;
  a.nrhs = 1;
  a.out_parity = 0;
  a.in = W;
  a.y = be;
  a.out = T;  // x_e
  a.coef = epi_scaled_minv(S.mut, S.f, lat->kappa);
  a.mode = 3;
  a.red = Reduce{lat->partials, lat->counters, lat->dscalars, nullptr, FIN_STORE};
  if ((st = hop_launch(lat, a, s)) != TM_OK) return st;
  if ((st = cuda_check(cudaMemcpyAsync(Pv, bo, S.hb[TM_F64], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK)
    return st;
  a.coef = epi_full_M(lat->kappa, S.mut, S.f);
  a.out_parity = 1;
  a.in = T;
  a.y = W;
  a.out = Pv;
  a.mode = 2;  // Pv -= 1 * (M x)_o
  a.alpha_src = nullptr;
  a.alpha_sign = 1.0;
  a.red = Reduce{lat->partials, lat->counters, lat->dscalars + 1, nullptr, FIN_STORE};
  if ((st = hop_launch(lat, a, s)) != TM_OK) return st;
  double* rr = reinterpret_cast<double*>(lat->flag_host);
  if ((st = cuda_check(cudaMemcpyAsync(rr, lat->dscalars, 2 * sizeof(double), cudaMemcpyDeviceToHost, s),
                       "readback")) != TM_OK)
    return st;
  if ((st = cuda_check(cudaStreamSynchronize(s), "synchronise")) != TM_OK) return st;
  const double rre = rr[0], rro = rr[1];
  *true_rel = bfull > 0.0 ? std::sqrt((rre + rro) / bfull) : 0.0;
  if (rr_odd) *rr_odd = rro;
  if ((st = unpack_full_parity(lat, TM_F64, x, T, 0, 0, s)) != TM_OK) return st;
  return unpack_full_parity(lat, TM_F64, x, W, 1, 0, s);
}

tm_status launch_accumulate(const Solver& S, void* X, void* xs) {
  const unsigned nb = blas_blocks(S.lat->geom.h);
  accumulate_kernel<TM_F32><<<nb, BNT, 0, S.s>>>(S.lat->geom.h, static_cast<char*>(X), static_cast<char*>(xs));
  count_launch();
  return cuda_check(cudaGetLastError(), "accumulate kernel");
}

// CG on A X = bp, A = Qhat^f Qhat^-f on the odd sites (eq. eo6), FP64 or mixed precision per
// P.mode; X holds an initial guess if `guess`, else it starts at 0.  bp, X, R, Pv, T, W are FP64
// half fields (R, Pv, T, W work space); bb = ||bp||^2.  The result is converged when the
// recomputed FP64 residual satisfies ||bp - A X||^2 < tol^2 bb.
tm_status cg_normal(const Solver& S, const tm_cg_params& P, const void* bp, double bb, void* X, bool guess, void* R,
                    void* Pv, void* T, void* W, NormalResult* res, bool defer_final) {
  tm_lattice lat = S.lat;
  cudaStream_t s = S.s;
  tm_status st = TM_OK;
  const double tol2 = P.tol * P.tol;
  const double stop2 = tol2 * bb;
  int iters = 0, updates = 0;
  bool converged = false;
  double rr_true = bb;
  // starting residual R = b' - A X (X = 0 unless a guess is given)
  bool w_valid = false;  // W = Qhat^{-f} X of the current X (K2 of the last FP64 residual)
  if (guess) {
    if ((st = true_residual(S, R, X, bp, T, W, &rr_true)) != TM_OK) return st;
    w_valid = true;
  } else {
    if ((st = cuda_check(cudaMemsetAsync(X, 0, S.hb[TM_F64], s), "memset")) != TM_OK) return st;
    if ((st = cuda_check(cudaMemcpyAsync(R, bp, S.hb[TM_F64], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK)
      return st;
  }
  if (!std::isfinite(rr_true)) return set_error(TM_ERR_NONFINITE, "tm_solve_cg: non-finite initial residual");
  if (rr_true < stop2) converged = true;
  const double rr0 = rr_true;

  if (P.mode == TM_CG_FP64) {
    // ---- plain FP64 CG, restarted from the recomputed residual if the iterated one drifted
    if ((st = cuda_check(cudaMemcpyAsync(Pv, R, S.hb[TM_F64], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK)
      return st;
    Stage v{TM_F64, 18, TM_F64, X, R, Pv, T, W};
    double rr = rr0;
    while (!converged) {
      CGState fin;
      if ((st = run_stage(S, v, fresh_state(rr, stop2, P.max_iter, iters, 0.0), &fin)) != TM_OK) return st;
      w_valid = false;
      trace_stage("fp64 stage", fin, bb);
      if (fin.nonfinite) return set_error(TM_ERR_NONFINITE, "tm_solve_cg: non-finite value in the iteration");
      const bool progress = fin.iter > iters;
      iters = fin.iter;
      if ((st = true_residual(S, R, X, bp, T, W, &rr_true)) != TM_OK) return st;
      w_valid = true;
      ++updates;
      trace_update(updates, rr_true, bb);
      if (rr_true < stop2) {
        converged = true;
        break;
      }
      if (iters >= P.max_iter || !fin.converged || !progress) break;
      // restart: p = r = b' - A X
      if ((st = cuda_check(cudaMemcpyAsync(Pv, R, S.hb[TM_F64], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK)
        return st;
      rr = rr_true;
    }
  } else {
    // ---- mixed precision
    const int sp = P.sloppy_prec, sl = P.sloppy_link;
    void *rs = nullptr, *xs = nullptr, *ps = nullptr, *Ts = nullptr, *Ws = nullptr;
    rs = workspace(lat, 8, S.hb[TM_F32], &st);
    if (st == TM_OK) xs = workspace(lat, 9, S.hb[TM_F32], &st);
    if (st == TM_OK) ps = workspace(lat, 10, S.hb[sp], &st);
    if (st == TM_OK) Ts = workspace(lat, 11, S.hb[sp], &st);
    if (st == TM_OK) Ws = workspace(lat, 12, S.hb[sp], &st);
    if (st != TM_OK) return st;
    Stage v{sp, sl, TM_F32, xs, rs, ps, Ts, Ws};
    if ((st = cuda_check(cudaMemsetAsync(xs, 0, S.hb[TM_F32], s), "memset")) != TM_OK) return st;
    double rr = rr0;
    if (P.mode == TM_CG_SQRT_EPS && !converged) {
      // FP64 until ||r||^2 < tol ||b'||^2 (i.e. ||r|| / ||b'|| < sqrt(tol)), Sec. 4.4
      if ((st = cuda_check(cudaMemcpyAsync(Pv, R, S.hb[TM_F64], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK)
        return st;
      Stage v64{TM_F64, 18, TM_F64, X, R, Pv, T, W};
      CGState fin;
      const double stop_sw = std::fmax(P.tol * bb, stop2);
      if ((st = run_stage(S, v64, fresh_state(rr, stop_sw, P.max_iter, 0, 0.0), &fin)) != TM_OK) return st;
      w_valid = false;
      trace_stage("fp64 stage (to sqrt(tol))", fin, bb);
      iters = fin.iter;
      if (fin.nonfinite) return set_error(TM_ERR_NONFINITE, "tm_solve_cg: non-finite value in the iteration");
      rr = fin.rr;
      // continue with the sloppy operator from the current r and p
      if ((st = convert_half(lat, TM_F32, rs, TM_F64, R, s)) != TM_OK) return st;
      if ((st = convert_half(lat, sp, ps, TM_F64, Pv, s)) != TM_OK) return st;
      // first sloppy stage runs without reliable updates (the paper's switch); only the
      // divergence guard can end it early
      if ((st = run_stage(S, v, fresh_state(rr, stop2, P.max_iter, iters, 0.0, SLOPPY_GROWTH), &fin)) != TM_OK)
        return st;
      trace_stage("sloppy stage", fin, bb);
      iters = fin.iter;
      if (fin.nonfinite) {  // drop the overflowed increment; continue from the FP64 solution
        if ((st = cuda_check(cudaMemsetAsync(xs, 0, S.hb[TM_F32], s), "memset")) != TM_OK) return st;
        fin.diverged = 1;
      } else {
        const unsigned nbb = blas_blocks(lat->geom.h);
        accumulate_kernel<TM_F32><<<nbb, BNT, 0, s>>>(lat->geom.h, static_cast<char*>(X), static_cast<char*>(xs));
        count_launch();
        w_valid = false;
      }
      if ((st = true_residual(S, R, X, bp, T, W, &rr_true)) != TM_OK) return st;
      w_valid = true;
      ++updates;
      trace_update(updates, rr_true, bb);
      converged = rr_true < stop2;
      rr = rr_true;
      if (!converged && iters < P.max_iter) {
        if ((st = convert_half(lat, TM_F32, rs, TM_F64, R, s)) != TM_OK) return st;
        if (fin.diverged && (st = convert_half(lat, sp, ps, TM_F64, R, s)) != TM_OK) return st;
      }
    } else {
      if ((st = convert_half(lat, TM_F32, rs, TM_F64, R, s)) != TM_OK) return st;
      if ((st = convert_half(lat, sp, ps, TM_F64, R, s)) != TM_OK) return st;
    }
    // reliable-update loop (also the defect correction of the sqrt(eps) mode)
    const double delta2 = P.delta * P.delta;
    int bad_stages = 0;
    bool dd_updates = P.update_prec == TM_DF64;
    // FP32 recomputations (update_prec TM_F32): r = r64 - A xs with the FP32 operator, r64 the
    // last FP64 residual and xs the FP32 increment since then; the FP64 recomputation (X += xs)
    // comes once ||r|| has fallen by F32_UPDATE_SPAN since the last one.  The FP32 result is off
    // by about u32 kappa(A) ||r64|| (1e-4 ||r64|| on 48^3 x 96), well inside that span.
    constexpr double F32_UPDATE_SPAN = 1e-2;
    const bool f32_updates = P.update_prec == TM_F32;
    void *rb32 = nullptr, *T32 = nullptr, *W32 = nullptr;
    double rr64 = rr;
    if (f32_updates) {
      rb32 = workspace(lat, 13, S.hb[TM_F32], &st);
      if (st == TM_OK) T32 = workspace(lat, 14, S.hb[TM_F32], &st);
      if (st == TM_OK) W32 = workspace(lat, 15, S.hb[TM_F32], &st);
      if (st == TM_OK) st = cuda_check(cudaMemcpyAsync(rb32, rs, S.hb[TM_F32], cudaMemcpyDeviceToDevice, s), "copy");
      if (st != TM_OK) return st;
    }
    void *bpd = nullptr, *Rd = nullptr, *Xd = nullptr, *Td = nullptr, *Wd = nullptr;
    if (dd_updates) {
      bpd = workspace(lat, 13, S.hb[TM_DF64], &st);
      if (st == TM_OK) Rd = workspace(lat, 14, S.hb[TM_DF64], &st);
      if (st == TM_OK) Xd = workspace(lat, 15, S.hb[TM_DF64], &st);
      if (st == TM_OK) Td = workspace(lat, 16, S.hb[TM_DF64], &st);
      if (st == TM_OK) Wd = workspace(lat, 17, S.hb[TM_DF64], &st);
      if (st == TM_OK) st = convert_half(lat, TM_DF64, bpd, TM_F64, bp, s);
      if (st != TM_OK) return st;
    }
    while (!converged && iters < P.max_iter) {
      CGState fin;
      if ((st = run_stage(S, v, fresh_state(rr, stop2, P.max_iter, iters, delta2, SLOPPY_GROWTH), &fin)) != TM_OK)
        return st;
      trace_stage("sloppy stage", fin, bb);
      if (fin.nonfinite) {
        // the sloppy iteration overflowed: drop its increment, restart from the FP64 solution
        if (++bad_stages > 3) return set_error(TM_ERR_NONFINITE, "tm_solve_cg: non-finite value in the iteration");
        iters = fin.iter;
        if ((st = cuda_check(cudaMemsetAsync(xs, 0, S.hb[TM_F32], s), "memset")) != TM_OK) return st;
        fin.diverged = 1;
      } else {
        bad_stages = 0;
        if (fin.iter == iters) break;  // no progress (breakdown of <p, A p>): stop, report not converged
        iters = fin.iter;
        if (f32_updates && !fin.converged && !fin.diverged && fin.rr > F32_UPDATE_SPAN * F32_UPDATE_SPAN * rr64) {
          // FP32 recomputation relative to the last FP64 residual; xs keeps accumulating
          if ((st = cuda_check(cudaMemcpyAsync(rs, rb32, S.hb[TM_F32], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK)
            return st;
          if ((st = normal_apply(S, TM_F32, sl, xs, T32, W32, rs, nullptr)) != TM_OK) return st;
          double rr32 = 0.0;
          if ((st = cuda_check(cudaMemcpyAsync(&lat->flag_host[0], lat->dscalars, sizeof(double),
                                               cudaMemcpyDeviceToHost, s), "readback")) != TM_OK)
            return st;
          if ((st = cuda_check(cudaStreamSynchronize(s), "synchronise")) != TM_OK) return st;
          memcpy(&rr32, &lat->flag_host[0], sizeof(double));
          ++updates;
          if (verbose())
            fprintf(stderr, "[tm_solve_cg] FP32 update %d: |r|/|b| %.3e\n", updates, std::sqrt(rr32 / bb));
          if (!(rr32 < 1e300)) return set_error(TM_ERR_NONFINITE, "tm_solve_cg: residual diverged");
          rr = rr32;
          continue;
        }
        const unsigned nbb = blas_blocks(lat->geom.h);
        accumulate_kernel<TM_F32><<<nbb, BNT, 0, s>>>(lat->geom.h, static_cast<char*>(X), static_cast<char*>(xs));
        count_launch();
        w_valid = false;
        if (defer_final && fin.converged && !dd_updates) {  // the caller confirms X in FP64
          if ((st = cuda_check(cudaGetLastError(), "accumulate kernel")) != TM_OK) return st;
          res->iters = iters;
          res->updates = updates;
          res->converged = false;
          res->rr_true = fin.rr;
          res->xo_in_W = false;
          res->pending = true;
          return TM_OK;
        }
      }
      if ((st = cuda_check(cudaGetLastError(), "accumulate kernel")) != TM_OK) return st;
      const void* rsrc = R;
      int rprec = TM_F64;
      if (dd_updates) {
        if ((st = true_residual_dd(S, Rd, X, bpd, Td, Wd, Xd, &rr_true)) != TM_OK) return st;
        rsrc = Rd;
        rprec = TM_DF64;
      } else {
        if ((st = true_residual(S, R, X, bp, T, W, &rr_true)) != TM_OK) return st;
        w_valid = true;
      }
      ++updates;
      trace_update(updates, rr_true, bb);
      if (rr_true < stop2) {
        if (!dd_updates) {
          converged = true;
          break;
        }
        // confirm in FP64; if the double-float residual was too optimistic, carry on in FP64
        if ((st = true_residual(S, R, X, bp, T, W, &rr_true)) != TM_OK) return st;
        w_valid = true;
        ++updates;
        trace_update(updates, rr_true, bb);
        if (rr_true < stop2) {
          converged = true;
          break;
        }
        dd_updates = false;
        rsrc = R;
        rprec = TM_F64;
      }
      if (!(rr_true < 1e300)) return set_error(TM_ERR_NONFINITE, "tm_solve_cg: residual diverged");
      if ((st = convert_half(lat, TM_F32, rs, rprec, rsrc, s)) != TM_OK) return st;
      // after a divergent stage the search direction restarts from the true residual
      if (fin.diverged && (st = convert_half(lat, sp, ps, rprec, rsrc, s)) != TM_OK) return st;
      rr = rr_true;
      rr64 = rr_true;
      if (f32_updates &&
          (st = cuda_check(cudaMemcpyAsync(rb32, rs, S.hb[TM_F32], cudaMemcpyDeviceToDevice, s), "copy")) != TM_OK)
        return st;
    }
  }
  res->iters = iters;
  res->updates = updates;
  res->converged = converged;
  res->rr_true = rr_true;
  res->xo_in_W = w_valid;
  res->pending = false;
  return TM_OK;
}

// Solves M^f x = b for one canonical full field (device pointers).
static tm_status solve_one(tm_lattice lat, double* x, const double* b, const tm_cg_params& P, tm_cg_info* info,
                           cudaStream_t s) {
  Solver S{lat, s, P.flavour, 2.0 * lat->kappa * lat->mu, {0, 0, 0, 0}};
  for (int p = 0; p < 4; ++p) S.hb[p] = spinor_bytes_per_site(p) * lat->h;
  tm_status st = TM_OK;
  // FP64 fields: 0 b_e, 1 b_o, 2 b', 3 X, 4 R, 5 P, 6 T, 7 W
  void* w[8];
  for (int k = 0; k < 8; ++k) {
    w[k] = workspace(lat, k, S.hb[TM_F64], &st);
    if (st != TM_OK) return st;
  }
  void *be = w[0], *bo = w[1], *bp = w[2], *X = w[3], *R = w[4], *Pv = w[5], *T = w[6], *W = w[7];

  // ---- source preparation (App. B.2): b' = gamma5 (b_o + kappa H_oe (M_ee^f)^-1 b_e)
  double bb = 0.0, bfull = 0.0;
  if ((st = prepare_source(S, b, be, bo, bp, T, &bb, &bfull)) != TM_OK) return st;
  if (!std::isfinite(bb) || !std::isfinite(bfull))
    return set_error(TM_ERR_NONFINITE, "tm_solve_cg: the source has non-finite entries");
  info->iters = 0;
  info->reliable_updates = 0;
  if (bfull == 0.0) {
    st = cuda_check(cudaMemsetAsync(x, 0, lat->V * 24 * sizeof(double), s), "memset");
    info->true_rel_residual = 0.0;
    info->schur_rel_residual = 0.0;
    info->status = TM_OK;
    return st;
  }
  // Mixed modes defer the last confirmation: when a sloppy stage reaches the tolerance, X is
  // confirmed by the reconstruction's FP64 residual of the full system, whose odd part
  // ||(b - M x)_o|| = ||varphi_o - Mhat x_o|| = ||b' - A X|| up to the rounding of x_e (the even
  // part vanishes but for that rounding).  That costs 4 FP64 hopping launches (x_o = Qhat^{-f} X,
  // x_e, the odd residual) where recomputing b' - A X first would cost 6.  If the FP64 residual
  // misses the tolerance the iteration continues from X (cg_normal recomputes b' - A X).
  const bool defer = P.mode != TM_CG_FP64 && P.update_prec != TM_DF64;
  const double stop2 = P.tol * P.tol * bb;
  NormalResult nr{};
  if ((st = cg_normal(S, P, bp, bb, X, false, R, Pv, T, W, &nr, defer)) != TM_OK) return st;
  int iters = nr.iters, updates = nr.updates;
  bool converged = nr.converged;
  double rr_true = nr.rr_true;
  bool reconstructed = false;
  while (nr.pending) {
    double rro = 0.0;
    if ((st = reconstruct_check(S, X, be, bo, bfull, x, T, W, R, Pv, &info->true_rel_residual, &rro)) != TM_OK)
      return st;
    ++updates;  // an FP64 residual recomputation
    rr_true = rro;
    if (verbose())
      fprintf(stderr, "[tm_solve_cg] confirmation: FP64 |(b - M x)_o|/|b'| %.3e (%s)\n", std::sqrt(rro / bb),
              rro < stop2 ? "converged" : "not confirmed, continuing");
    if (rro < stop2) {
      converged = true;
      reconstructed = true;
      break;
    }
    if (iters >= P.max_iter) break;
    tm_cg_params Q = P;
    Q.max_iter = P.max_iter - iters;
    if ((st = cg_normal(S, Q, bp, bb, X, true, R, Pv, T, W, &nr, defer)) != TM_OK) return st;
    iters += nr.iters;
    updates += nr.updates;
    converged = nr.converged;
    rr_true = nr.rr_true;
  }
  info->iters = iters;
  info->reliable_updates = updates;
  info->schur_rel_residual = std::sqrt(rr_true / bb);

  // ---- reconstruction and the FP64 residual of the full system (x_o = Qhat^{-f} X is already in W
  // when the last operation was the FP64 residual of the final X)
  if (reconstructed)
    st = TM_OK;
  else if (nr.xo_in_W)
    st = reconstruct_xo(S, W, be, bo, bfull, x, T, R, Pv, &info->true_rel_residual);
  else
    st = reconstruct_check(S, X, be, bo, bfull, x, T, W, R, Pv, &info->true_rel_residual);
  if (st != TM_OK) return st;
  info->status = converged ? TM_OK : TM_ERR_NOT_CONVERGED;
  if (!converged)
    return set_error(TM_ERR_NOT_CONVERGED, "tm_solve_cg: not converged after %d iterations (||r||/||b|| = %.3e)",
                     iters, info->schur_rel_residual);
  return TM_OK;
}

}  // namespace tmq

using namespace tmq;

extern "C" {

void tm_cg_params_default(tm_cg_params* p) {
  if (!p) return;
  p->tol = 1e-10;
  p->max_iter = 100000;
  p->mode = TM_CG_FP64;
  p->sloppy_prec = TM_F32;
  p->sloppy_link = TM_LINK12;
  p->delta = 0.1;
  p->use_x0 = 0;
  p->flavour = 1;
  p->update_prec = TM_F64;
}

tm_status tm_solve_cg(tm_lattice lat, double* x, const double* b, int nrhs, const tm_cg_params* params,
                      tm_cg_info* info, void* stream) {
  return solve_driver(lat, x, b, nrhs, params, info, stream, SOLVER_CG);
}

}  // extern "C"

namespace tmq {

// Validation, host staging, the loop over right-hand sides and the defect correction from an
// initial guess, shared by tm_solve_cg and tm_solve_bicgstab.
tm_status solve_driver(tm_lattice lat, double* x, const double* b, int nrhs, const tm_cg_params* params,
                       tm_cg_info* info, void* stream, int kind) {
  const auto t0 = std::chrono::steady_clock::now();
  const char* nm = kind == SOLVER_CG ? "tm_solve_cg" : (kind == SOLVER_MR ? "tm_solve_mr" : "tm_solve_bicgstab");
  if (!lat || !x || !b || nrhs < 1) return set_error(TM_ERR_ARG, "%s: bad argument", nm);
  if (!lat->has_gauge) return set_error(TM_ERR_NO_GAUGE, "%s: no gauge field", nm);
  tm_cg_params P;
  if (params)
    P = *params;
  else
    tm_cg_params_default(&P);
  if (P.flavour == 0) P.flavour = 1;
  if (P.flavour != 1 && P.flavour != -1) return set_error(TM_ERR_ARG, "%s: flavour must be +1 or -1", nm);
  if (!(P.tol > 0.0) || P.max_iter < 1) return set_error(TM_ERR_ARG, "%s: tol > 0 and max_iter >= 1", nm);
  if (P.mode < TM_CG_FP64 || P.mode > TM_CG_RELIABLE) return set_error(TM_ERR_ARG, "%s: mode %d", nm, P.mode);
  if (P.mode != TM_CG_FP64) {
    if (P.sloppy_prec != TM_F32 && P.sloppy_prec != TM_F16)
      return set_error(TM_ERR_ARG, "%s: sloppy precision must be TM_F32 or TM_F16", nm);
    if (P.sloppy_link != 18 && P.sloppy_link != 12 && P.sloppy_link != 8)
      return set_error(TM_ERR_ARG, "%s: sloppy link format %d", nm, P.sloppy_link);
    if (!(P.delta > 0.0 && P.delta < 1.0)) return set_error(TM_ERR_ARG, "%s: delta must be in (0, 1)", nm);
    if (P.update_prec != TM_F64 && P.update_prec != TM_DF64 && P.update_prec != TM_F32)
      return set_error(TM_ERR_ARG, "%s: update_prec must be TM_F64, TM_F32 or TM_DF64", nm);
  }
  if (kind != SOLVER_CG && (P.mode == TM_CG_SQRT_EPS || (P.mode == TM_CG_RELIABLE && P.update_prec != TM_F64)))
    return set_error(TM_ERR_UNSUPPORTED, "%s: modes TM_CG_FP64 and TM_CG_RELIABLE with FP64 updates only", nm);
  if (kind == SOLVER_MR && P.mode == TM_CG_RELIABLE && P.sloppy_prec != TM_F32)
    return set_error(TM_ERR_UNSUPPORTED, "%s: sloppy storage TM_F32 only", nm);
  const size_t fbytes = lat->V * 24 * sizeof(double);
  if (x == b) return set_error(TM_ERR_ARG, "%s: x and b must differ", nm);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tm_status st;
  const double* db = static_cast<const double*>(stage_in(lat, WS_STAGE_IN, b, fbytes * nrhs, s, &st));
  if (st != TM_OK) return st;
  double* dx = static_cast<double*>(stage_out(lat, WS_STAGE_OUT, x, fbytes * nrhs, &st));
  if (st != TM_OK) return st;
  if (P.use_x0 && dx != x) {
    st = cuda_check(cudaMemcpyAsync(dx, x, fbytes * nrhs, cudaMemcpyHostToDevice, s), "x0 copy");
    if (st != TM_OK) return st;
  }
  tm_cg_info worst{};
  worst.status = TM_OK;
  tm_status result = TM_OK;
  // several right-hand sides in the reliable-update mode: solved together by the batched solver
  // (their sloppy iterations share launches and link reads)
  const bool batched = kind == SOLVER_CG && nrhs > 1 && P.mode == TM_CG_RELIABLE && P.update_prec == TM_F64 &&
                       !P.use_x0;
  if (batched) {
    std::vector<tm_system> sys(nrhs);
    std::vector<tm_cg_info> infos(nrhs);
    for (int r = 0; r < nrhs; ++r)
      sys[r] = tm_system{lat, lat->mu, P.flavour, dx + (size_t)r * lat->V * 24, db + (size_t)r * lat->V * 24};
    st = tm_solve_cg_batch(sys.data(), nrhs, &P, infos.data(), stream);
    if (st != TM_OK && st != TM_ERR_NOT_CONVERGED) return st;
    result = st;
    for (int r = 0; r < nrhs; ++r) {
      if (r == 0 || infos[r].true_rel_residual > worst.true_rel_residual) worst = infos[r];
      if (infos[r].iters > worst.iters) worst.iters = infos[r].iters;
    }
  }
  for (int r = 0; r < (batched ? 0 : nrhs); ++r) {
    double* xr = dx + (size_t)r * lat->V * 24;
    const double* br = db + (size_t)r * lat->V * 24;
    tm_cg_info one{};
    if (P.use_x0) {
      // defect correction from the initial guess: x = x0 + M^-1 (b - M x0)
      double* d = static_cast<double*>(workspace(lat, WS_X0, 2 * fbytes, &st));
      if (st != TM_OK) return st;
      double* r0 = d;
      double* delta = d + lat->V * 24;
      const size_t n = lat->V * 24;
      const unsigned nb = (unsigned)std::min<size_t>((n + BNT - 1) / BNT, 152 * 16);
      if ((st = tm_apply_D(lat, r0, xr, P.flavour, 0, 1, stream)) != TM_OK) return st;
      axpby_kernel<<<nb, BNT, 0, s>>>(n, 1.0, br, -1.0, r0);  // r0 = b - M x0
      count_launch();
      st = kind == SOLVER_CG ? solve_one(lat, delta, r0, P, &one, s)
           : kind == SOLVER_MR ? solve_one_mr(lat, delta, r0, P, &one, s)
                               : solve_one_bicgstab(lat, delta, r0, P, &one, s);
      if (st != TM_OK && st != TM_ERR_NOT_CONVERGED) return st;
      axpby_kernel<<<nb, BNT, 0, s>>>(n, 1.0, delta, 1.0, xr);  // x = x0 + delta
      count_launch();
      tm_status st2 = cuda_check(cudaGetLastError(), "axpby kernel");
      if (st2 != TM_OK) return st2;
      {
        // true residual relative to b
        double* rfull = r0;
        if ((st2 = tm_apply_D(lat, rfull, xr, P.flavour, 0, 1, stream)) != TM_OK) return st2;
        axpby_kernel<<<nb, BNT, 0, s>>>(n, 1.0, br, -1.0, rfull);
        count_launch();
        double num = 0.0, den = 0.0;
        if ((st2 = full_norm2(lat, rfull, &num, s)) != TM_OK) return st2;
        if ((st2 = full_norm2(lat, br, &den, s)) != TM_OK) return st2;
        one.true_rel_residual = den > 0 ? std::sqrt(num / den) : 0.0;
      }
    } else {
      st = kind == SOLVER_CG ? solve_one(lat, xr, br, P, &one, s)
           : kind == SOLVER_MR ? solve_one_mr(lat, xr, br, P, &one, s)
                               : solve_one_bicgstab(lat, xr, br, P, &one, s);
    }
    if (st != TM_OK && st != TM_ERR_NOT_CONVERGED) return st;
    if (st == TM_ERR_NOT_CONVERGED) result = st;
    if (r == 0 || one.true_rel_residual > worst.true_rel_residual) worst = one;
    if (one.iters > worst.iters) worst.iters = one.iters;
  }
  if (dx != x) {
    if ((st = stage_out_finish(x, dx, fbytes * nrhs, s)) != TM_OK) return st;
  }
  if ((st = cuda_check(cudaStreamSynchronize(s), "solve: synchronise")) != TM_OK) return st;
  worst.status = result;
  worst.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = worst;
  return result;
}

}  // namespace tmq
