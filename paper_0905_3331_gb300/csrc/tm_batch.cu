// tm_batch.cu -- many systems M_s^f x_s = b_s solved together (tm_solve_cg_batch).
//
// Systems may differ in source, twisted mass and lattice (geometry and gauge field).  Every
// system runs the mixed-precision reliable-update CG of tm_solver.cu, but the sloppy
// iterations of all systems go through the same kernels: one launch of K1..K4 and of the
// update covers every system, its blocks mapped to (system, block of sites) by a table, with
// the blocks of systems that share a lattice interleaved so that each link is fetched from
// HBM once and served to the other systems from L2.  Each system keeps its own device-side
// CG state and reductions.  The whole solve is one CUDA graph launch: a WHILE node over one
// batched iteration followed by an IF node that runs the FP64 service -- the reliable update of
// every system that stopped in that iteration (its trigger, convergence of the sloppy residual,
// divergence, a non-finite value, its iteration bound): X += x, r = b' - A X in FP64, and the
// decision to finish the system or resume it from r -- in batched kernels as well.  The loop
// ends when every system is finished; the host then reconstructs and checks each solution.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "tm_dslash.cuh"
#include "tm_solver.cuh"

namespace tmq {

// Per-system descriptor (device memory).
struct BatchSys {
  Geom g;
  const char* links;   // sloppy gauge copy of the system's lattice
  EpiCoef coef[4];     // epilogues of K1..K4 (this system's mu)
  void* vec[5];        // 0 p, 1 T, 2 W (sloppy storage), 3 r, 4 x increment (FP32)
  CGState* st;
  double* partials;    // reduction partials of this system (nblocks entries)
  unsigned* counters;  // [0] reductions, [1] update kernel
  int nblocks;         // hopping blocks (HOP_NT sites each)
  int nblocks_upd;     // update-kernel blocks
  double* result;      // the FP64 service's ||b' - A X||^2 (reductions of kind FIN_STORE)
};

struct BatchGlobal {
  int unfinished;    // systems not yet done for good
  int loops;         // iterations executed (bodies of the graph loop)
  int loop_cap;      // hard bound on loops
  unsigned counter;  // update-kernel blocks arrived
  int nsys;          // systems in the batch
  int pad;
  double delta2;     // reliable-update trigger of a resumed system
  double grow2;      // divergence guard of a resumed system
};

// Up to 4 systems of one lattice whose hopping terms one block computes together.
struct BatchGroup {
  int n;       // systems in the group (1 .. K of the kernel)
  int sys[4];  // their indices in the system table (the first one's geometry and links serve all)
};

// The hopping operator of K systems at once: thread = site, the K systems of the block's group
// are its lanes.  Each of the 8 links of the site is loaded and reconstructed ONCE and applied to
// the K systems' neighbour spinors (the same direction-pair arithmetic as hop_kernel, per lane),
// so a link's bytes and its reconstruction are shared by K right-hand sides in registers.  Each
// system keeps its own epilogue coefficients (its mu), output, CG state and reduction.  A system
// that has stopped (its stage trigger, convergence) is skipped; the block returns when all of its
// group have.  K = 1 is the one-system case.  Register budgets: 6 blocks of 128 per SM for K = 1
// (80 registers; latency bound: 12-system solve on 24^3 x 48 1060 -> 990 ms), 4 for K = 2, 2 for
// K = 4 (the accumulators of K spinors).  SERV: the FP64 service of stopped systems (FP64 storage,
// 18-real links): the live systems are those stopped and not finished, the residual update uses
// alpha = 1 (r = b' - A X from r = b'), and the last reduction stores ||r||^2 in B.result.
template <int PREC, int NREAL, bool HAS_Y, int MODE, int K, bool SERV = false>
__global__ void __launch_bounds__(HOP_NT, (PREC == TM_F64 ? 1 : (K == 1 ? 6 : (K == 2 ? 4 : 2))))
    hop_group_kernel(const BatchSys* __restrict__ systems, const BatchGroup* __restrict__ groups,
                     const int2* __restrict__ map, int in_sel, int y_sel, int out_sel, int kk, int out_parity) {
  typedef typename SpinorFmt<PREC>::real R;
  typedef SpinorFmt<PREC> F;
  typedef typename LinkStore<PREC>::type St;
  constexpr int BYTES = NREAL * LinkStore<PREC>::size;
  __shared__ double sh[HOP_NT / 32];
  const int2 m = map[blockIdx.x];
  const BatchGroup G = groups[m.x];
  const BatchSys* S[K];
  bool live[K];
  bool any = false;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    S[j] = systems + G.sys[j < G.n ? j : 0];
    const CGState* sj = S[j]->st;
    live[j] = j < G.n && (SERV ? (sj->done && !sj->finished) : !sj->done);
    any = any || live[j];
  }
  if (!any) return;
  const Geom g = S[0]->g;
  const int cb = m.y * HOP_NT + threadIdx.x;
  const bool active = cb < g.h;
  cpx<R> acc[K][12];
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int q = 0; q < 12; ++q) acc[j][q] = mk<R>(R(0), R(0));
  if (active) {
    const SiteCoord c = site_of(g, cb, out_parity);
    int nb[8];
    neighbours(g, cb, c, nb);
    const size_t slab = link_bytes(PREC, NREAL) * (size_t)g.h;
    const char* lf = S[0]->links + (size_t)(out_parity * 4) * slab;
    const char* lo = S[0]->links + (size_t)((1 - out_parity) * 4) * slab;
    const bool tf = (c.t == g.T - 1), tb = (c.t == 0);
#define TM_GROUP_DIR(MU, FIRST)                                                                     \
  {                                                                                                 \
    cpx<R> u0[K][3], u1[K][3], p[12];                                                               \
    R scale;                                                                                        \
    Mat3<R> U;                                                                                      \
    LinkRecon<R, St, NREAL>::unpack(load_raw<BYTES>(lf + MU * slab, g.h, cb), U);                   \
    _Pragma("unroll") for (int j = 0; j < K; ++j) if (live[j]) {                                    \
      F::load_unscaled(S[j]->vec[in_sel], g.h, nb[MU], p, scale);                                   \
      pair_fwd_mat<PREC, MU>(u0[j], u1[j], U, p, scale, MU == 0 && tf);                             \
    }                                                                                               \
    LinkRecon<R, St, NREAL>::unpack(load_raw<BYTES>(lo + MU * slab, g.h, nb[4 + MU]), U);           \
    _Pragma("unroll") for (int j = 0; j < K; ++j) if (live[j]) {                                    \
      F::load_unscaled(S[j]->vec[in_sel], g.h, nb[4 + MU], p, scale);                               \
      pair_bwd_mat<PREC, MU, FIRST>(acc[j], u0[j], u1[j], U, p, scale, MU == 0 && tb);              \
    }                                                                                               \
  }
    TM_GROUP_DIR(0, true)
    TM_GROUP_DIR(1, false)
    TM_GROUP_DIR(2, false)
    TM_GROUP_DIR(3, false)
#undef TM_GROUP_DIR
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (!live[j]) continue;  // block-uniform
    const BatchSys& B = *S[j];
    CGState* st = B.st;
    const EpiCoef coef = B.coef[kk];
    const R cc = (R)coef.c;
    const cpx<R> Du = mk<R>((R)coef.d_up_re, (R)coef.d_up_im), Dl = mk<R>((R)coef.d_lo_re, (R)coef.d_lo_im);
    cpx<R> o[12];
    if (HAS_Y) {
      const cpx<R> Eu = mk<R>((R)coef.e_up_re, (R)coef.e_up_im), El = mk<R>((R)coef.e_lo_re, (R)coef.e_lo_im);
      cpx<R> yv[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) yv[q] = mk<R>(R(0), R(0));
      if (active) F::load(B.vec[y_sel], g.h, cb, yv);
#pragma unroll
      for (int q = 0; q < 12; ++q) o[q] = ((q < 6) ? Du : Dl) * (cc * acc[j][q] + ((q < 6) ? Eu : El) * yv[q]);
    } else {
#pragma unroll
      for (int q = 0; q < 12; ++q) o[q] = ((q < 6) ? Du : Dl) * (cc * acc[j][q]);
    }
    typedef typename SiteSum<R>::type SR;
    SR nrm = SR(0);
    void* outp = B.vec[out_sel];
    if (MODE == 2) {
      if (active) {
        const R al = SERV ? R(1) : (R)st->alpha;
        constexpr int PR = ResidPrec<PREC>::value;
        cpx<R> r[12];
        SpinorFmt<PR>::load(outp, g.h, cb, r);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          r[q] = r[q] - al * o[q];
          nrm += (SR)norm2(r[q]);
        }
        SpinorFmt<PR>::store(outp, g.h, cb, r);
      }
    } else if (active) {
      if (MODE == 1) {
#pragma unroll
        for (int q = 0; q < 12; ++q) nrm += (SR)norm2(o[q]);
      }
      F::store(outp, g.h, cb, o);
    }
    if (MODE >= 1) {
      const Reduce red{B.partials, B.counters, B.result, st, SERV ? FIN_STORE : (MODE == 1 ? FIN_CG_ALPHA : FIN_CG_RR)};
      const double bs = block_sum<HOP_NT>((double)nrm, sh);
      grid_reduce<HOP_NT>(red, 0, B.nblocks, m.y, bs, sh);
      __syncthreads();  // sh and the reduction's shared flag are reused by the next system
    }
  }
}

// x += alpha p, p = r + beta p per system.  The last block of all sets the graph's conditions: the
// loop runs again while a system is not finished (and below the loop cap), and the FP64 service
// runs when a system has stopped (its reliable-update trigger, convergence of the sloppy residual,
// divergence, a non-finite value, or its iteration bound).
template <int PP>
__global__ void __launch_bounds__(BNT) cg_update_batch_kernel(const BatchSys* __restrict__ systems,
                                                              const int2* __restrict__ map, BatchGlobal* gl,
                                                              cudaGraphConditionalHandle cond_loop,
                                                              cudaGraphConditionalHandle cond_serv, int use_cond) {
  typedef typename SpinorFmt<PP>::real RP;
  const int2 m = map[blockIdx.x];
  const BatchSys& B = systems[m.x];
  CGState& S = *B.st;
  const int iter = S.iter;
  const bool work = iter != S.applied;
  if (work) {
    const double alpha = S.alpha, beta = S.beta;
    const int h = B.g.h;
    char* x = static_cast<char*>(B.vec[4]);
    char* p = static_cast<char*>(B.vec[0]);
    const char* r = static_cast<const char*>(B.vec[3]);
    for (int i = m.y * BNT + threadIdx.x; i < h; i += B.nblocks_upd * BNT) {
      cpx<float> xv[12], rv[12];
      cpx<RP> pv[12];
      SpinorFmt<TM_F32>::load(x, h, i, xv);
      SpinorFmt<PP>::load(p, h, i, pv);
      SpinorFmt<TM_F32>::load(r, h, i, rv);
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        xv[q] = xv[q] + (float)alpha * mk<float>((float)pv[q].re, (float)pv[q].im);
        pv[q] = rv[q] + (RP)beta * pv[q];
      }
      SpinorFmt<TM_F32>::store(x, h, i, xv);
      SpinorFmt<PP>::store(p, h, i, pv);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (work && arrive_acq_rel(B.counters + 1) == (unsigned)B.nblocks_upd - 1) {
      S.applied = iter;
      B.counters[1] = 0u;
    }
    if (arrive_acq_rel(&gl->counter) == gridDim.x - 1) {  // every block's update of `applied` is visible
      gl->counter = 0u;
      gl->loops += 1;
      int need = 0;
      for (int k = 0; k < gl->nsys; ++k) {
        const CGState& q = *systems[k].st;
        need |= (q.done && !q.finished) ? 1 : 0;
      }
      if (use_cond) {
        cudaGraphSetConditional(cond_serv, need ? 1u : 0u);
        cudaGraphSetConditional(cond_loop, (gl->unfinished > 0 && gl->loops < gl->loop_cap) ? 1u : 0u);
      }
    }
  }
}

// ---- the FP64 service of the systems that stopped (all inside the solve's graph)
// 1. X (FP64) += x_s (FP32; dropped after a non-finite value), x_s = 0; r (FP64) = b'.
__global__ void __launch_bounds__(BNT) serv_begin_kernel(const BatchSys* __restrict__ sys, const BatchSys* __restrict__ sys64,
                                                         const int2* __restrict__ map) {
  const int2 m = map[blockIdx.x];
  const BatchSys& B = sys[m.x];
  const BatchSys& D = sys64[m.x];
  const CGState& S = *B.st;
  if (!S.done || S.finished) return;
  const int h = B.g.h;
  char* xs = static_cast<char*>(B.vec[4]);
  char* X = static_cast<char*>(D.vec[0]);
  char* R = static_cast<char*>(D.vec[3]);
  const char* bp = static_cast<const char*>(D.vec[4]);
  for (int i = m.y * BNT + threadIdx.x; i < h; i += B.nblocks_upd * BNT) {
    cpx<double> a[12], b[12];
    cpx<float> d[12];
    SpinorFmt<TM_F32>::load(xs, h, i, d);
    if (!S.nonfinite) {
      SpinorFmt<TM_F64>::load(X, h, i, a);
#pragma unroll
      for (int q = 0; q < 12; ++q) a[q] = a[q] + mk<double>((double)d[q].re, (double)d[q].im);
      SpinorFmt<TM_F64>::store(X, h, i, a);
    }
#pragma unroll
    for (int q = 0; q < 12; ++q) d[q] = mk<float>(0.f, 0.f);
    SpinorFmt<TM_F32>::store(xs, h, i, d);
    SpinorFmt<TM_F64>::load(bp, h, i, b);
    SpinorFmt<TM_F64>::store(R, h, i, b);
  }
}

// 3. The decision per stopped system, from its FP64 residual rr64 = ||b' - A X||^2 (one block).
__global__ void serv_decide_kernel(const BatchSys* __restrict__ sys, BatchGlobal* gl) {
  for (int k = threadIdx.x; k < gl->nsys; k += blockDim.x) {
    const BatchSys& B = sys[k];
    CGState& S = *B.st;
    S.rearm = 0;
    S.restart = 0;
    if (!S.done || S.finished) continue;
    const double rr = *B.result;
    S.updates += 1;
    S.rr64 = rr;
    bool fin = false;
    if (S.nonfinite) {
      fin = (++S.bad > 1000);  // the increment was dropped; resume from the FP64 solution
    } else if (S.iter == S.serv_iter) {
      fin = true;  // a breakdown without progress since the last service
    }
    if (!fin) {
      if (rr < S.stop2) {
        fin = true;
        S.ok = 1;
      } else if (!(rr < 1e300) || S.iter >= S.max_iter) {
        fin = true;
      }
    }
    if (fin) {
      S.finished = 1;
      atomicSub(&gl->unfinished, 1);
      continue;
    }
    if (S.converged) S.missed += 1;  // the sloppy residual's convergence was not confirmed
    S.restart = (S.diverged || S.nonfinite || S.converged) ? 1 : 0;
    S.rearm = 1;
    S.serv_iter = S.iter;
    // a fresh stage from the FP64 residual
    S.rr = rr;
    S.rr_ref = rr;
    S.rr_min = rr;
    S.delta2 = gl->delta2;
    S.grow2 = gl->grow2;
    S.applied = S.iter;
    S.done = 0;
    S.converged = 0;
    S.nonfinite = 0;
    S.want_update = 0;
    S.diverged = 0;
  }
}

// 4. r_s (FP32) = r, and p = r (sloppy) for a restart, for the systems the decision resumed.
template <int PP>
__global__ void __launch_bounds__(BNT) serv_convert_kernel(const BatchSys* __restrict__ sys,
                                                           const BatchSys* __restrict__ sys64,
                                                           const int2* __restrict__ map) {
  const int2 m = map[blockIdx.x];
  const BatchSys& B = sys[m.x];
  const CGState& S = *B.st;
  if (!S.rearm) return;
  const int h = B.g.h;
  const char* R = static_cast<const char*>(sys64[m.x].vec[3]);
  char* rs = static_cast<char*>(B.vec[3]);
  char* ps = static_cast<char*>(B.vec[0]);
  for (int i = m.y * BNT + threadIdx.x; i < h; i += B.nblocks_upd * BNT) {
    cpx<double> a[12];
    SpinorFmt<TM_F64>::load(R, h, i, a);
    SpinorFmt<TM_F32>::store(rs, h, i, a);
    if (S.restart) SpinorFmt<PP>::store(ps, h, i, a);
  }
}

template <int PREC, int NREAL, int K, bool SERV>
static tm_status launch_hop_group(const BatchSys* d_sys, const BatchGroup* d_grp, const int2* d_map, int nblocks,
                                  int in_sel, int y_sel, int out_sel, int kk, int parity, int mode, bool has_y,
                                  cudaStream_t s) {
#define TM_GARGS d_sys, d_grp, d_map, in_sel, y_sel, out_sel, kk, parity
  if (!has_y && mode == 0)
    hop_group_kernel<PREC, NREAL, false, 0, K, SERV><<<nblocks, HOP_NT, 0, s>>>(TM_GARGS);
  else if (has_y && mode == 0)
    hop_group_kernel<PREC, NREAL, true, 0, K, SERV><<<nblocks, HOP_NT, 0, s>>>(TM_GARGS);
  else if (has_y && mode == 1)
    hop_group_kernel<PREC, NREAL, true, 1, K, SERV><<<nblocks, HOP_NT, 0, s>>>(TM_GARGS);
  else
    hop_group_kernel<PREC, NREAL, true, 2, K, SERV><<<nblocks, HOP_NT, 0, s>>>(TM_GARGS);
#undef TM_GARGS
  count_launch();
  return cuda_check(cudaGetLastError(), "batched hopping kernel");
}

// The batched hopping launch of one storage form with K systems per group (FP64 with K = 1 for the
// service of stopped systems).
struct GroupLaunch {
  int prec, nreal, K;
  const BatchSys* sys;
  const BatchGroup* grp;
  const int2* map;
  int nblocks;
};

static tm_status hop_batch(const GroupLaunch& L, int in_sel, int y_sel, int out_sel, int kk, int parity, int mode,
                           bool has_y, cudaStream_t s) {
  if (L.prec == TM_F64)
    return launch_hop_group<TM_F64, 18, 1, true>(L.sys, L.grp, L.map, L.nblocks, in_sel, y_sel, out_sel, kk, parity,
                                                 mode, has_y, s);
#define TM_B(P, N, KK)                                                                                    \
  if (L.prec == P && L.nreal == N && L.K == KK)                                                          \
    return launch_hop_group<P, N, KK, false>(L.sys, L.grp, L.map, L.nblocks, in_sel, y_sel, out_sel, kk, parity, \
                                             mode, has_y, s);
#define TM_BK(P, N) TM_B(P, N, 1) TM_B(P, N, 2) TM_B(P, N, 4)
  TM_BK(TM_F32, 18) TM_BK(TM_F32, 12) TM_BK(TM_F32, 8) TM_BK(TM_F16, 18) TM_BK(TM_F16, 12) TM_BK(TM_F16, 8)
#undef TM_BK
#undef TM_B
  return set_error(TM_ERR_UNSUPPORTED, "batched solve: sloppy form not supported");
}

// One batched CG iteration: K1..K4 of every running system, then the update (which sets the graph
// conditions).
static tm_status batch_iteration(const GroupLaunch& L, const int2* d_umap, int nu, BatchGlobal* d_gl,
                                 cudaGraphConditionalHandle cond_loop, cudaGraphConditionalHandle cond_serv,
                                 int use_cond, cudaStream_t s) {
  tm_status st;
  // K1: T = (M_ee^-f)^-1 H_eo p ; K2: W = Qhat^-f p, <p,Ap> ; K3: T = (M_ee^f)^-1 H_eo W ; K4: r -= alpha Qhat^f W
  if ((st = hop_batch(L, 0, 0, 1, 0, 0, 0, false, s)) != TM_OK) return st;
  if ((st = hop_batch(L, 1, 0, 2, 1, 1, 1, true, s)) != TM_OK) return st;
  if ((st = hop_batch(L, 2, 0, 1, 2, 0, 0, false, s)) != TM_OK) return st;
  if ((st = hop_batch(L, 1, 2, 3, 3, 1, 2, true, s)) != TM_OK) return st;
  if (L.prec == TM_F32)
    cg_update_batch_kernel<TM_F32><<<nu, BNT, 0, s>>>(L.sys, d_umap, d_gl, cond_loop, cond_serv, use_cond);
  else
    cg_update_batch_kernel<TM_F16><<<nu, BNT, 0, s>>>(L.sys, d_umap, d_gl, cond_loop, cond_serv, use_cond);
  count_launch();
  return cuda_check(cudaGetLastError(), "batched update kernel");
}

// The FP64 service of the stopped systems: X += x_s, r = b' - A X in FP64 (the normal operator's four
// hopping launches, K2 without its reduction, K4 storing ||r||^2), the decision, and the conversions
// of the resumed systems.  Systems that did not stop skip every launch.
static tm_status batch_service(const GroupLaunch& D, const BatchSys* d_sys, int sp, const int2* d_umap, int nu,
                               BatchGlobal* d_gl, cudaStream_t s) {
  tm_status st;
  serv_begin_kernel<<<nu, BNT, 0, s>>>(d_sys, D.sys, d_umap);
  count_launch();
  if ((st = cuda_check(cudaGetLastError(), "batched service")) != TM_OK) return st;
  // FP64 vectors: 0 X, 1 T, 2 W, 3 r
  if ((st = hop_batch(D, 0, 0, 1, 0, 0, 0, false, s)) != TM_OK) return st;
  if ((st = hop_batch(D, 1, 0, 2, 1, 1, 0, true, s)) != TM_OK) return st;
  if ((st = hop_batch(D, 2, 0, 1, 2, 0, 0, false, s)) != TM_OK) return st;
  if ((st = hop_batch(D, 1, 2, 3, 3, 1, 2, true, s)) != TM_OK) return st;
  serv_decide_kernel<<<1, 128, 0, s>>>(d_sys, d_gl);
  count_launch();
  if (sp == TM_F32)
    serv_convert_kernel<TM_F32><<<nu, BNT, 0, s>>>(d_sys, D.sys, d_umap);
  else
    serv_convert_kernel<TM_F16><<<nu, BNT, 0, s>>>(d_sys, D.sys, d_umap);
  count_launch();
  return cuda_check(cudaGetLastError(), "batched service");
}

namespace {

// TM_VERBOSE=1 traces the confirmation of each converged system
bool batch_verbose() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("TM_VERBOSE");
    v = (e && *e == '1') ? 1 : 0;
  }
  return v == 1;
}

struct SysWork {
  Solver S;
  tm_lattice lat;
  double mu;
  double* x;
  const double* b;
  // FP64 half fields
  void *be, *bo, *bp, *X;
  // FP32 and sloppy
  void *rs, *xs, *ps, *Ts, *Ws;
  double bb, bfull, rr, stop2;
  int iters, updates;
  bool converged;
  int lat_index;
};

struct LatWork {
  tm_lattice lat;
  void *R, *Pv, *T, *W;  // FP64 scratch for reliable updates and the final check
};

// Groups of up to K systems per lattice (in the order given) and the block map: for every
// lattice, for every block of its sites, the blocks of its groups one after another.
void build_groups(const std::vector<SysWork>& W, const std::vector<LatWork>& lats, int K,
                  std::vector<BatchGroup>& grp, std::vector<int2>& map) {
  grp.clear();
  map.clear();
  for (size_t li = 0; li < lats.size(); ++li) {
    std::vector<int> mine;
    const size_t g0 = grp.size();
    for (size_t k = 0; k < W.size(); ++k)
      if (W[k].lat_index == (int)li) mine.push_back((int)k);
    for (size_t a = 0; a < mine.size(); a += K) {
      BatchGroup G{};
      G.n = (int)std::min<size_t>(K, mine.size() - a);
      for (int j = 0; j < G.n; ++j) G.sys[j] = mine[a + j];
      grp.push_back(G);
    }
    const int nbl = (int)hop_grid_blocks(lats[li].lat->h, 1);
    for (int blk = 0; blk < nbl; ++blk)
      for (size_t g = g0; g < grp.size(); ++g) map.push_back(make_int2((int)g, blk));
  }
}

tm_status upload_groups(const std::vector<BatchGroup>& grp, const std::vector<int2>& map, GroupLaunch& L,
                        cudaStream_t s) {
  tm_status st = cuda_check(cudaMemcpyAsync(const_cast<BatchGroup*>(L.grp), grp.data(), sizeof(BatchGroup) * grp.size(),
                                            cudaMemcpyHostToDevice, s),
                            "table");
  if (st == TM_OK)
    st = cuda_check(cudaMemcpyAsync(const_cast<int2*>(L.map), map.data(), sizeof(int2) * map.size(),
                                    cudaMemcpyHostToDevice, s),
                    "table");
  L.nblocks = (int)map.size();
  return st;
}

// Systems per thread of the batched hopping kernel (K = 1, 2 or 4; the batch split of the
// systems of each lattice into groups).  TM_BATCH_K=1|2|4 fixes it.  Otherwise the candidates up
// to the largest number of systems on one lattice are timed on this batch's own vectors (a
// plain application of the hopping operator to every system, CUDA events, the fastest of three
// interleaved rounds of two launches each), and the fastest kept -- K > 1 must win by 3% -- and
// remembered for later batches of the same signature (storage form, each lattice's extents and
// number of systems).
int env_batch_k() {
  const char* e = getenv("TM_BATCH_K");
  if (!e) return 0;
  const int v = atoi(e);
  return (v == 1 || v == 2 || v == 4) ? v : 0;
}

tm_status choose_batch_k(const std::vector<SysWork>& W, const std::vector<LatWork>& lats, int sp, int sl,
                         GroupLaunch& L, cudaStream_t s) {
  static std::mutex mu;
  static std::vector<std::pair<std::vector<long long>, int>> cache;
  std::vector<long long> sig = {sp, sl};
  int most = 1;
  for (size_t li = 0; li < lats.size(); ++li) {
    int n = 0;
    for (auto& w : W) n += (w.lat_index == (int)li);
    most = std::max(most, n);
    sig.push_back(lats[li].lat->T);
    sig.push_back(lats[li].lat->L);
    sig.push_back(n);
  }
  int K = env_batch_k();
  if (K == 0) {
    std::lock_guard<std::mutex> lock(mu);
    for (auto& c : cache)
      if (c.first == sig) K = c.second;
  }
  std::vector<BatchGroup> grp;
  std::vector<int2> map;
  tm_status st = TM_OK;
  if (K == 0) {
    const int cands[3] = {1, 2, 4};
    float score[3] = {1e30f, 1e30f, 1e30f};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    st = cuda_check(cudaEventCreate(&e0), "event");
    if (st == TM_OK) st = cuda_check(cudaEventCreate(&e1), "event");
    for (int round = 0; round < 4 && st == TM_OK; ++round)
      for (int c = 0; c < 3 && st == TM_OK; ++c) {
        if (cands[c] > 1 && cands[c] > most) continue;
        build_groups(W, lats, cands[c], grp, map);
        L.K = cands[c];
        if ((st = upload_groups(grp, map, L, s)) != TM_OK) break;
        if ((st = cuda_check(cudaEventRecord(e0, s), "event")) != TM_OK) break;
        for (int q = 0; q < 2 && st == TM_OK; ++q) st = hop_batch(L, 0, 0, 1, 0, q & 1, 0, false, s);
        if (st == TM_OK) st = cuda_check(cudaEventRecord(e1, s), "event");
        if (st == TM_OK) st = cuda_check(cudaEventSynchronize(e1), "tuner");
        float ms = 0.f;
        if (st == TM_OK) st = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "event");
        if (round > 0 && ms < score[c]) score[c] = ms;  // round 0 warms up
      }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != TM_OK) return st;
    int bi = 0;
    for (int c = 1; c < 3; ++c)
      if (score[c] < 0.97f * score[bi]) bi = c;
    K = cands[bi];
    std::lock_guard<std::mutex> lock(mu);
    cache.emplace_back(sig, K);
  }
  build_groups(W, lats, K, grp, map);
  L.K = K;
  return upload_groups(grp, map, L, s);
}

}  // namespace

}  // namespace tmq

using namespace tmq;

extern "C" tm_status tm_solve_cg_batch(const tm_system* systems, int nsys, const tm_cg_params* params,
                                       tm_cg_info* infos, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!systems || nsys < 1) return set_error(TM_ERR_ARG, "tm_solve_cg_batch: no systems");
  tm_cg_params P;
  if (params)
    P = *params;
  else
    tm_cg_params_default(&P);
  if (P.mode != TM_CG_RELIABLE) return set_error(TM_ERR_UNSUPPORTED, "tm_solve_cg_batch: mode must be TM_CG_RELIABLE");
  if (P.sloppy_prec != TM_F32 && P.sloppy_prec != TM_F16)
    return set_error(TM_ERR_ARG, "tm_solve_cg_batch: sloppy precision must be TM_F32 or TM_F16");
  if (P.sloppy_link != 18 && P.sloppy_link != 12 && P.sloppy_link != 8)
    return set_error(TM_ERR_ARG, "tm_solve_cg_batch: sloppy link format %d", P.sloppy_link);
  if (!(P.tol > 0.0) || P.max_iter < 1 || !(P.delta > 0.0 && P.delta < 1.0))
    return set_error(TM_ERR_ARG, "tm_solve_cg_batch: tol > 0, max_iter >= 1, 0 < delta < 1");
  if (P.use_x0) return set_error(TM_ERR_UNSUPPORTED, "tm_solve_cg_batch: initial guesses are not supported");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int sp = P.sloppy_prec, sl = P.sloppy_link;

  // ---- validate systems, group by lattice
  std::vector<LatWork> lats;
  std::vector<SysWork> W(nsys);
  for (int k = 0; k < nsys; ++k) {
    const tm_system& y = systems[k];
    if (!y.lat || !y.x || !y.b) return set_error(TM_ERR_ARG, "tm_solve_cg_batch: system %d has a NULL member", k);
    if (!y.lat->has_gauge) return set_error(TM_ERR_NO_GAUGE, "tm_solve_cg_batch: system %d has no gauge field", k);
    const int f = y.flavour == 0 ? 1 : y.flavour;
    if (f != 1 && f != -1) return set_error(TM_ERR_ARG, "tm_solve_cg_batch: system %d flavour", k);
    if (!std::isfinite(y.mu)) return set_error(TM_ERR_ARG, "tm_solve_cg_batch: system %d mu", k);
    if (!is_device_pointer(y.x) || !is_device_pointer(y.b))
      return set_error(TM_ERR_ARG, "tm_solve_cg_batch: system %d: x and b must be device memory", k);
    int li = -1;
    for (size_t q = 0; q < lats.size(); ++q)
      if (lats[q].lat == y.lat) li = (int)q;
    if (li < 0) {
      lats.push_back(LatWork{y.lat, nullptr, nullptr, nullptr, nullptr});
      li = (int)lats.size() - 1;
    }
    SysWork& w = W[k];
    memset(&w, 0, sizeof(w));
    w.lat = y.lat;
    w.mu = y.mu;
    w.x = y.x;
    w.b = y.b;
    w.lat_index = li;
    w.S = Solver{y.lat, s, f, 2.0 * y.lat->kappa * y.mu, {0, 0, 0, 0}};
    for (int q = 0; q < 4; ++q) w.S.hb[q] = spinor_bytes_per_site(q) * y.lat->h;
  }
  tm_status st = TM_OK;
  for (auto& L : lats) {
    if ((st = ensure_links(L.lat, sp, sl, s)) != TM_OK) return st;
    if ((st = ensure_links(L.lat, TM_F64, 18, s)) != TM_OK) return st;
  }

  // ---- one allocation for every work field
  size_t total = 0;
  auto add = [&](size_t bytes) {
    const size_t off = total;
    total += (bytes + 255) / 256 * 256;
    return off;
  };
  std::vector<size_t> offs;
  for (auto& L : lats)
    for (int q = 0; q < 4; ++q) offs.push_back(add(spinor_bytes_per_site(TM_F64) * L.lat->h));
  for (auto& w : W) {
    const size_t h = w.lat->h;
    for (int q = 0; q < 7; ++q) offs.push_back(add(192 * h));  // be, bo, bp, X, T64, W64, R64
    for (int q = 0; q < 2; ++q) offs.push_back(add(96 * h));
    for (int q = 0; q < 3; ++q) offs.push_back(add(spinor_bytes_per_site(sp) * h));
  }
  // device tables (a block map has at most one entry per system and block of sites: K = 1)
  int npart = 0, nu = 0;
  for (auto& w : W) {
    npart += (int)hop_grid_blocks(w.lat->h, 1);
    nu += (int)blas_blocks(w.lat->geom.h);
  }
  const size_t off_sys = add(sizeof(BatchSys) * nsys);
  const size_t off_sys64 = add(sizeof(BatchSys) * nsys);
  const size_t off_grp = add(sizeof(BatchGroup) * nsys);
  const size_t off_grp1 = add(sizeof(BatchGroup) * nsys);
  const size_t off_hmap = add(sizeof(int2) * npart);
  const size_t off_hmap1 = add(sizeof(int2) * npart);
  const size_t off_umap = add(sizeof(int2) * nu);
  const size_t off_state = add(sizeof(CGState) * nsys);
  const size_t off_gl = add(sizeof(BatchGlobal));
  const size_t off_part = add(sizeof(double) * npart);
  const size_t off_ctr = add(sizeof(unsigned) * 2 * nsys);
  const size_t off_res = add(sizeof(double) * nsys);
  char* base = nullptr;
  if ((st = cuda_check(cudaMalloc(&base, total), "tm_solve_cg_batch: work space")) != TM_OK) return st;
  std::vector<BatchSys> hsys(nsys), hsys64(nsys);
  std::vector<CGState> hst(nsys);
  BatchGlobal hgl{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  tm_status result = TM_OK;
  std::vector<void*> T64(nsys), W64(nsys), R64(nsys);
  {
    size_t oi = 0;
    for (auto& L : lats) {
      L.R = base + offs[oi++];
      L.Pv = base + offs[oi++];
      L.T = base + offs[oi++];
      L.W = base + offs[oi++];
    }
    for (int k = 0; k < nsys; ++k) {
      SysWork& w = W[k];
      w.be = base + offs[oi++];
      w.bo = base + offs[oi++];
      w.bp = base + offs[oi++];
      w.X = base + offs[oi++];
      T64[k] = base + offs[oi++];
      W64[k] = base + offs[oi++];
      R64[k] = base + offs[oi++];
      w.rs = base + offs[oi++];
      w.xs = base + offs[oi++];
      w.ps = base + offs[oi++];
      w.Ts = base + offs[oi++];
      w.Ws = base + offs[oi++];
    }
  }
  BatchSys* d_sys = reinterpret_cast<BatchSys*>(base + off_sys);
  BatchSys* d_sys64 = reinterpret_cast<BatchSys*>(base + off_sys64);
  BatchGroup* d_grp = reinterpret_cast<BatchGroup*>(base + off_grp);
  BatchGroup* d_grp1 = reinterpret_cast<BatchGroup*>(base + off_grp1);
  int2* d_hmap = reinterpret_cast<int2*>(base + off_hmap);
  int2* d_hmap1 = reinterpret_cast<int2*>(base + off_hmap1);
  GroupLaunch GL{sp, sl, 1, d_sys, d_grp, d_hmap, 0};
  GroupLaunch GD{TM_F64, 18, 1, d_sys64, d_grp1, d_hmap1, 0};
  int2* d_umap = reinterpret_cast<int2*>(base + off_umap);
  CGState* d_st = reinterpret_cast<CGState*>(base + off_state);
  BatchGlobal* d_gl = reinterpret_cast<BatchGlobal*>(base + off_gl);
  double* d_part = reinterpret_cast<double*>(base + off_part);
  unsigned* d_ctr = reinterpret_cast<unsigned*>(base + off_ctr);
  double* d_res = reinterpret_cast<double*>(base + off_res);
  const double delta2 = P.delta * P.delta;
  int unfinished = 0;

  do {
    // ---- per system: source preparation (FP64), initial vectors
    for (int k = 0; k < nsys && st == TM_OK; ++k) {
      SysWork& w = W[k];
      LatWork& L = lats[w.lat_index];
      st = prepare_source(w.S, w.b, w.be, w.bo, w.bp, L.T, &w.bb, &w.bfull);
      if (st != TM_OK) break;
      if (!std::isfinite(w.bb) || !std::isfinite(w.bfull)) {
        st = set_error(TM_ERR_NONFINITE, "tm_solve_cg_batch: system %d has a non-finite source", k);
        break;
      }
      w.stop2 = P.tol * P.tol * w.bb;
      w.rr = w.bb;
      st = cuda_check(cudaMemsetAsync(w.X, 0, w.S.hb[TM_F64], s), "memset");
      if (st == TM_OK) st = cuda_check(cudaMemsetAsync(w.xs, 0, w.S.hb[TM_F32], s), "memset");
      if (st == TM_OK) st = convert_half(w.lat, TM_F32, w.rs, TM_F64, w.bp, s);
      if (st == TM_OK) st = convert_half(w.lat, sp, w.ps, TM_F64, w.bp, s);
      if (w.bfull == 0.0) w.converged = true;
    }
    if (st != TM_OK) break;
    // ---- descriptor tables; the blocks of the groups on one lattice interleaved site-block by
    // site-block, so the K systems of a group share each link in registers and the groups of a
    // lattice share it through L2
    {
      std::vector<int2> umap;
      int pfirst = 0;
      std::vector<int> first(nsys);
      for (int k = 0; k < nsys; ++k) {
        first[k] = pfirst;
        pfirst += (int)hop_grid_blocks(W[k].lat->h, 1);
      }
      for (size_t li = 0; li < lats.size(); ++li) {
        const int nub = (int)blas_blocks(lats[li].lat->geom.h);
        for (int blk = 0; blk < nub; ++blk)
          for (int k = 0; k < nsys; ++k)
            if (W[k].lat_index == (int)li) umap.push_back(make_int2(k, blk));
      }
      for (int k = 0; k < nsys; ++k) {
        SysWork& w = W[k];
        BatchSys& B = hsys[k];
        memset(&B, 0, sizeof(B));
        B.g = w.lat->geom;
        B.links = static_cast<const char*>(w.lat->links[sp][link_index(sl)]);
        B.coef[0] = epi_mdiag_inv_hop(w.S.mut, -w.S.f);
        B.coef[1] = epi_schur_q(w.lat->kappa, w.S.mut, -w.S.f);
        B.coef[2] = epi_mdiag_inv_hop(w.S.mut, w.S.f);
        B.coef[3] = epi_schur_q(w.lat->kappa, w.S.mut, w.S.f);
        B.vec[0] = w.ps;
        B.vec[1] = w.Ts;
        B.vec[2] = w.Ws;
        B.vec[3] = w.rs;
        B.vec[4] = w.xs;
        B.st = d_st + k;
        B.partials = d_part + first[k];
        B.counters = d_ctr + 2 * k;
        B.nblocks = (int)hop_grid_blocks(w.lat->h, 1);
        B.nblocks_upd = (int)blas_blocks(w.lat->geom.h);
        B.result = d_res + k;
        // the FP64 service's table: the FP64 gauge copy, X, T, W, r and b'
        BatchSys& D = hsys64[k];
        D = B;
        D.links = static_cast<const char*>(w.lat->links[TM_F64][link_index(18)]);
        D.vec[0] = w.X;
        D.vec[1] = T64[k];
        D.vec[2] = W64[k];
        D.vec[3] = R64[k];
        D.vec[4] = w.bp;
      }
      st = cuda_check(cudaMemcpyAsync(d_sys, hsys.data(), sizeof(BatchSys) * nsys, cudaMemcpyHostToDevice, s), "table");
      if (st == TM_OK)
        st = cuda_check(cudaMemcpyAsync(d_sys64, hsys64.data(), sizeof(BatchSys) * nsys, cudaMemcpyHostToDevice, s),
                        "table");
      if (st == TM_OK)
        st = cuda_check(cudaMemcpyAsync(d_umap, umap.data(), sizeof(int2) * nu, cudaMemcpyHostToDevice, s), "table");
      if (st == TM_OK) st = cuda_check(cudaMemsetAsync(d_ctr, 0, sizeof(unsigned) * 2 * nsys, s), "memset");
      // states with nothing stopped, for the tuner's launches
      for (int k = 0; k < nsys && st == TM_OK; ++k) hst[k] = fresh_state(W[k].rr, W[k].stop2, P.max_iter, 0, 0.0, 0.0);
      if (st == TM_OK)
        st = cuda_check(cudaMemcpyAsync(d_st, hst.data(), sizeof(CGState) * nsys, cudaMemcpyHostToDevice, s), "state");
      if (st == TM_OK) st = choose_batch_k(W, lats, sp, sl, GL, s);
      if (st == TM_OK) {  // the service's map: one system per group
        std::vector<BatchGroup> g1;
        std::vector<int2> m1;
        build_groups(W, lats, 1, g1, m1);
        st = upload_groups(g1, m1, GD, s);
      }
      if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "tables");
    }
    if (st != TM_OK) break;
    // ---- initial states: every system with a non-zero source iterates; the loop runs until every
    // system is finished (or the loop cap, which the iteration bound implies, is reached)
    unfinished = 0;
    for (int k = 0; k < nsys; ++k) {
      SysWork& w = W[k];
      hst[k] = fresh_state(w.rr, w.stop2, P.max_iter, 0, delta2, SLOPPY_GROWTH);
      if (w.converged) {  // zero source: x = 0
        hst[k].done = 1;
        hst[k].finished = 1;
        hst[k].ok = 1;
      } else {
        ++unfinished;
      }
    }
    hgl = BatchGlobal{unfinished, 0, P.max_iter + 16, 0u, nsys, 0, delta2, SLOPPY_GROWTH * SLOPPY_GROWTH};
    st = cuda_check(cudaMemcpyAsync(d_st, hst.data(), sizeof(CGState) * nsys, cudaMemcpyHostToDevice, s), "state");
    if (st == TM_OK) st = cuda_check(cudaMemcpyAsync(d_gl, &hgl, sizeof(hgl), cudaMemcpyHostToDevice, s), "state");
    if (st != TM_OK) break;
    // ---- the solve: ONE graph launch, a WHILE loop over { batched iteration; IF (a system stopped)
    // { FP64 service } }.  With TM_NO_GRAPH=1 the same kernels run from the host in chunks of 8
    // iterations, the service after every iteration (it skips the systems that did not stop).
    if (unfinished == 0) {  // every source is zero
    } else if (use_graphs()) {
      cudaGraphConditionalHandle cond_loop, cond_serv;
      cudaGraphNode_t node;
      cudaGraphNodeParams cp = {};
      const unsigned long long before = tm_launch_count();
      st = cuda_check(cudaGraphCreate(&graph, 0), "cudaGraphCreate");
      if (st == TM_OK)
        st = cuda_check(cudaGraphConditionalHandleCreate(&cond_loop, graph, 1, cudaGraphCondAssignDefault),
                        "conditional");
      if (st == TM_OK) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond_loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        st = cuda_check(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp), "conditional node");
      }
      cudaGraph_t body = nullptr;
      if (st == TM_OK) {
        body = cp.conditional.phGraph_out[0];
        st = cuda_check(cudaGraphConditionalHandleCreate(&cond_serv, body, 0, cudaGraphCondAssignDefault),
                        "conditional");
      }
      if (st == TM_OK) st = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
      cudaGraph_t serv_body = nullptr;
      if (st == TM_OK) {
        st = cuda_check(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                        "begin capture");
        if (st == TM_OK) {
          tm_status st1 = batch_iteration(GL, d_umap, nu, d_gl, cond_loop, cond_serv, 1, cs);
          // the IF node after the iteration, added to the graph being captured
          if (st1 == TM_OK) {
            cudaStreamCaptureStatus cst;
            cudaGraph_t capg = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            size_t ndeps = 0;
            st1 = cuda_check(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, nullptr, &ndeps), "capture info");
            cudaGraphNodeParams ip = {};
            ip.type = cudaGraphNodeTypeConditional;
            ip.conditional.handle = cond_serv;
            ip.conditional.type = cudaGraphCondTypeIf;
            ip.conditional.size = 1;
            cudaGraphNode_t ifnode;
            if (st1 == TM_OK)
              st1 = cuda_check(cudaGraphAddNode(&ifnode, capg, deps, nullptr, ndeps, &ip), "conditional node");
            if (st1 == TM_OK)
              st1 = cuda_check(cudaStreamUpdateCaptureDependencies(cs, &ifnode, nullptr, 1, cudaStreamSetCaptureDependencies),
                               "capture dependencies");
            if (st1 == TM_OK) serv_body = ip.conditional.phGraph_out[0];
          }
          cudaGraph_t captured = nullptr;
          tm_status st2 = cuda_check(cudaStreamEndCapture(cs, &captured), "end capture");
          st = st1 != TM_OK ? st1 : st2;
        }
      }
      if (st == TM_OK) {  // the service body
        st = cuda_check(cudaStreamBeginCaptureToGraph(cs, serv_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                        "begin capture");
        if (st == TM_OK) {
          tm_status st1 = batch_service(GD, d_sys, sp, d_umap, nu, d_gl, cs);
          cudaGraph_t captured = nullptr;
          tm_status st2 = cuda_check(cudaStreamEndCapture(cs, &captured), "end capture");
          st = st1 != TM_OK ? st1 : st2;
        }
      }
      if (st == TM_OK) st = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
      tm_reset_launch_count();
      count_launch((unsigned)before);
      if (st == TM_OK) st = cuda_check(cudaGraphLaunch(exec, s), "graph launch");
      if (st == TM_OK)
        st = cuda_check(cudaMemcpyAsync(hst.data(), d_st, sizeof(CGState) * nsys, cudaMemcpyDeviceToHost, s), "state");
      if (st == TM_OK) st = cuda_check(cudaMemcpyAsync(&hgl, d_gl, sizeof(hgl), cudaMemcpyDeviceToHost, s), "state");
      if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "batched solve");
      if (st != TM_OK) break;
      count_launch(5u * (unsigned)hgl.loops);
    } else {
      for (;;) {
        for (int q = 0; q < 8 && st == TM_OK; ++q) {
          st = batch_iteration(GL, d_umap, nu, d_gl, 0, 0, 0, s);
          if (st == TM_OK) st = batch_service(GD, d_sys, sp, d_umap, nu, d_gl, s);
        }
        if (st == TM_OK) st = cuda_check(cudaMemcpyAsync(&hgl, d_gl, sizeof(hgl), cudaMemcpyDeviceToHost, s), "state");
        if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "batched chunk");
        if (st != TM_OK || hgl.unfinished <= 0 || hgl.loops >= hgl.loop_cap) break;
      }
      if (st == TM_OK)
        st = cuda_check(cudaMemcpyAsync(hst.data(), d_st, sizeof(CGState) * nsys, cudaMemcpyDeviceToHost, s), "state");
      if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "batched solve");
      if (st != TM_OK) break;
    }
    for (int k = 0; k < nsys; ++k) {
      SysWork& w = W[k];
      const CGState& c = hst[k];
      if (w.bfull == 0.0) continue;
      w.converged = c.ok != 0;
      w.iters = c.iter;
      w.updates = c.updates;
      w.rr = c.rr64;
      if (batch_verbose())
        fprintf(stderr,
                "[tm_solve_cg_batch] system %d: %d iterations, %d FP64 residuals, %d sloppy convergences not "
                "confirmed, %s (FP64 |b' - A X|/|b'| %.3e); one graph launch for the batch: %s\n",
                k, c.iter, c.updates, c.missed, c.ok ? "converged" : "not converged",
                w.bb > 0 ? std::sqrt(c.rr64 / w.bb) : 0.0, exec ? "yes" : "no (host loop)");
    }
    // ---- reconstruction and FP64 check per system
    for (int k = 0; k < nsys && st == TM_OK; ++k) {
      SysWork& w = W[k];
      LatWork& L = lats[w.lat_index];
      tm_cg_info info{};
      info.iters = w.iters;
      info.reliable_updates = w.updates;
      info.schur_rel_residual = w.bb > 0.0 ? std::sqrt(w.rr / w.bb) : 0.0;
      if (w.bfull == 0.0) {
        st = cuda_check(cudaMemsetAsync(w.x, 0, w.lat->V * 24 * sizeof(double), s), "memset");
      } else {
        st = reconstruct_check(w.S, w.X, w.be, w.bo, w.bfull, w.x, L.T, L.W, L.R, L.Pv, &info.true_rel_residual);
      }
      info.status = w.converged ? TM_OK : TM_ERR_NOT_CONVERGED;
      if (!w.converged) result = TM_ERR_NOT_CONVERGED;
      if (infos) infos[k] = info;
    }
    if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "synchronise");
  } while (false);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cs) cudaStreamDestroy(cs);
  cudaFree(base);
  if (st != TM_OK) return st;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (infos)
    for (int k = 0; k < nsys; ++k) infos[k].seconds = secs;
  if (result != TM_OK) return set_error(result, "tm_solve_cg_batch: some systems did not converge");
  return TM_OK;
}
