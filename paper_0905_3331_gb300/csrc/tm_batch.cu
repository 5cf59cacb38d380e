// tm_batch.cu -- many systems M_s^f x_s = b_s solved together (tm_solve_cg_batch).
//
// Systems may differ in source, twisted mass and lattice (geometry and gauge field).  Every
// system runs the mixed-precision reliable-update CG of tm_solver.cu, but the sloppy
// iterations of all systems go through the same kernels: one launch of K1..K4 and of the
// update covers every running system, its blocks mapped to (system, block of sites) by a work
// list rebuilt inside the graph, with the blocks of systems that share a lattice interleaved so
// that each link is fetched from HBM once and served to the other systems from L2.  The hopping
// launches run the single-system kernel's body per system (1, 2 or 4 threads per site) or K = 2,
// 4 systems per thread (tm_batch_group.cu), as a tuner picks per batch shape.  Each system keeps its own device-side
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

#include "tm_batch.cuh"
#include "tm_solver.cuh"

namespace tmq {

// Rebuilds a work list (one warp, all lanes): the candidates of a lattice are taken 32 at a time
// and compacted with a ballot, one round of dependent loads per 32 candidates.
// Candidates: the positions in `order` (systems; groups == nullptr), or the group ids.
__device__ void plan_build(const Plan& P, const int* order, const CGState* st, bool stopped,
                           const BatchGroup* groups = nullptr) {
  const unsigned lane = threadIdx.x & 31u;
  int v = 0;
  for (int li = 0; li < P.nlat; ++li) {
    const int b0 = P.base[li], nc = P.ncand[li];
    int n = 0;
    for (int c0 = 0; c0 < nc; c0 += 32) {
      const int c = c0 + (int)lane;
      int id = -1;
      if (c < nc && groups) {  // a group runs while one of its systems does
        const BatchGroup G = groups[b0 + c];
        for (int j = 0; j < G.n; ++j)
          if (!st[G.sys[j]].done) id = b0 + c;
      } else if (c < nc) {
        const int k = order[b0 + c];
        const CGState& q = st[k];
        if (stopped ? (q.done && !q.finished) : !q.done) id = k;
      }
      const unsigned live = __ballot_sync(0xffffffffu, id >= 0);
      if (id >= 0) P.items[b0 + n + __popc(live & ((1u << lane) - 1u))] = id;
      n += __popc(live);
    }
    if (lane == 0) {
      P.start[li] = v;
      P.count[li] = n;
    }
    v += n * P.blocks[li];
  }
  if (lane == 0) P.start[P.nlat] = v;
}

// Work list w (0 hop, 1 upd: the running systems; 2 shop, 3 supd: the systems that stopped and are
// not finished; 4 ghop: the running groups), rebuilt by one warp from the states as they stand.
constexpr int NPLANS = 5;
__device__ void plan_rebuild(const Plans& L, int w) {
  if (w == 4) {
    plan_build(L.ghop, L.order, L.states, false, L.groups);
    return;
  }
  const Plan& P = w == 0 ? L.hop : (w == 1 ? L.upd : (w == 2 ? L.shop : L.supd));
  plan_build(P, L.order, L.states, w >= 2);
}

// All five (before the solve, and for the tuner); one warp each.
__global__ void plans_init_kernel(Plans L) {
  const int w = threadIdx.x >> 5;
  if (w < NPLANS) plan_rebuild(L, w);
}

// The batched hopping kernel: the blocks of the listed systems, each computed by the hopping
// kernels' own body (TPS threads per site, hop_spb(TPS) sites per block) on that system's fields,
// epilogue coefficients (its mu), CG state and reduction.  serv = 0: the running systems, sloppy
// storage; serv = 1: the FP64 service of stopped systems, where K4's residual update uses alpha = 1
// (r = b' - A X from r = b') and the reduction stores ||r||^2 in B.result.  A system that stopped
// since the list was built (a breakdown in K2) is skipped.
constexpr int hop_batch_min_blocks(int prec, int nreal, int tps) {
  return (tps == 1 && (prec == TM_F32 || prec == TM_F16)) ? 512 / hop_spb(1) : 1;  // 8 blocks of 64 (128 registers)
}

template <int PREC, int NREAL, bool HAS_Y, int MODE, int TPS>
__global__ void __launch_bounds__(hop_spb(TPS) * TPS, hop_batch_min_blocks(PREC, NREAL, TPS))
    hop_batch_kernel(const BatchSys* __restrict__ systems, const CGState* __restrict__ states, Plan plan, int serv,
                     int in_sel, int y_sel, int out_sel, int kk, int out_parity) {
  const int total = plan.start[plan.nlat];
  for (int v = blockIdx.x; v < total; v += gridDim.x) {
    const int2 m = plan_item(plan, v);
    const CGState& S = states[m.x];
    if (serv ? !(S.done && !S.finished) : S.done) continue;  // block-uniform
    const BatchSys& B = systems[m.x];
    const Reduce red{B.partials, B.counters, B.result, B.st, serv ? FIN_STORE : (MODE == 1 ? FIN_CG_ALPHA : FIN_CG_RR)};
    hop_sites<PREC, NREAL, HAS_Y, MODE, TPS, false, ListBlock, hop_spb(TPS)>(
        B.g, out_parity, B.links, B.vec[in_sel], 0, B.vec[out_sel], 0, B.vec[y_sel], 0, B.coef[kk],
        serv ? nullptr : B.st, 1.0, red, ListBlock{m.y, B.nblocks});
    __syncthreads();  // the body's shared memory is reused by the next block
  }
}

// x += alpha p, p = r + beta p per system.  The last block of all rebuilds the work lists (the
// running systems for the next iteration, the stopped ones for the service) and sets the graph's
// conditions: the loop runs again while a system is not finished (and below the loop cap), and
// the FP64 service runs when a system has stopped (its reliable-update trigger, convergence of the
// sloppy residual, divergence, a non-finite value, or its iteration bound).
template <int PP>
__global__ void __launch_bounds__(BNT) cg_update_batch_kernel(const BatchSys* __restrict__ systems, Plans L,
                                                              BatchGlobal* gl, cudaGraphConditionalHandle cond_loop,
                                                              cudaGraphConditionalHandle cond_serv, int use_cond) {
  typedef typename SpinorFmt<PP>::real RP;
  const int total = L.upd.start[L.upd.nlat];
  for (int v = blockIdx.x; v < total; v += gridDim.x) {
    const int2 m = plan_item(L.upd, v);
    const BatchSys& B = systems[m.x];
    CGState& S = L.states[m.x];
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
    __syncthreads();  // every thread has read `applied` before the last block of the system sets it
    if (threadIdx.x == 0 && work && arrive_acq_rel(B.counters + 1) == (unsigned)B.nblocks_upd - 1) {
      S.applied = iter;
      B.counters[1] = 0u;
    }
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) last = arrive_acq_rel(&gl->counter) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  // the last block: every block's work is visible; warps 0..4 rebuild the five work lists
  if ((threadIdx.x >> 5) < NPLANS) plan_rebuild(L, threadIdx.x >> 5);
  __syncthreads();
  if (threadIdx.x == 0) {
    gl->counter = 0u;
    gl->loops += 1;
    if (use_cond) {
      cudaGraphSetConditional(cond_serv, L.supd.start[L.supd.nlat] > 0 ? 1u : 0u);
      cudaGraphSetConditional(cond_loop, (gl->unfinished > 0 && gl->loops < gl->loop_cap) ? 1u : 0u);
    }
  }
}

// ---- the FP64 service of the systems that stopped (all inside the solve's graph)
// 1. X (FP64) += x_s (FP32; dropped after a non-finite value), x_s = 0; r (FP64) = b'.
__global__ void __launch_bounds__(BNT) serv_begin_kernel(const BatchSys* __restrict__ sys, const BatchSys* __restrict__ sys64,
                                                         Plan supd) {
  const int total = supd.start[supd.nlat];
  for (int v = blockIdx.x; v < total; v += gridDim.x) {
    const int2 m = plan_item(supd, v);
    const BatchSys& B = sys[m.x];
    const BatchSys& D = sys64[m.x];
    const CGState& S = *B.st;
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
}

// 3. The decision per stopped system, from its FP64 residual rr64 = ||b' - A X||^2 (one block);
// then the running systems' work lists, with the resumed systems in them.
__global__ void serv_decide_kernel(const BatchSys* __restrict__ sys, Plans L,
                                   BatchGlobal* gl) {
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
  __syncthreads();
  const int w = threadIdx.x >> 5;  // the running systems' lists (hop, upd, ghop)
  if (w < 2 || w == 4) plan_rebuild(L, w);
  if (threadIdx.x == 0) gl->services += 1;
}

// 4. r_s (FP32) = r, and p = r (sloppy) for a restart, for the systems the decision resumed.
template <int PP>
__global__ void __launch_bounds__(BNT) serv_convert_kernel(const BatchSys* __restrict__ sys,
                                                           const BatchSys* __restrict__ sys64, Plan supd) {
  const int total = supd.start[supd.nlat];
  for (int v = blockIdx.x; v < total; v += gridDim.x) {
    const int2 m = plan_item(supd, v);
    const BatchSys& B = sys[m.x];
    const CGState& S = *B.st;
    if (!S.rearm) continue;
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
}

template <int PREC, int NREAL, int TPS>
static tm_status launch_hop_batch(const BatchSys* d_sys, const CGState* d_st, const Plan& plan, int cap, int serv,
                                  int in_sel, int y_sel, int out_sel, int kk, int parity, int mode, bool has_y,
                                  cudaStream_t s) {
  constexpr int NT = hop_spb(TPS) * TPS;
#define TM_GL(HY, MD)                                                                                  \
  {                                                                                                    \
    auto kern = hop_batch_kernel<PREC, NREAL, HY, MD, TPS>;                                            \
    kern<<<resident_grid(kern, NT, cap), NT, 0, s>>>(d_sys, d_st, plan, serv, in_sel, y_sel, out_sel, kk, \
                                                     parity);                                          \
  }
  if (!has_y && mode == 0)
    TM_GL(false, 0)
  else if (has_y && mode == 0)
    TM_GL(true, 0)
  else if (has_y && mode == 1)
    TM_GL(true, 1)
  else
    TM_GL(true, 2)
#undef TM_GL
  count_launch();
  return cuda_check(cudaGetLastError(), "batched hopping kernel");
}

// The batched hopping launches of one storage form: TPS threads per site (K = 1), or K = 2, 4
// systems per thread over the groups (FP64 with TPS 1 for the service of stopped systems).
struct BatchLaunch {
  int prec, nreal, tps;
  int serv;
  const BatchSys* sys;
  const CGState* st;
  Plan plan;
  int cap;  // blocks of the full list
  int K;                    // systems per thread
  const BatchGroup* grp;    // the groups (K > 1)
  Plan gplan;               // their work list
};

static tm_status hop_batch(const BatchLaunch& L, int in_sel, int y_sel, int out_sel, int kk, int parity, int mode,
                           bool has_y, cudaStream_t s) {
  if (L.K > 1)
    return launch_hop_group(L.prec, L.nreal, L.K, L.sys, L.grp, L.st, L.gplan, L.cap, in_sel, y_sel, out_sel, kk,
                            parity, mode, has_y, s);
  if (L.prec == TM_F64)
    return launch_hop_batch<TM_F64, 18, 1>(L.sys, L.st, L.plan, L.cap, L.serv, in_sel, y_sel, out_sel, kk, parity, mode,
                                           has_y, s);
#define TM_B(P, N, T)                                                                                      \
  if (L.prec == P && L.nreal == N && L.tps == T)                                                          \
    return launch_hop_batch<P, N, T>(L.sys, L.st, L.plan, L.cap, L.serv, in_sel, y_sel, out_sel, kk, parity, mode, \
                                     has_y, s);
#define TM_BT(P, N) TM_B(P, N, 1) TM_B(P, N, 2) TM_B(P, N, 4)
  TM_BT(TM_F32, 18) TM_BT(TM_F32, 12) TM_BT(TM_F32, 8) TM_BT(TM_F16, 18) TM_BT(TM_F16, 12) TM_BT(TM_F16, 8)
#undef TM_BT
#undef TM_B
  return set_error(TM_ERR_UNSUPPORTED, "batched solve: sloppy form not supported");
}

// One batched CG iteration: K1..K4 of every running system, then the update (which rebuilds the
// work lists and sets the graph conditions).
static tm_status batch_iteration(const BatchLaunch& L, const Plans& plans, int ucap, BatchGlobal* d_gl,
                                 cudaGraphConditionalHandle cond_loop, cudaGraphConditionalHandle cond_serv,
                                 int use_cond, cudaStream_t s) {
  tm_status st;
  // K1: T = (M_ee^-f)^-1 H_eo p ; K2: W = Qhat^-f p, <p,Ap> ; K3: T = (M_ee^f)^-1 H_eo W ; K4: r -= alpha Qhat^f W
  if ((st = hop_batch(L, 0, 0, 1, 0, 0, 0, false, s)) != TM_OK) return st;
  if ((st = hop_batch(L, 1, 0, 2, 1, 1, 1, true, s)) != TM_OK) return st;
  if ((st = hop_batch(L, 2, 0, 1, 2, 0, 0, false, s)) != TM_OK) return st;
  if ((st = hop_batch(L, 1, 2, 3, 3, 1, 2, true, s)) != TM_OK) return st;
  if (L.prec == TM_F32) {
    auto kern = cg_update_batch_kernel<TM_F32>;
    kern<<<resident_grid(kern, BNT, ucap), BNT, 0, s>>>(L.sys, plans, d_gl, cond_loop, cond_serv, use_cond);
  } else {
    auto kern = cg_update_batch_kernel<TM_F16>;
    kern<<<resident_grid(kern, BNT, ucap), BNT, 0, s>>>(L.sys, plans, d_gl, cond_loop, cond_serv, use_cond);
  }
  count_launch();
  return cuda_check(cudaGetLastError(), "batched update kernel");
}

// The FP64 service of the stopped systems: X += x_s, r = b' - A X in FP64 (the normal operator's four
// hopping launches, K2 without its reduction, K4 storing ||r||^2), the decision, and the conversions
// of the resumed systems.  Each launch walks the stopped systems' work lists only.
static tm_status batch_service(const BatchLaunch& D, const BatchSys* d_sys, int sp,
                               const Plans& plans, int ucap, BatchGlobal* d_gl, cudaStream_t s) {
  tm_status st;
  serv_begin_kernel<<<resident_grid(serv_begin_kernel, BNT, ucap), BNT, 0, s>>>(d_sys, D.sys, plans.supd);
  count_launch();
  if ((st = cuda_check(cudaGetLastError(), "batched service")) != TM_OK) return st;
  // FP64 vectors: 0 X, 1 T, 2 W, 3 r
  if ((st = hop_batch(D, 0, 0, 1, 0, 0, 0, false, s)) != TM_OK) return st;
  if ((st = hop_batch(D, 1, 0, 2, 1, 1, 0, true, s)) != TM_OK) return st;
  if ((st = hop_batch(D, 2, 0, 1, 2, 0, 0, false, s)) != TM_OK) return st;
  if ((st = hop_batch(D, 1, 2, 3, 3, 1, 2, true, s)) != TM_OK) return st;
  serv_decide_kernel<<<1, 32 * NPLANS, 0, s>>>(d_sys, plans, d_gl);
  count_launch();
  if (sp == TM_F32) {
    auto kern = serv_convert_kernel<TM_F32>;
    kern<<<resident_grid(kern, BNT, ucap), BNT, 0, s>>>(d_sys, D.sys, plans.supd);
  } else {
    auto kern = serv_convert_kernel<TM_F16>;
    kern<<<resident_grid(kern, BNT, ucap), BNT, 0, s>>>(d_sys, D.sys, plans.supd);
  }
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

// The batch by lattice, and the device arrays of its work lists.  Device ints, in this order:
// order[nsys]; per lattice sys_base, sys_cnt, hop_blk (blocks per system of the sloppy hopping
// launch), upd_blk (of the update), shop_blk (of the FP64 service's hopping launch), grp_base,
// grp_cnt (the groups of K systems), ghop_blk (blocks per group); then for each of the five lists
// start[nlat + 1], count[nlat], items[nsys].
struct BatchLayout {
  static constexpr int NPER = 8;
  int nlat = 0, nsys = 0;
  std::vector<int> host;  // the static part (order and the per-lattice arrays)
  int* dev = nullptr;
  CGState* states = nullptr;
  BatchGroup* groups = nullptr;  // device, nsys entries at most
  static size_t ints(int nlat, int nsys) {
    return (size_t)nsys + NPER * nlat + NPLANS * ((size_t)2 * nlat + 1 + nsys);
  }
  int* at(int q) const { return dev + nsys + q * nlat; }        // q-th per-lattice array (device)
  int& hat(int q, int li) { return host[nsys + q * nlat + li]; }  // ... and its host copy
  Plans plans() const {
    Plans L;
    int* dyn = dev + nsys + NPER * nlat;
    Plan* all[NPLANS] = {&L.hop, &L.upd, &L.shop, &L.supd, &L.ghop};
    const int blocks[NPLANS] = {2, 3, 4, 3, 7};
    for (int q = 0; q < NPLANS; ++q) {
      Plan& P = *all[q];
      P.nlat = nlat;
      P.base = at(q == 4 ? 5 : 0);   // the groups' lists: grp_base, grp_cnt
      P.ncand = at(q == 4 ? 6 : 1);
      P.blocks = at(blocks[q]);
      P.start = dyn;
      P.count = dyn + nlat + 1;
      P.items = dyn + 2 * nlat + 1;
      dyn += 2 * nlat + 1 + nsys;
    }
    L.order = dev;
    L.states = states;
    L.groups = groups;
    return L;
  }
  tm_status upload(cudaStream_t s) const {
    tm_status st = cuda_check(cudaMemcpyAsync(dev, host.data(), sizeof(int) * host.size(), cudaMemcpyHostToDevice, s),
                              "work lists");
    if (st != TM_OK) return st;
    plans_init_kernel<<<1, 32 * NPLANS, 0, s>>>(plans());
    count_launch();
    return cuda_check(cudaGetLastError(), "work lists");
  }
};

// The batch split of the sloppy hopping launch: K = 1 with TPS threads per site (1, 2 or 4;
// hop_spb(TPS) sites per block), or K = 2, 4 systems per thread (HOP_NT sites per block) over
// groups of K systems of one lattice.  Sets the blocks per system (and group) in the layout and
// the system table, builds the groups, and uploads them.
tm_status set_batch_split(int K, int tps, const std::vector<SysWork>& W, const std::vector<LatWork>& lats,
                          BatchLayout& Y, std::vector<BatchSys>& hsys, BatchSys* d_sys, BatchLaunch& L,
                          cudaStream_t s) {
  const int spb = K > 1 ? HOP_NT : hop_spb(tps);
  std::vector<BatchGroup> grp;
  for (int li = 0; li < Y.nlat; ++li) {
    const int nbl = (int)((lats[li].lat->h + spb - 1) / spb);
    Y.hat(2, li) = nbl;
    Y.hat(7, li) = nbl;
    Y.hat(5, li) = (int)grp.size();
    const int first = Y.hat(0, li), n = Y.hat(1, li);
    for (int a = 0; a < n; a += K) {  // the lattice's systems in order, K to a group
      BatchGroup G{};
      G.n = std::min(K, n - a);
      for (int j = 0; j < G.n; ++j) G.sys[j] = Y.host[first + a + j];
      grp.push_back(G);
    }
    Y.hat(6, li) = (int)grp.size() - Y.hat(5, li);
  }
  for (size_t k = 0; k < W.size(); ++k) hsys[k].nblocks = (int)((W[k].lat->h + spb - 1) / spb);
  L.tps = K > 1 ? 1 : tps;
  L.K = K;
  tm_status st = cuda_check(
      cudaMemcpyAsync(d_sys, hsys.data(), sizeof(BatchSys) * hsys.size(), cudaMemcpyHostToDevice, s), "table");
  if (st == TM_OK)
    st = cuda_check(cudaMemcpyAsync(Y.groups, grp.data(), sizeof(BatchGroup) * grp.size(), cudaMemcpyHostToDevice, s),
                    "groups");
  return st == TM_OK ? Y.upload(s) : st;
}

// The batch split of the batched hopping kernel.  TM_BATCH_TPS=1|2|4 fixes one system per thread
// with that many threads per site, TM_BATCH_K=2|4 that many systems per thread.  Otherwise the
// candidates -- (K = 1; 1, 2, 4 threads per site), K = 2, K = 4 (up to the most systems on one
// lattice) -- are timed on this batch's own vectors (a plain application of the hopping operator
// to every system, CUDA events, the fastest of three interleaved rounds of two launches each) and
// the fastest kept (another candidate must win by 3% over one thread per site and K = 1), and
// remembered for later batches of the same signature (storage form, each lattice's extents and
// number of systems).
int env_batch(const char* name, bool allow2, bool allow4) {
  const char* e = getenv(name);
  if (!e) return 0;
  const int v = atoi(e);
  return (v == 1 || (v == 2 && allow2) || (v == 4 && allow4)) ? v : 0;
}

tm_status choose_batch_split(const std::vector<SysWork>& W, const std::vector<LatWork>& lats, int sp, int sl,
                             BatchLayout& Y, std::vector<BatchSys>& hsys, BatchSys* d_sys, BatchLaunch& L,
                             cudaStream_t s) {
  static std::mutex mu;
  static std::vector<std::pair<std::vector<long long>, std::pair<int, int>>> cache;
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
  int K = 0, tps = 0;
  if (const int ek = env_batch("TM_BATCH_K", true, true)) {
    K = ek;
    tps = 1;
  } else if (const int et = env_batch("TM_BATCH_TPS", true, true)) {
    K = 1;
    tps = et;
  } else {
    std::lock_guard<std::mutex> lock(mu);
    for (auto& c : cache)
      if (c.first == sig) {
        K = c.second.first;
        tps = c.second.second;
      }
  }
  tm_status st = TM_OK;
  if (K == 0) {
    const int candK[5] = {1, 1, 1, 2, 4}, candT[5] = {1, 2, 4, 1, 1};
    float score[5] = {1e30f, 1e30f, 1e30f, 1e30f, 1e30f};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    st = cuda_check(cudaEventCreate(&e0), "event");
    if (st == TM_OK) st = cuda_check(cudaEventCreate(&e1), "event");
    for (int round = 0; round < 4 && st == TM_OK; ++round)
      for (int c = 0; c < 5 && st == TM_OK; ++c) {
        if (candK[c] > most) continue;
        if ((st = set_batch_split(candK[c], candT[c], W, lats, Y, hsys, d_sys, L, s)) != TM_OK) break;
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
    for (int c = 1; c < 5; ++c)
      if (score[c] < 0.97f * score[0] && score[c] < score[bi]) bi = c;
    K = candK[bi];
    tps = candT[bi];
    if (batch_verbose())
      fprintf(stderr,
              "[tm_solve_cg_batch] split tuner (ms for two launches): K1/TPS1 %.3f, K1/TPS2 %.3f, K1/TPS4 %.3f, "
              "K2 %.3f, K4 %.3f -> K%d TPS%d\n",
              score[0], score[1], score[2], score[3] < 1e29f ? score[3] : 0.f, score[4] < 1e29f ? score[4] : 0.f,
              K, tps);
    std::lock_guard<std::mutex> lock(mu);
    cache.emplace_back(sig, std::make_pair(K, tps));
  }
  return set_batch_split(K, tps, W, lats, Y, hsys, d_sys, L, s);
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
  // device tables; npart bounds the blocks of a full hopping work list (32 sites per block at
  // least) and so the reduction partials, nu is the blocks of a full update work list
  int npart = 0, nu = 0;
  std::vector<int> first(nsys);
  for (int k = 0; k < nsys; ++k) {
    first[k] = npart;
    npart += (int)((W[k].lat->h + 31) / 32);
    nu += (int)blas_blocks(W[k].lat->geom.h);
  }
  const size_t off_sys = add(sizeof(BatchSys) * nsys);
  const size_t off_sys64 = add(sizeof(BatchSys) * nsys);
  const size_t off_ints = add(sizeof(int) * BatchLayout::ints((int)lats.size(), nsys));
  const size_t off_grp = add(sizeof(BatchGroup) * nsys);
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
  BatchLayout Y;
  Y.nlat = (int)lats.size();
  Y.nsys = nsys;
  Y.dev = reinterpret_cast<int*>(base + off_ints);
  Y.states = reinterpret_cast<CGState*>(base + off_state);
  Y.groups = reinterpret_cast<BatchGroup*>(base + off_grp);
  Y.host.assign((size_t)nsys + BatchLayout::NPER * Y.nlat, 0);
  for (int li = 0, c = 0; li < Y.nlat; ++li) {  // order, sys_base, sys_cnt, hop_blk, upd_blk, shop_blk
    Y.hat(0, li) = c;
    for (int k = 0; k < nsys; ++k)
      if (W[k].lat_index == li) Y.host[c++] = k;
    Y.hat(1, li) = c - Y.hat(0, li);
    Y.hat(2, li) = (int)((lats[li].lat->h + hop_spb(1) - 1) / hop_spb(1));
    Y.hat(3, li) = (int)blas_blocks(lats[li].lat->geom.h);
    Y.hat(4, li) = (int)((lats[li].lat->h + hop_spb(1) - 1) / hop_spb(1));
  }
  const Plans plans = Y.plans();
  BatchLaunch GL{sp, sl, 1, 0, d_sys, plans.states, plans.hop, npart, 1, Y.groups, plans.ghop};
  BatchLaunch GD{TM_F64, 18, 1, 1, d_sys64, plans.states, plans.shop, npart, 1, nullptr, plans.ghop};
  CGState* d_st = reinterpret_cast<CGState*>(base + off_state);
  BatchGlobal* d_gl = reinterpret_cast<BatchGlobal*>(base + off_gl);
  double* d_part = reinterpret_cast<double*>(base + off_part);
  unsigned* d_ctr = reinterpret_cast<unsigned*>(base + off_ctr);
  double* d_res = reinterpret_cast<double*>(base + off_res);
  const double delta2 = P.delta * P.delta;
  int unfinished = 0;
  // TM_VERBOSE=1: the host time of each phase (the stream synchronised at each mark)
  char phases[256] = "";
  auto tprev = std::chrono::steady_clock::now();
  auto mark = [&](const char* name) {
    if (!batch_verbose()) return;
    cudaStreamSynchronize(s);
    const auto now = std::chrono::steady_clock::now();
    const size_t n = strlen(phases);
    snprintf(phases + n, sizeof(phases) - n, " %s %.2f ms", name,
             std::chrono::duration<double, std::milli>(now - tprev).count());
    tprev = now;
  };

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
    mark("sources");
    // ---- descriptor tables, groups and work lists
    {
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
        B.nblocks = (int)((w.lat->h + hop_spb(1) - 1) / hop_spb(1));  // the FP64 service's; the sloppy per TPS
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
      if (st == TM_OK) st = cuda_check(cudaMemsetAsync(d_ctr, 0, sizeof(unsigned) * 2 * nsys, s), "memset");
      // states with nothing stopped, for the tuner's launches
      for (int k = 0; k < nsys && st == TM_OK; ++k) hst[k] = fresh_state(W[k].rr, W[k].stop2, P.max_iter, 0, 0.0, 0.0);
      if (st == TM_OK)
        st = cuda_check(cudaMemcpyAsync(d_st, hst.data(), sizeof(CGState) * nsys, cudaMemcpyHostToDevice, s), "state");
      if (st == TM_OK) st = choose_batch_split(W, lats, sp, sl, Y, hsys, d_sys, GL, s);
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
    if (st == TM_OK) {
      plans_init_kernel<<<1, 32 * NPLANS, 0, s>>>(plans);
      count_launch();
      st = cuda_check(cudaGetLastError(), "work lists");
    }
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
          tm_status st1 = batch_iteration(GL, plans, nu, d_gl, cond_loop, cond_serv, 1, cs);
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
          tm_status st1 = batch_service(GD, d_sys, sp, plans, nu, d_gl, cs);
          cudaGraph_t captured = nullptr;
          tm_status st2 = cuda_check(cudaStreamEndCapture(cs, &captured), "end capture");
          st = st1 != TM_OK ? st1 : st2;
        }
      }
      if (st == TM_OK) st = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
      mark("tables+graph");
      tm_reset_launch_count();
      count_launch((unsigned)before);
      if (st == TM_OK) st = cuda_check(cudaGraphLaunch(exec, s), "graph launch");
      if (st == TM_OK)
        st = cuda_check(cudaMemcpyAsync(hst.data(), d_st, sizeof(CGState) * nsys, cudaMemcpyDeviceToHost, s), "state");
      if (st == TM_OK) st = cuda_check(cudaMemcpyAsync(&hgl, d_gl, sizeof(hgl), cudaMemcpyDeviceToHost, s), "state");
      if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "batched solve");
      if (st != TM_OK) break;
      mark("solve");
      count_launch(5u * (unsigned)hgl.loops + 7u * (unsigned)hgl.services);
    } else {
      mark("tables");
      for (;;) {
        for (int q = 0; q < 8 && st == TM_OK; ++q) {
          st = batch_iteration(GL, plans, nu, d_gl, 0, 0, 0, s);
          if (st == TM_OK) st = batch_service(GD, d_sys, sp, plans, nu, d_gl, s);
        }
        if (st == TM_OK) st = cuda_check(cudaMemcpyAsync(&hgl, d_gl, sizeof(hgl), cudaMemcpyDeviceToHost, s), "state");
        if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "batched chunk");
        if (st != TM_OK || hgl.unfinished <= 0 || hgl.loops >= hgl.loop_cap) break;
      }
      if (st == TM_OK)
        st = cuda_check(cudaMemcpyAsync(hst.data(), d_st, sizeof(CGState) * nsys, cudaMemcpyDeviceToHost, s), "state");
      if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "batched solve");
      if (st != TM_OK) break;
      mark("solve");
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
    mark("reconstruction");
    if (batch_verbose())
      fprintf(stderr, "[tm_solve_cg_batch] %d loops, %d FP64 services;%s\n", hgl.loops, hgl.services, phases);
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
