// tm_batch.cu -- many systems M_s^f x_s = b_s solved together (tm_solve_cg_batch).
//
// Systems may differ in source, twisted mass and lattice (geometry and gauge field).  Every
// system runs the mixed-precision reliable-update CG of tm_solver.cu, but the sloppy
// iterations of all systems go through the same kernels: one launch of K1..K4 and of the
// update covers every system, its blocks mapped to (system, block of sites) by a table, with
// the blocks of systems that share a lattice interleaved so that each link is fetched from
// HBM once and served to the other systems from L2.  Each system keeps its own device-side
// CG state and reductions; a system that reaches its reliable-update trigger (or converges)
// idles while the others continue.  A stage -- iterations until every system has reached its
// trigger -- is one CUDA graph launch (a WHILE node over one batched iteration).  Between
// stages the host performs the FP64 reliable updates of the systems that need them.
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
};

struct BatchGlobal {
  int active;        // systems still iterating in this stage
  int loops;         // iteration bodies executed
  int loop_cap;      // hard bound on loops
  unsigned counter;  // update-kernel blocks arrived
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
// K = 4 (the accumulators of K spinors).
template <int PREC, int NREAL, bool HAS_Y, int MODE, int K>
__global__ void __launch_bounds__(HOP_NT, (K == 1 ? 6 : (K == 2 ? 4 : 2)))
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
    live[j] = j < G.n && !S[j]->st->done;
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
        const R al = (R)st->alpha;
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
      const Reduce red{B.partials, B.counters, nullptr, st, MODE == 1 ? FIN_CG_ALPHA : FIN_CG_RR};
      const double bs = block_sum<HOP_NT>((double)nrm, sh);
      grid_reduce<HOP_NT>(red, 0, B.nblocks, m.y, bs, sh);
      __syncthreads();  // sh and the reduction's shared flag are reused by the next system
    }
  }
}

// x += alpha p, p = r + beta p per system; the last block of all sets the loop condition.
template <int PP>
__global__ void __launch_bounds__(BNT) cg_update_batch_kernel(const BatchSys* __restrict__ systems,
                                                              const int2* __restrict__ map, BatchGlobal* gl,
                                                              cudaGraphConditionalHandle cond, int use_cond) {
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
    if (work) {
      if (arrive_acq_rel(B.counters + 1) == (unsigned)B.nblocks_upd - 1) {
        S.applied = iter;
        B.counters[1] = 0u;
        if (S.done && !S.retired) {
          S.retired = 1;
          atomicSub(&gl->active, 1);
        }
      }
    } else if (m.y == 0 && S.done && !S.retired) {  // stopped without a step to apply
      S.retired = 1;
      atomicSub(&gl->active, 1);
    }
    if (arrive_acq_rel(&gl->counter) == gridDim.x - 1) {  // after this block's changes to `active`
      gl->counter = 0u;
      gl->loops += 1;
      const bool again = atomicAdd(&gl->active, 0) > 0 && gl->loops < gl->loop_cap;
      if (use_cond) cudaGraphSetConditional(cond, again ? 1u : 0u);
    }
  }
}

template <int PREC, int NREAL, int K>
static tm_status launch_hop_group(const BatchSys* d_sys, const BatchGroup* d_grp, const int2* d_map, int nblocks,
                                  int in_sel, int y_sel, int out_sel, int kk, int parity, int mode, bool has_y,
                                  cudaStream_t s) {
#define TM_GARGS d_sys, d_grp, d_map, in_sel, y_sel, out_sel, kk, parity
  if (!has_y && mode == 0)
    hop_group_kernel<PREC, NREAL, false, 0, K><<<nblocks, HOP_NT, 0, s>>>(TM_GARGS);
  else if (has_y && mode == 1)
    hop_group_kernel<PREC, NREAL, true, 1, K><<<nblocks, HOP_NT, 0, s>>>(TM_GARGS);
  else
    hop_group_kernel<PREC, NREAL, true, 2, K><<<nblocks, HOP_NT, 0, s>>>(TM_GARGS);
#undef TM_GARGS
  count_launch();
  return cuda_check(cudaGetLastError(), "batched hopping kernel");
}

// The batched hopping launch of one sloppy form with K systems per group.
struct GroupLaunch {
  int prec, nreal, K;
  const BatchSys* sys;
  const BatchGroup* grp;
  const int2* map;
  int nblocks;
};

static tm_status hop_batch(const GroupLaunch& L, int in_sel, int y_sel, int out_sel, int kk, int parity, int mode,
                           bool has_y, cudaStream_t s) {
#define TM_B(P, N, KK)                                                                                    \
  if (L.prec == P && L.nreal == N && L.K == KK)                                                          \
    return launch_hop_group<P, N, KK>(L.sys, L.grp, L.map, L.nblocks, in_sel, y_sel, out_sel, kk, parity, mode, \
                                      has_y, s);
#define TM_BK(P, N) TM_B(P, N, 1) TM_B(P, N, 2) TM_B(P, N, 4)
  TM_BK(TM_F32, 18) TM_BK(TM_F32, 12) TM_BK(TM_F32, 8) TM_BK(TM_F16, 18) TM_BK(TM_F16, 12) TM_BK(TM_F16, 8)
#undef TM_BK
#undef TM_B
  return set_error(TM_ERR_UNSUPPORTED, "batched solve: sloppy form not supported");
}

// One batched CG iteration: K1..K4 of every system, then the update.
static tm_status batch_iteration(const GroupLaunch& L, const int2* d_umap, int nu, BatchGlobal* d_gl,
                                 cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) {
  tm_status st;
  // K1: T = (M_ee^-f)^-1 H_eo p ; K2: W = Qhat^-f p, <p,Ap> ; K3: T = (M_ee^f)^-1 H_eo W ; K4: r -= alpha Qhat^f W
  if ((st = hop_batch(L, 0, 0, 1, 0, 0, 0, false, s)) != TM_OK) return st;
  if ((st = hop_batch(L, 1, 0, 2, 1, 1, 1, true, s)) != TM_OK) return st;
  if ((st = hop_batch(L, 2, 0, 1, 2, 0, 0, false, s)) != TM_OK) return st;
  if ((st = hop_batch(L, 1, 2, 3, 3, 1, 2, true, s)) != TM_OK) return st;
  if (L.prec == TM_F32)
    cg_update_batch_kernel<TM_F32><<<nu, BNT, 0, s>>>(L.sys, d_umap, d_gl, cond, use_cond);
  else
    cg_update_batch_kernel<TM_F16><<<nu, BNT, 0, s>>>(L.sys, d_umap, d_gl, cond, use_cond);
  count_launch();
  return cuda_check(cudaGetLastError(), "batched update kernel");
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
  bool converged, failed;
  bool reconstructed;  // x written and checked by the confirmation of a converged stage
  double true_rel;     // its full-system FP64 residual
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
    for (int q = 0; q < 4; ++q) offs.push_back(add(192 * h));
    for (int q = 0; q < 2; ++q) offs.push_back(add(96 * h));
    for (int q = 0; q < 3; ++q) offs.push_back(add(spinor_bytes_per_site(sp) * h));
  }
  // device tables (the block map has at most one entry per system and block of sites: K = 1)
  int npart = 0, nu = 0;
  for (auto& w : W) {
    npart += (int)hop_grid_blocks(w.lat->h, 1);
    nu += (int)blas_blocks(w.lat->geom.h);
  }
  const size_t off_sys = add(sizeof(BatchSys) * nsys);
  const size_t off_grp = add(sizeof(BatchGroup) * nsys);
  const size_t off_hmap = add(sizeof(int2) * npart);
  const size_t off_umap = add(sizeof(int2) * nu);
  const size_t off_state = add(sizeof(CGState) * nsys);
  const size_t off_gl = add(sizeof(BatchGlobal));
  const size_t off_part = add(sizeof(double) * npart);
  const size_t off_ctr = add(sizeof(unsigned) * 2 * nsys);
  char* base = nullptr;
  if ((st = cuda_check(cudaMalloc(&base, total), "tm_solve_cg_batch: work space")) != TM_OK) return st;
  std::vector<BatchSys> hsys(nsys);
  std::vector<CGState> hst(nsys);
  BatchGlobal hgl{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  tm_status result = TM_OK;
  {
    size_t oi = 0;
    for (auto& L : lats) {
      L.R = base + offs[oi++];
      L.Pv = base + offs[oi++];
      L.T = base + offs[oi++];
      L.W = base + offs[oi++];
    }
    for (auto& w : W) {
      w.be = base + offs[oi++];
      w.bo = base + offs[oi++];
      w.bp = base + offs[oi++];
      w.X = base + offs[oi++];
      w.rs = base + offs[oi++];
      w.xs = base + offs[oi++];
      w.ps = base + offs[oi++];
      w.Ts = base + offs[oi++];
      w.Ws = base + offs[oi++];
    }
  }
  BatchSys* d_sys = reinterpret_cast<BatchSys*>(base + off_sys);
  BatchGroup* d_grp = reinterpret_cast<BatchGroup*>(base + off_grp);
  int2* d_hmap = reinterpret_cast<int2*>(base + off_hmap);
  GroupLaunch GL{sp, sl, 1, d_sys, d_grp, d_hmap, 0};
  int2* d_umap = reinterpret_cast<int2*>(base + off_umap);
  CGState* d_st = reinterpret_cast<CGState*>(base + off_state);
  BatchGlobal* d_gl = reinterpret_cast<BatchGlobal*>(base + off_gl);
  double* d_part = reinterpret_cast<double*>(base + off_part);
  unsigned* d_ctr = reinterpret_cast<unsigned*>(base + off_ctr);

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
      }
      st = cuda_check(cudaMemcpyAsync(d_sys, hsys.data(), sizeof(BatchSys) * nsys, cudaMemcpyHostToDevice, s), "table");
      if (st == TM_OK)
        st = cuda_check(cudaMemcpyAsync(d_umap, umap.data(), sizeof(int2) * nu, cudaMemcpyHostToDevice, s), "table");
      if (st == TM_OK) st = cuda_check(cudaMemsetAsync(d_ctr, 0, sizeof(unsigned) * 2 * nsys, s), "memset");
      // states with nothing stopped, for the tuner's launches
      for (int k = 0; k < nsys && st == TM_OK; ++k) hst[k] = fresh_state(W[k].rr, W[k].stop2, P.max_iter, 0, 0.0, 0.0);
      if (st == TM_OK)
        st = cuda_check(cudaMemcpyAsync(d_st, hst.data(), sizeof(CGState) * nsys, cudaMemcpyHostToDevice, s), "state");
      if (st == TM_OK) st = choose_batch_k(W, lats, sp, sl, GL, s);
      if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "tables");
    }
    if (st != TM_OK) break;
    // ---- the stage graph: WHILE (any system active) { one batched iteration }; with TM_NO_GRAPH=1
    // the stages run as host-driven chunks of iterations instead
    if (use_graphs()) {
      cudaGraphConditionalHandle cond;
      cudaGraphNode_t node;
      cudaGraphNodeParams cp = {};
      const unsigned long long before = tm_launch_count();
      st = cuda_check(cudaGraphCreate(&graph, 0), "cudaGraphCreate");
      if (st == TM_OK)
        st = cuda_check(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault), "conditional");
      if (st == TM_OK) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        st = cuda_check(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp), "conditional node");
      }
      if (st == TM_OK) st = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
      if (st == TM_OK) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        st = cuda_check(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                        "begin capture");
        if (st == TM_OK) {
          tm_status st1 = TM_OK;
          for (int u = 0; u < cg_unroll() && st1 == TM_OK; ++u)
            st1 = batch_iteration(GL, d_umap, nu, d_gl, cond, 1, cs);
          cudaGraph_t captured = nullptr;
          tm_status st2 = cuda_check(cudaStreamEndCapture(cs, &captured), "end capture");
          st = st1 != TM_OK ? st1 : st2;
        }
      }
      if (st == TM_OK) st = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
      tm_reset_launch_count();
      count_launch((unsigned)before);
    }
    if (st != TM_OK) break;
    // ---- stages
    const double delta2 = P.delta * P.delta;
    for (;;) {
      int active = 0, cap = 0;
      for (int k = 0; k < nsys; ++k) {
        SysWork& w = W[k];
        const bool run = !w.converged && !w.failed && w.iters < P.max_iter;
        hst[k] = fresh_state(w.rr, w.stop2, P.max_iter, w.iters, delta2, SLOPPY_GROWTH);
        if (!run) {
          hst[k].done = 1;
          hst[k].retired = 1;
        } else {
          ++active;
          cap = std::max(cap, P.max_iter - w.iters + 2);
        }
      }
      if (active == 0) break;
      hgl = BatchGlobal{active, 0, cap, 0u};
      st = cuda_check(cudaMemcpyAsync(d_st, hst.data(), sizeof(CGState) * nsys, cudaMemcpyHostToDevice, s), "state");
      if (st == TM_OK) st = cuda_check(cudaMemcpyAsync(d_gl, &hgl, sizeof(hgl), cudaMemcpyHostToDevice, s), "state");
      if (exec) {
        if (st == TM_OK) st = cuda_check(cudaGraphLaunch(exec, s), "graph launch");
        if (st == TM_OK)
          st = cuda_check(cudaMemcpyAsync(hst.data(), d_st, sizeof(CGState) * nsys, cudaMemcpyDeviceToHost, s),
                          "state");
        if (st == TM_OK) st = cuda_check(cudaMemcpyAsync(&hgl, d_gl, sizeof(hgl), cudaMemcpyDeviceToHost, s), "state");
        if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "batched stage");
        if (st != TM_OK) break;
        count_launch(5u * (unsigned)hgl.loops);
      } else {  // host-driven: chunks of 8 batched iterations until no system is active
        for (;;) {
          for (int q = 0; q < 8 && st == TM_OK; ++q)
            st = batch_iteration(GL, d_umap, nu, d_gl, 0, 0, s);
          if (st == TM_OK) st = cuda_check(cudaMemcpyAsync(&hgl, d_gl, sizeof(hgl), cudaMemcpyDeviceToHost, s), "state");
          if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "batched chunk");
          if (st != TM_OK || hgl.active <= 0 || hgl.loops >= hgl.loop_cap) break;
        }
        if (st == TM_OK)
          st = cuda_check(cudaMemcpyAsync(hst.data(), d_st, sizeof(CGState) * nsys, cudaMemcpyDeviceToHost, s),
                          "state");
        if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "batched stage");
        if (st != TM_OK) break;
      }
      // ---- reliable updates (FP64) of every system that stopped
      for (int k = 0; k < nsys && st == TM_OK; ++k) {
        SysWork& w = W[k];
        if (w.converged || w.failed || w.iters >= P.max_iter) continue;
        const CGState& c = hst[k];
        if (!c.done) {  // the loop bound ended the stage first
          w.iters = c.iter;
          continue;
        }
        LatWork& L = lats[w.lat_index];
        if (c.nonfinite) {
          st = cuda_check(cudaMemsetAsync(w.xs, 0, w.S.hb[TM_F32], s), "memset");
          w.failed = (++w.updates > 1000);
        } else {
          if (c.iter == w.iters) {  // breakdown without progress
            w.failed = true;
            continue;
          }
          st = launch_accumulate(w.S, w.X, w.xs);
        }
        w.iters = c.iter;
        bool missed = false;  // a converged stage whose confirmation failed
        if (st == TM_OK && !c.nonfinite && c.converged) {
          // confirm through the reconstruction's FP64 residual of the full system, whose odd part
          // is ||b' - A X|| up to the rounding of x_e (4 FP64 hopping launches instead of the
          // residual's 4 now and the reconstruction's 4 at the end); if it misses, update as usual
          double rro = 0.0;
          st = reconstruct_check(w.S, w.X, w.be, w.bo, w.bfull, w.x, L.T, L.W, L.R, L.Pv, &w.true_rel, &rro);
          if (st != TM_OK) break;
          ++w.updates;
          if (batch_verbose())
            fprintf(stderr, "[tm_solve_cg_batch] system %d confirmation: FP64 |(b - M x)_o|/|b'| %.3e (%s)\n", k,
                    std::sqrt(rro / w.bb), rro < w.stop2 ? "converged" : "not confirmed, continuing");
          if (rro < w.stop2) {
            w.converged = w.reconstructed = true;
            w.rr = rro;
            continue;
          }
          missed = true;
        }
        double rr_true = 0.0;
        if (st == TM_OK) st = true_residual(w.S, L.R, w.X, w.bp, L.T, L.W, &rr_true);
        if (st != TM_OK) break;
        ++w.updates;
        if (rr_true < w.stop2) {
          w.converged = true;
          w.rr = rr_true;
          continue;
        }
        if (!(rr_true < 1e300)) {
          w.failed = true;
          continue;
        }
        st = convert_half(w.lat, TM_F32, w.rs, TM_F64, L.R, s);
        // the search direction restarts from the true residual after a divergent or overflowed
        // stage, and after a converged stage that the FP64 residual did not confirm: that stage's
        // p is scaled to its (drifted) iterated residual, not to the true one
        if (st == TM_OK && (c.diverged || c.nonfinite || missed))
          st = convert_half(w.lat, sp, w.ps, TM_F64, L.R, s);
        w.rr = rr_true;
      }
      if (st != TM_OK) break;
    }
    if (st != TM_OK) break;
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
      } else if (w.reconstructed) {
        info.true_rel_residual = w.true_rel;
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
