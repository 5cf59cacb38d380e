// tm_batch_group.cu -- the batched solver's hopping kernel with K = 2 or 4 systems per thread.
//
// Thread = output site; the K systems of a group (same lattice) are its lanes.  Each of the
// site's 8 links is loaded and reconstructed ONCE and applied to the K systems' neighbour
// spinors (the direction-pair arithmetic of hop_kernel, per lane), so a link's bytes and its
// reconstruction serve K right-hand sides from registers.  Each system keeps its own epilogue
// coefficients (its mu), output, CG state and reduction.  The launch walks a work list of the
// running groups (tm_batch.cuh); a group whose systems have all stopped is not on it, a system
// of a listed group that has stopped is skipped.  The batch tuner (tm_batch.cu) times K = 2, 4
// against the one-system kernel on the batch's own vectors and keeps the fastest.
#include "tm_batch.cuh"

namespace tmq {

template <int PREC, int NREAL, bool HAS_Y, int MODE, int K>
__device__ __forceinline__ void group_block(const BatchSys* __restrict__ systems, const BatchGroup* __restrict__ groups,
                                            const CGState* __restrict__ states, const int2 m, int in_sel, int y_sel,
                                            int out_sel, int kk, int out_parity, double* sh) {
  typedef typename SpinorFmt<PREC>::real R;
  typedef SpinorFmt<PREC> F;
  typedef typename LinkStore<PREC>::type St;
  constexpr int BYTES = NREAL * LinkStore<PREC>::size;
  const BatchGroup G = groups[m.x];
  const BatchSys* S[K];
  bool live[K];
  bool any = false;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int k = G.sys[j < G.n ? j : 0];
    S[j] = systems + k;
    live[j] = j < G.n && !states[k].done;
    any = any || live[j];
  }
  if (!any) return;  // block-uniform
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
#define TM_GROUP_DIR(MU, FIRST)                                                            \
  {                                                                                        \
    cpx<R> u0[K][3], u1[K][3], p[12];                                                      \
    R scale;                                                                               \
    Mat3<R> U;                                                                             \
    LinkRecon<R, St, NREAL>::unpack(load_raw<BYTES>(lf + MU * slab, g.h, cb), U);          \
    _Pragma("unroll") for (int j = 0; j < K; ++j) if (live[j]) {                           \
      F::load_unscaled(S[j]->vec[in_sel], g.h, nb[MU], p, scale);                          \
      pair_fwd_mat<PREC, MU>(u0[j], u1[j], U, p, scale, MU == 0 && tf);                    \
    }                                                                                      \
    LinkRecon<R, St, NREAL>::unpack(load_raw<BYTES>(lo + MU * slab, g.h, nb[4 + MU]), U);  \
    _Pragma("unroll") for (int j = 0; j < K; ++j) if (live[j]) {                           \
      F::load_unscaled(S[j]->vec[in_sel], g.h, nb[4 + MU], p, scale);                      \
      pair_bwd_mat<PREC, MU, FIRST>(acc[j], u0[j], u1[j], U, p, scale, MU == 0 && tb);     \
    }                                                                                      \
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
    const EpiCoef& coef = B.coef[kk];
    // o = (D c) acc + (D E) y with the FP32 products folded on the host (epi_finish)
    const cpx<R> DCu = mk<R>(coef.f_dcu_re, coef.f_dcu_im), DCl = mk<R>(coef.f_dcl_re, coef.f_dcl_im);
    cpx<R> o[12];
    if (HAS_Y) {
      const cpx<R> DEu = mk<R>(coef.f_deu_re, coef.f_deu_im), DEl = mk<R>(coef.f_del_re, coef.f_del_im);
      cpx<R> yv[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) yv[q] = mk<R>(R(0), R(0));
      if (active) F::load(B.vec[y_sel], g.h, cb, yv);
#pragma unroll
      for (int q = 0; q < 12; ++q) o[q] = ((q < 6) ? DCu : DCl) * acc[j][q] + ((q < 6) ? DEu : DEl) * yv[q];
    } else {
#pragma unroll
      for (int q = 0; q < 12; ++q) o[q] = ((q < 6) ? DCu : DCl) * acc[j][q];
    }
    float nrm = 0.f;
    void* outp = B.vec[out_sel];
    if (MODE == 2) {
      if (active) {
        const R al = (R)B.st->alpha;
        constexpr int PR = ResidPrec<PREC>::value;
        cpx<R> r[12];
        SpinorFmt<PR>::load(outp, g.h, cb, r);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          r[q] = r[q] - al * o[q];
          nrm += norm2(r[q]);
        }
        SpinorFmt<PR>::store(outp, g.h, cb, r);
      }
    } else if (active) {
      if (MODE == 1) {
#pragma unroll
        for (int q = 0; q < 12; ++q) nrm += norm2(o[q]);
      }
      F::store(outp, g.h, cb, o);
    }
    if (MODE >= 1) {
      const Reduce red{B.partials, B.counters, B.result, B.st, MODE == 1 ? FIN_CG_ALPHA : FIN_CG_RR};
      const double bs = block_sum<HOP_NT>(nrm, sh);
      grid_reduce<HOP_NT>(red, 0, B.nblocks, m.y, bs, sh);
      __syncthreads();  // sh and the reduction's shared flag are reused by the next system
    }
  }
}

// Register budgets: 3 blocks of 128 threads per SM for K = 2, 2 for K = 4 (the accumulators of K
// spinors).
template <int PREC, int NREAL, bool HAS_Y, int MODE, int K>
__global__ void __launch_bounds__(HOP_NT, K == 2 ? 3 : 2)
    hop_group_kernel(const BatchSys* __restrict__ systems, const BatchGroup* __restrict__ groups,
                     const CGState* __restrict__ states, Plan plan, int in_sel, int y_sel, int out_sel, int kk,
                     int out_parity) {
  __shared__ double sh[HOP_NT / 32];
  const int total = plan.start[plan.nlat];
  for (int v = blockIdx.x; v < total; v += gridDim.x)
    group_block<PREC, NREAL, HAS_Y, MODE, K>(systems, groups, states, plan_item(plan, v), in_sel, y_sel, out_sel, kk,
                                             out_parity, sh);
}

template <int PREC, int NREAL, int K>
static tm_status launch_t(const BatchSys* d_sys, const BatchGroup* d_grp, const CGState* d_st, const Plan& plan,
                          int cap, int in_sel, int y_sel, int out_sel, int kk, int parity, int mode, bool has_y,
                          cudaStream_t s) {
#define TM_GL(HY, MD)                                                                                   \
  {                                                                                                     \
    auto kern = hop_group_kernel<PREC, NREAL, HY, MD, K>;                                               \
    kern<<<resident_grid(kern, HOP_NT, cap), HOP_NT, 0, s>>>(d_sys, d_grp, d_st, plan, in_sel, y_sel, out_sel, \
                                                             kk, parity);                              \
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
  return cuda_check(cudaGetLastError(), "batched group hopping kernel");
}

tm_status launch_hop_group(int prec, int nreal, int K, const BatchSys* d_sys, const BatchGroup* d_grp,
                           const CGState* d_st, const Plan& plan, int cap, int in_sel, int y_sel, int out_sel, int kk,
                           int parity, int mode, bool has_y, cudaStream_t s) {
#define TM_B(P, N, KK)                                                                                          \
  if (prec == P && nreal == N && K == KK)                                                                       \
    return launch_t<P, N, KK>(d_sys, d_grp, d_st, plan, cap, in_sel, y_sel, out_sel, kk, parity, mode, has_y, s);
#define TM_BK(P, N) TM_B(P, N, 2) TM_B(P, N, 4)
  TM_BK(TM_F32, 18) TM_BK(TM_F32, 12) TM_BK(TM_F32, 8) TM_BK(TM_F16, 18) TM_BK(TM_F16, 12) TM_BK(TM_F16, 8)
#undef TM_BK
#undef TM_B
  return set_error(TM_ERR_UNSUPPORTED, "batched group kernel: form or K not supported");
}

}  // namespace tmq
