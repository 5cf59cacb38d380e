// tm_solver.cuh -- pieces of the even/odd CG shared by the single-system and batched solvers.
#pragma once

#include <functional>

#include "tm_internal.cuh"

namespace tmq {

constexpr int BNT = 256;                // threads per block of the vector kernels
constexpr double SLOPPY_GROWTH = 100.0;  // a sloppy stage ends when ||r|| grows this much over its minimum

// One system's solver context: lattice, stream, flavour sign f and mu~ = 2 kappa mu.
struct Solver {
  tm_lattice lat;
  cudaStream_t s;
  int f;
  double mut;
  size_t hb[4];  // half-field bytes per precision
};

unsigned blas_blocks(int h);
tm_status norm2_half(const Solver& S, int prec, const void* x, double* out_host);
// r -= alpha Qhat^f Qhat^{-f} in (iteration form with `state`, else alpha = 1 and ||r||^2 in dscalars[0])
tm_status normal_apply(const Solver& S, int prec, int nreal, const void* in, void* T, void* W, void* r,
                       CGState* state);
// r = b' - A X in FP64; ||r||^2 returned
tm_status true_residual(const Solver& S, void* r, const void* X, const void* bp, void* T, void* W, double* rr);
CGState fresh_state(double rr, double stop2, int max_iter, int iter0, double delta2, double growth = 0.0);
tm_status prepare_source(const Solver& S, const double* b, void* be, void* bo, void* bp, void* T, double* bb,
                         double* bfull);
// rr_odd (optional): ||(b - M x)_o||^2, the odd part of the full residual
tm_status reconstruct_check(const Solver& S, const void* X, const void* be, const void* bo, double bfull, double* x,
                            void* T, void* W, void* R, void* Pv, double* true_rel, double* rr_odd = nullptr);
tm_status reconstruct_xo(const Solver& S, const void* xo, const void* be, const void* bo, double bfull, double* x,
                         void* T, void* R, void* Pv, double* true_rel, double* rr_odd = nullptr);
tm_status launch_accumulate(const Solver& S, void* X, void* xs);  // X (FP64) += xs (FP32); xs = 0

struct NormalResult {
  int iters, updates;
  bool converged;
  double rr_true;   // ||bp - A X||^2, recomputed in FP64 (the iterated one when `pending`)
  bool xo_in_W;     // W holds Qhat^{-f} X for the final X (left by the last FP64 residual)
  bool pending;     // the last sloppy stage reached the tolerance; X is not yet confirmed in FP64
};
// With defer_final (mixed modes, FP64 updates), a sloppy stage that reaches the tolerance ends
// the call with `pending` instead of an FP64 recomputation of bp - A X: the caller confirms X
// through the FP64 residual of the full system, whose odd part is the same quantity.
tm_status cg_normal(const Solver& S, const tm_cg_params& P, const void* bp, double bb, void* X, bool guess, void* R,
                    void* Pv, void* T, void* W, NormalResult* res, bool defer_final = false);

bool use_graphs();  // CUDA-graph stage loops (TM_NO_GRAPH=1 selects host-driven chunks)
int cg_unroll();    // iterations per body of a graph loop (TM_CG_UNROLL)
int cg_unroll_for(size_t h);  // the same for a lattice of h sites per parity

// A cached CUDA graph whose only node is a WHILE conditional; its body is whatever `body`
// enqueues on the capture stream (the body's last kernel sets the condition).  Graphs are
// cached on the lattice under the 16-word key (the caller includes every buffer address and
// parameter the body bakes in).
typedef std::function<tm_status(cudaStream_t, cudaGraphConditionalHandle)> LoopBody;
tm_status aux_loop_graph(tm_lattice lat, const unsigned long long key[16], cudaStream_t s, const LoopBody& body,
                         cudaGraphExec_t* out);

// x += alpha p; p = r + beta p over n "sites" of the given formats (n = h for one half field;
// 2h for two stacked half fields of the same formats), once per iteration (see cg_update_kernel)
tm_status launch_update_n(const Solver& S, int n, int px, int pp, void* x, void* p, const void* r, CGState* state,
                          cudaGraphConditionalHandle cond, int use_cond);
// sum of |x|^2 over n sites of format prec into *out_host (synchronises)
tm_status norm2_n(const Solver& S, int prec, int n, const void* x, double* out_host);

enum { SOLVER_CG = 0, SOLVER_BICGSTAB = 1, SOLVER_MR = 2 };
tm_status solve_driver(tm_lattice lat, double* x, const double* b, int nrhs, const tm_cg_params* params,
                       tm_cg_info* info, void* stream, int kind);
// BiCGstab on Mhat^f x_o = varphi_o for one canonical full field (tm_bicgstab.cu)
tm_status solve_one_bicgstab(tm_lattice lat, double* x, const double* b, const tm_cg_params& P, tm_cg_info* info,
                             cudaStream_t s);
// MR on Mhat^f x_o = varphi_o for one canonical full field (tm_bicgstab.cu)
tm_status solve_one_mr(tm_lattice lat, double* x, const double* b, const tm_cg_params& P, tm_cg_info* info,
                       cudaStream_t s);

}  // namespace tmq
