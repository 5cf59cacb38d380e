// tm_normal.cu -- the normal equations directly: tm_solve_normal and tm_chrono_guess.
//
// tm_solve_normal solves Qhat^f Qhat^-f X = phi on the odd sites (eq. eo6; the solve the
// pseudofermion force needs, X_o = (Qhat+ Qhat-)^-1 phi_o) with the CG of tm_solver.cu.
// tm_chrono_guess builds the chronological initial guess of eq. chrono: given earlier
// solutions chi_i it solves sum_i <chi_j, A chi_i> c_i = <chi_j, phi> for the coefficients
// and returns X0 = sum_i c_i chi_i.
#include <cmath>
#include <complex>
#include <vector>

#include "tm_solver.cuh"

namespace tmq {

constexpr int DNB = 256;  // blocks of the dot-product kernel (fixed: deterministic sums)

// partial[b] = sum over this block's sites of conj(a) b (complex), FP64 half fields
__global__ void __launch_bounds__(BNT) cdot_kernel(int h, const char* a, const char* b, double* partial) {
  __shared__ double sre[BNT / 32], sim[BNT / 32];
  double re = 0.0, im = 0.0;
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    cpx<double> x[12], y[12];
    SpinorFmt<TM_F64>::load(a, h, i, x);
    SpinorFmt<TM_F64>::load(b, h, i, y);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const cpx<double> z = cjmul(x[k], y[k]);
      re += z.re;
      im += z.im;
    }
  }
  const double br = block_sum<BNT>(re, sre);
  __syncthreads();
  const double bi = block_sum<BNT>(im, sim);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = br;
    partial[2 * blockIdx.x + 1] = bi;
  }
}

__global__ void cdot_finish_kernel(const double* partial, int nb, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double re = 0.0, im = 0.0;
    for (int b = 0; b < nb; ++b) {
      re += partial[2 * b];
      im += partial[2 * b + 1];
    }
    out[0] = re;
    out[1] = im;
  }
}

// y += c x (complex c), FP64 half fields
__global__ void __launch_bounds__(BNT) caxpy_kernel(int h, char* y, const char* x, double cr, double ci) {
  const cpx<double> c = mk(cr, ci);
  for (int i = blockIdx.x * BNT + threadIdx.x; i < h; i += gridDim.x * BNT) {
    cpx<double> a[12], b[12];
    SpinorFmt<TM_F64>::load(y, h, i, a);
    SpinorFmt<TM_F64>::load(x, h, i, b);
#pragma unroll
    for (int k = 0; k < 12; ++k) a[k] = a[k] + c * b[k];
    SpinorFmt<TM_F64>::store(y, h, i, a);
  }
}

// <a, b> into dst (2 doubles, device); uses lat->partials as scratch
static tm_status cdot(tm_lattice lat, const void* a, const void* b, double* dst, cudaStream_t s) {
  tm_status st = ensure_reduce(lat, 2 * DNB, 4);
  if (st != TM_OK) return st;
  cdot_kernel<<<DNB, BNT, 0, s>>>(lat->geom.h, static_cast<const char*>(a), static_cast<const char*>(b),
                                  lat->partials);
  count_launch();
  cdot_finish_kernel<<<1, 32, 0, s>>>(lat->partials, DNB, dst);
  count_launch();
  return cuda_check(cudaGetLastError(), "dot kernel");
}

static Solver make_solver(tm_lattice lat, int flavour, cudaStream_t s) {
  Solver S{lat, s, flavour, 2.0 * lat->kappa * lat->mu, {0, 0, 0, 0}};
  for (int p = 0; p < 4; ++p) S.hb[p] = spinor_bytes_per_site(p) * lat->h;
  return S;
}

}  // namespace tmq

using namespace tmq;

extern "C" tm_status tm_solve_normal(tm_lattice lat, void* X, const void* phi, const tm_cg_params* params,
                                     tm_cg_info* info, void* stream) {
  if (!lat || !X || !phi) return set_error(TM_ERR_ARG, "tm_solve_normal: NULL argument");
  if (!lat->has_gauge) return set_error(TM_ERR_NO_GAUGE, "tm_solve_normal: no gauge field");
  if (X == phi) return set_error(TM_ERR_ARG, "tm_solve_normal: X and phi must differ");
  if (!is_device_pointer(X) || !is_device_pointer(phi))
    return set_error(TM_ERR_ARG, "tm_solve_normal: X and phi must be device half fields");
  tm_cg_params P;
  if (params)
    P = *params;
  else
    tm_cg_params_default(&P);
  if (P.flavour == 0) P.flavour = 1;
  if (P.flavour != 1 && P.flavour != -1) return set_error(TM_ERR_ARG, "tm_solve_normal: flavour must be +1 or -1");
  if (!(P.tol > 0.0) || P.max_iter < 1) return set_error(TM_ERR_ARG, "tm_solve_normal: tol > 0 and max_iter >= 1");
  if (P.mode < TM_CG_FP64 || P.mode > TM_CG_RELIABLE) return set_error(TM_ERR_ARG, "tm_solve_normal: mode %d", P.mode);
  if (P.mode != TM_CG_FP64) {
    if (P.sloppy_prec != TM_F32 && P.sloppy_prec != TM_F16)
      return set_error(TM_ERR_ARG, "tm_solve_normal: sloppy precision must be TM_F32 or TM_F16");
    if (P.sloppy_link != 18 && P.sloppy_link != 12 && P.sloppy_link != 8)
      return set_error(TM_ERR_ARG, "tm_solve_normal: sloppy link format %d", P.sloppy_link);
    if (!(P.delta > 0.0 && P.delta < 1.0)) return set_error(TM_ERR_ARG, "tm_solve_normal: delta must be in (0, 1)");
    if (P.update_prec != TM_F64 && P.update_prec != TM_DF64 && P.update_prec != TM_F32)
      return set_error(TM_ERR_ARG, "tm_solve_normal: update_prec must be TM_F64, TM_F32 or TM_DF64");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Solver S = make_solver(lat, P.flavour, s);
  tm_status st = TM_OK;
  void* w[4];
  for (int k = 0; k < 4; ++k) {
    w[k] = workspace(lat, 4 + k, S.hb[TM_F64], &st);
    if (st != TM_OK) return st;
  }
  double bb = 0.0;
  if ((st = norm2_half(S, TM_F64, phi, &bb)) != TM_OK) return st;
  if (!std::isfinite(bb)) return set_error(TM_ERR_NONFINITE, "tm_solve_normal: phi has non-finite entries");
  tm_cg_info one{};
  if (bb == 0.0) {
    st = cuda_check(cudaMemsetAsync(X, 0, S.hb[TM_F64], s), "memset");
    if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "synchronise");
    if (info) *info = one;
    return st;
  }
  NormalResult nr{};
  if ((st = cg_normal(S, P, phi, bb, X, P.use_x0 != 0, w[0], w[1], w[2], w[3], &nr)) != TM_OK) return st;
  if ((st = cuda_check(cudaStreamSynchronize(s), "synchronise")) != TM_OK) return st;
  one.iters = nr.iters;
  one.reliable_updates = nr.updates;
  one.schur_rel_residual = std::sqrt(nr.rr_true / bb);
  one.true_rel_residual = one.schur_rel_residual;
  one.status = nr.converged ? TM_OK : TM_ERR_NOT_CONVERGED;
  if (info) *info = one;
  if (!nr.converged)
    return set_error(TM_ERR_NOT_CONVERGED, "tm_solve_normal: not converged after %d iterations (%.3e)", nr.iters,
                     one.schur_rel_residual);
  return TM_OK;
}

extern "C" tm_status tm_chrono_guess(tm_lattice lat, void* X0, const void* const* chi, int n, const void* phi,
                                     int flavour, void* stream) {
  if (!lat || !X0 || !phi || (n > 0 && !chi) || n < 0 || n > 64)
    return set_error(TM_ERR_ARG, "tm_chrono_guess: bad argument (0 <= n <= 64)");
  if (!lat->has_gauge) return set_error(TM_ERR_NO_GAUGE, "tm_chrono_guess: no gauge field");
  if (flavour == 0) flavour = 1;
  if (flavour != 1 && flavour != -1) return set_error(TM_ERR_ARG, "tm_chrono_guess: flavour must be +1 or -1");
  for (int i = 0; i < n; ++i)
    if (!chi[i] || chi[i] == X0) return set_error(TM_ERR_ARG, "tm_chrono_guess: chi[%d] is NULL or X0", i);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Solver S = make_solver(lat, flavour, s);
  tm_status st = TM_OK;
  if ((st = cuda_check(cudaMemsetAsync(X0, 0, S.hb[TM_F64], s), "memset")) != TM_OK) return st;
  if (n == 0) return cuda_check(cudaStreamSynchronize(s), "synchronise");
  void* w[3];
  for (int k = 0; k < 3; ++k) {
    w[k] = workspace(lat, 4 + k, S.hb[TM_F64], &st);
    if (st != TM_OK) return st;
  }
  void *Achi = w[0], *T = w[1], *W = w[2];
  // G[j][i] = <chi_j, A chi_i>, rhs[j] = <chi_j, phi>; scalars staged in device memory
  const size_t nsc = (size_t)2 * (n * n + n);
  double* dev = static_cast<double*>(workspace(lat, WS_CHRONO, nsc * sizeof(double), &st));
  if (st != TM_OK) return st;
  for (int i = 0; i < n && st == TM_OK; ++i) {
    // Achi = A chi_i: normal_apply computes r -= A in, so start from r = 0 and negate the dots.
    // A is hermitian: only j <= i is computed, the rest mirrored below.
    st = cuda_check(cudaMemsetAsync(Achi, 0, S.hb[TM_F64], s), "memset");
    if (st == TM_OK) st = normal_apply(S, TM_F64, 18, chi[i], T, W, Achi, nullptr);
    for (int j = 0; j <= i && st == TM_OK; ++j) st = cdot(lat, chi[j], Achi, dev + 2 * (j * n + i), s);
  }
  for (int j = 0; j < n && st == TM_OK; ++j) st = cdot(lat, chi[j], phi, dev + 2 * (n * n + j), s);
  std::vector<double> h(nsc);
  if (st == TM_OK) st = cuda_check(cudaMemcpyAsync(h.data(), dev, nsc * sizeof(double), cudaMemcpyDeviceToHost, s), "readback");
  if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "synchronise");
  if (st != TM_OK) return st;
  typedef std::complex<double> C;
  std::vector<C> G(n * n), c(n);
  double gmax = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      const C g = -C(h[2 * (j * n + i)], h[2 * (j * n + i) + 1]);  // Achi held -A chi_i
      if (!std::isfinite(g.real()) || !std::isfinite(g.imag()))
        return set_error(TM_ERR_NONFINITE, "tm_chrono_guess: non-finite inner product");
      G[j * n + i] = g;
      G[i * n + j] = std::conj(g);
      gmax = std::max(gmax, std::abs(g));
    }
  for (int j = 0; j < n; ++j) {
    c[j] = C(h[2 * (n * n + j)], h[2 * (n * n + j) + 1]);
    if (!std::isfinite(c[j].real()) || !std::isfinite(c[j].imag()))
      return set_error(TM_ERR_NONFINITE, "tm_chrono_guess: non-finite inner product");
  }
  // Gaussian elimination with partial pivoting; a direction whose pivot vanishes (the history
  // is linearly dependent) gets coefficient 0
  std::vector<int> keep(n, 1);
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int r = k + 1; r < n; ++r)
      if (std::abs(G[r * n + k]) > std::abs(G[piv * n + k])) piv = r;
    if (std::abs(G[piv * n + k]) <= 1e-13 * gmax) {
      keep[k] = 0;
      continue;
    }
    if (piv != k) {
      for (int q = 0; q < n; ++q) std::swap(G[k * n + q], G[piv * n + q]);
      std::swap(c[k], c[piv]);
    }
    for (int r = k + 1; r < n; ++r) {
      const C m = G[r * n + k] / G[k * n + k];
      if (m == C(0)) continue;
      for (int q = k; q < n; ++q) G[r * n + q] -= m * G[k * n + q];
      c[r] -= m * c[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    if (!keep[k]) {
      c[k] = 0.0;
      continue;
    }
    C v = c[k];
    for (int q = k + 1; q < n; ++q) v -= G[k * n + q] * c[q];
    c[k] = v / G[k * n + k];
  }
  const unsigned nb = blas_blocks(lat->geom.h);
  for (int i = 0; i < n && st == TM_OK; ++i) {
    caxpy_kernel<<<nb, BNT, 0, s>>>(lat->geom.h, static_cast<char*>(X0), static_cast<const char*>(chi[i]), c[i].real(),
                                    c[i].imag());
    count_launch();
    st = cuda_check(cudaGetLastError(), "caxpy kernel");
  }
  return st;
}
