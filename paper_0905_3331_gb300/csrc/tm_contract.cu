// tm_contract.cu -- meson contraction of a point-source propagator (tm_meson_contract).
//
// The correlators of Sec. 4.3 (one-end trick) are, for a point source at the origin,
//   C_PG(t) = sum_{x, x_t = t} tr[ G(x,0)^dag G(x,0) G~ ]  with G~ = Gamma gamma5 on source spin,
// where G(x,0) is the 12 x 12 spin-colour propagator (column j = the solution for the source
// of spin-colour j).  This file computes the timeslice sums of its Gram matrix
//   A_t[j][k] = sum_{x, x_t = t} <psi^(j)(x), psi^(k)(x)>   (conjugate on j),
// from which every C_PG(t) follows as a 12 x 12 trace (tm_correlator, below).  Deterministic
// two-pass FP64 sums.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "tm_internal.cuh"

namespace tmq {

// The contraction is a Gram matrix per timeslice, 12 x 12 complex, of 12-component colour-spin
// vectors: 13.8 kflop per site in FP64 (144 pairs), 7.5 kflop with the hermitian symmetry used
// (78 pairs j <= k), against 2304 bytes read per site -- bound by the FP64 units, not HBM.
// A block stages a tile of CS sites of all 12 propagators in shared memory with coalesced
// 16-byte loads, then one thread per pair (j, k), j <= k, accumulates its dot products.
constexpr int CS = 16;                 // sites per tile
constexpr int CNT = 128;               // threads per block (78 compute, all load)
constexpr int NPAIR = 78;              // pairs j <= k of 12 indices
constexpr int ROW = CS * 24 + 2;       // doubles per propagator row in shared memory (padded)

__device__ __forceinline__ void pair_of(int p, int* j, int* k) {
  int jj = 0, n = 12;
  while (p >= n) {
    p -= n;
    ++jj;
    --n;
  }
  *j = jj;
  *k = jj + p;
}

// partial[t][bx][pair] (complex): block bx of timeslice t sums its tiles of sites
__global__ void __launch_bounds__(CNT) contract_kernel(const double* __restrict__ props, size_t V, int spatial,
                                                       int nbx, double* __restrict__ partial) {
  __shared__ __align__(16) double tile[12 * ROW];
  const int t = blockIdx.y;
  const int tid = threadIdx.x;
  int j = 0, k = 0;
  if (tid < NPAIR) pair_of(tid, &j, &k);
  double re = 0.0, im = 0.0;
  const int ntile = (spatial + CS - 1) / CS;
  for (int tl = blockIdx.x; tl < ntile; tl += nbx) {
    const int s0 = tl * CS;
    const int ns = min(CS, spatial - s0);
    // 12 rows of ns * 24 doubles, each contiguous in HBM: 16-byte loads
    for (int idx = tid; idx < 12 * CS * 12; idx += CNT) {
      const int row = idx / (CS * 12), c2 = idx % (CS * 12);
      double2 v = make_double2(0.0, 0.0);
      if (c2 < ns * 12)
        v = *reinterpret_cast<const double2*>(props + ((size_t)row * V + (size_t)t * spatial + s0) * 24 + 2 * c2);
      *reinterpret_cast<double2*>(&tile[row * ROW + 2 * c2]) = v;
    }
    __syncthreads();
    if (tid < NPAIR) {
      const double* a = tile + j * ROW;
      const double* b = tile + k * ROW;
#pragma unroll 4
      for (int q = 0; q < CS * 12; ++q) {  // conj(a) b over the tile's sites and components
        const double ar = a[2 * q], ai = a[2 * q + 1], br = b[2 * q], bi = b[2 * q + 1];
        re = fma(ar, br, fma(ai, bi, re));
        im = fma(ar, bi, fma(-ai, br, im));
      }
    }
    __syncthreads();
  }
  if (tid < NPAIR) {
    double* out = partial + (((size_t)t * nbx + blockIdx.x) * NPAIR + tid) * 2;
    out[0] = re;
    out[1] = im;
  }
}

// out[t][j][k] = sum over bx of partial[t][bx][pair], in order; out[t][k][j] = its conjugate
__global__ void contract_finish_kernel(const double* __restrict__ partial, int nbx, int T, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (t, pair)
  if (i >= T * NPAIR) return;
  const int t = i / NPAIR, p = i % NPAIR;
  double re = 0.0, im = 0.0;
  for (int b = 0; b < nbx; ++b) {
    const double* q = partial + (((size_t)t * nbx + b) * NPAIR + p) * 2;
    re += q[0];
    im += q[1];
  }
  int j, k;
  pair_of(p, &j, &k);
  double* o = out + (size_t)t * 12 * 12 * 2;
  o[(j * 12 + k) * 2] = re;
  o[(j * 12 + k) * 2 + 1] = im;
  o[(k * 12 + j) * 2] = re;
  o[(k * 12 + j) * 2 + 1] = j == k ? im : -im;
}

// C[g][t] = tr[A_t (X_g (x) 1_colour)] = sum_{s, s', c} A_t[3s+c][3s'+c] X_g[s'][s]: one thread
// per (g, t), the 48 complex products summed in the order s, s', c (FP64, deterministic).
__global__ void correlator_kernel(const double* __restrict__ A, const double* __restrict__ X, int T, int ngamma,
                                  double* __restrict__ C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (g, t)
  if (i >= T * ngamma) return;
  const int g = i / T, t = i % T;
  const double* a = A + (size_t)t * 144 * 2;
  const double* x = X + (size_t)g * 16 * 2;
  double re = 0.0, im = 0.0;
  for (int s = 0; s < 4; ++s)
    for (int sp = 0; sp < 4; ++sp) {
      const double xr = x[(sp * 4 + s) * 2], xi = x[(sp * 4 + s) * 2 + 1];
      for (int c = 0; c < 3; ++c) {
        const int jk = (3 * s + c) * 12 + (3 * sp + c);
        const double ar = a[jk * 2], ai = a[jk * 2 + 1];
        re = fma(ar, xr, fma(-ai, xi, re));
        im = fma(ar, xi, fma(ai, xr, im));
      }
    }
  C[(size_t)i * 2] = re;
  C[(size_t)i * 2 + 1] = im;
}

}  // namespace tmq

using namespace tmq;

extern "C" tm_status tm_correlator(tm_lattice lat, const double* A, const double* X, int ngamma, double* C,
                                   void* stream) {
  if (!lat || !A || !X || !C || ngamma < 1 || ngamma > 1024)
    return set_error(TM_ERR_ARG, "tm_correlator: NULL argument or ngamma not in 1..1024");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int T = lat->T;
  tm_status st;
  const double* dA = static_cast<const double*>(stage_in(lat, WS_STAGE_IN, A, (size_t)T * 144 * 2 * sizeof(double), s, &st));
  if (st != TM_OK) return st;
  const double* dX = static_cast<const double*>(stage_in(lat, WS_GAMMA, X, (size_t)ngamma * 16 * 2 * sizeof(double), s, &st));
  if (st != TM_OK) return st;
  const size_t out_bytes = (size_t)ngamma * T * 2 * sizeof(double);
  double* dC = static_cast<double*>(stage_out(lat, WS_STAGE_OUT, C, out_bytes, &st));
  if (st != TM_OK) return st;
  const int n = T * ngamma;
  correlator_kernel<<<(n + 127) / 128, 128, 0, s>>>(dA, dX, T, ngamma, dC);
  count_launch();
  if ((st = cuda_check(cudaGetLastError(), "tm_correlator")) != TM_OK) return st;
  return stage_out_finish(C, dC, out_bytes, s);
}

extern "C" tm_status tm_meson_contract(tm_lattice lat, const double* props, double* out, void* stream) {
  if (!lat || !props || !out) return set_error(TM_ERR_ARG, "tm_meson_contract: NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t V = lat->V;
  const int spatial = lat->L * lat->L * lat->L;
  const int T = lat->T;
  tm_status st;
  const double* dp = static_cast<const double*>(stage_in(lat, WS_STAGE_IN, props, 12 * V * 24 * sizeof(double), s, &st));
  if (st != TM_OK) return st;
  if (reinterpret_cast<uintptr_t>(dp) % 16 != 0)
    return set_error(TM_ERR_ARG, "tm_meson_contract: device props must be 16-byte aligned");
  const size_t out_bytes = (size_t)T * 12 * 12 * 2 * sizeof(double);
  double* dout = static_cast<double*>(stage_out(lat, WS_STAGE_OUT, out, out_bytes, &st));
  if (st != TM_OK) return st;
  // about eight blocks per SM over all timeslices; each block loops over its tiles
  const int ntile = (spatial + CS - 1) / CS;
  const int nbx = std::max(1, std::min(ntile, (152 * 8 + T - 1) / T));
  double* partial =
      static_cast<double*>(workspace(lat, WS_X0 + 1, (size_t)T * nbx * NPAIR * 2 * sizeof(double), &st));
  if (st != TM_OK) return st;
  contract_kernel<<<dim3(nbx, T), CNT, 0, s>>>(dp, V, spatial, nbx, partial);
  count_launch();
  const int n = T * NPAIR;
  contract_finish_kernel<<<(n + 255) / 256, 256, 0, s>>>(partial, nbx, T, dout);
  count_launch();
  if ((st = cuda_check(cudaGetLastError(), "tm_meson_contract")) != TM_OK) return st;
  return stage_out_finish(out, dout, out_bytes, s);
}
