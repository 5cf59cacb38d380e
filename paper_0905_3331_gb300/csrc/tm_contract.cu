// tm_contract.cu -- meson contraction of a point-source propagator (tm_meson_contract).
//
// The correlators of Sec. 4.3 (one-end trick) are, for a point source at the origin,
//   C_PG(t) = sum_{x, x_t = t} tr[ G(x,0)^dag G(x,0) G~ ]  with G~ = Gamma gamma5 on source spin,
// where G(x,0) is the 12 x 12 spin-colour propagator (column j = the solution for the source
// of spin-colour j).  This file computes the timeslice sums of its Gram matrix
//   A_t[j][k] = sum_{x, x_t = t} <psi^(j)(x), psi^(k)(x)>   (conjugate on j),
// from which every C_PG(t) follows as a 12 x 12 trace.  Deterministic two-pass FP64 sums.
#include <algorithm>
#include <vector>

#include "tm_internal.cuh"

namespace tmq {

constexpr int CSITES = 16;  // site lanes per block (x 12 source indices = 192 threads)
constexpr int CNT = CSITES * 12;

// partial[t][bx][j][k] (complex): block bx of timeslice t, thread (lane, j) sums over its sites
__global__ void __launch_bounds__(CNT) contract_kernel(const double* __restrict__ props, size_t V, int spatial,
                                                       int nbx, double* __restrict__ partial) {
  __shared__ double red[CNT][2 * 12 + 1];
  const int t = blockIdx.y;
  const int lane = threadIdx.x / 12, j = threadIdx.x % 12;
  double acc[24];
#pragma unroll
  for (int q = 0; q < 24; ++q) acc[q] = 0.0;
  for (int xs = blockIdx.x * CSITES + lane; xs < spatial; xs += nbx * CSITES) {
    const size_t lex = (size_t)t * spatial + xs;
    const double* pj = props + ((size_t)j * V + lex) * 24;
    double a[24];
#pragma unroll
    for (int q = 0; q < 24; ++q) a[q] = pj[q];
#pragma unroll 1
    for (int k = 0; k < 12; ++k) {
      const double* pk = props + ((size_t)k * V + lex) * 24;
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int q = 0; q < 12; ++q) {  // conj(a) * b
        const double br = pk[2 * q], bi = pk[2 * q + 1];
        re += a[2 * q] * br + a[2 * q + 1] * bi;
        im += a[2 * q] * bi - a[2 * q + 1] * br;
      }
      acc[2 * k] += re;
      acc[2 * k + 1] += im;
    }
  }
#pragma unroll
  for (int q = 0; q < 24; ++q) red[threadIdx.x][q] = acc[q];
  __syncthreads();
  // thread (lane == 0, j) sums the 16 lanes of its j in order
  if (lane == 0) {
    double* out = partial + (((size_t)t * nbx + blockIdx.x) * 12 + j) * 24;
    for (int q = 0; q < 24; ++q) {
      double s = 0.0;
      for (int l = 0; l < CSITES; ++l) s += red[l * 12 + j][q];
      out[q] = s;
    }
  }
}

// out[t][j][k] = sum over bx of partial[t][bx][j][k], in order
__global__ void contract_finish_kernel(const double* __restrict__ partial, int nbx, int T, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (t, j, 2k + reim)
  if (i >= T * 12 * 24) return;
  const int t = i / (12 * 24), r = i % (12 * 24);
  double s = 0.0;
  for (int b = 0; b < nbx; ++b) s += partial[((size_t)t * nbx + b) * 12 * 24 + r];
  out[i] = s;
}

}  // namespace tmq

using namespace tmq;

extern "C" tm_status tm_meson_contract(tm_lattice lat, const double* props, double* out, void* stream) {
  if (!lat || !props || !out) return set_error(TM_ERR_ARG, "tm_meson_contract: NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t V = lat->V;
  const int spatial = lat->L * lat->L * lat->L;
  const int T = lat->T;
  tm_status st;
  const double* dp = static_cast<const double*>(stage_in(lat, WS_STAGE_IN, props, 12 * V * 24 * sizeof(double), s, &st));
  if (st != TM_OK) return st;
  const size_t out_bytes = (size_t)T * 12 * 12 * 2 * sizeof(double);
  double* dout = static_cast<double*>(stage_out(lat, WS_STAGE_OUT, out, out_bytes, &st));
  if (st != TM_OK) return st;
  const int nbx = std::min(64, (spatial + CSITES - 1) / CSITES);
  double* partial = static_cast<double*>(workspace(lat, WS_X0 + 1, (size_t)T * nbx * 12 * 24 * sizeof(double), &st));
  if (st != TM_OK) return st;
  contract_kernel<<<dim3(nbx, T), CNT, 0, s>>>(dp, V, spatial, nbx, partial);
  count_launch();
  const int n = T * 12 * 24;
  contract_finish_kernel<<<(n + 255) / 256, 256, 0, s>>>(partial, nbx, T, dout);
  count_launch();
  if ((st = cuda_check(cudaGetLastError(), "tm_meson_contract")) != TM_OK) return st;
  return stage_out_finish(out, dout, out_bytes, s);
}
