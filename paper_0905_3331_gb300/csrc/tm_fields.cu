// tm_fields.cu -- conversions between the canonical FP64 spinor order (t, z, y, x, spin,
// colour; Sec. 4.7.2) and the device half-field layouts, precision conversions, and the
// site-diagonal operator (M_ee^f)^{-1} = (1 - i f mu~ gamma5) / (1 + mu~^2) of eq. eo3.
#include "tm_internal.cuh"

namespace tmq {

constexpr int FNT = 128;

template <typename R>
__device__ __forceinline__ void load_canon(const double* src, cpx<R> s[12]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) s[k] = mk<R>((R)src[2 * k], (R)src[2 * k + 1]);
}
template <typename R>
__device__ __forceinline__ void store_canon(double* dst, const cpx<R> s[12]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    dst[2 * k] = (double)s[k].re;
    dst[2 * k + 1] = (double)s[k].im;
  }
}
template <typename R>
__device__ __forceinline__ void apply_g5(cpx<R> s[12]) {
#pragma unroll
  for (int k = 6; k < 12; ++k) s[k] = R(-1) * s[k];
}

// canonical half field [rhs][cb][24] <-> device layout [rhs][field]
template <int PREC>
__global__ void pack_half_kernel(int h, const double* __restrict__ src, char* __restrict__ dst, size_t dstride) {
  const int cb = blockIdx.x * FNT + threadIdx.x, r = blockIdx.y;
  if (cb >= h) return;
  cpx<double> s[12];
  load_canon(src + ((size_t)r * h + cb) * 24, s);
  SpinorFmt<PREC>::store(dst + r * dstride, h, cb, s);
}
template <int PREC>
__global__ void unpack_half_kernel(int h, const char* __restrict__ src, size_t sstride, double* __restrict__ dst) {
  const int cb = blockIdx.x * FNT + threadIdx.x, r = blockIdx.y;
  if (cb >= h) return;
  cpx<double> s[12];
  SpinorFmt<PREC>::load(src + r * sstride, h, cb, s);
  store_canon(dst + ((size_t)r * h + cb) * 24, s);
}

// parity p of a canonical full field <-> device half field (optionally times gamma5)
__device__ __forceinline__ size_t lex_of_cb(const Geom& g, int cb, int p) {
  const int r = cb / g.Lh;
  const int y = r % g.L, z = (r / g.L) % g.L, t = r / (g.L * g.L);
  return 2 * (size_t)cb + ((t + z + y + p) & 1);
}
template <int PREC>
__global__ void pack_full_kernel(Geom g, const double* __restrict__ src, char* __restrict__ dst, int p, int g5) {
  const int cb = blockIdx.x * FNT + threadIdx.x;
  if (cb >= g.h) return;
  cpx<double> s[12];
  load_canon(src + lex_of_cb(g, cb, p) * 24, s);
  if (g5) apply_g5(s);
  SpinorFmt<PREC>::store(dst, g.h, cb, s);
}
template <int PREC>
__global__ void unpack_full_kernel(Geom g, const char* __restrict__ src, double* __restrict__ dst, int p, int g5) {
  const int cb = blockIdx.x * FNT + threadIdx.x;
  if (cb >= g.h) return;
  cpx<double> s[12];
  SpinorFmt<PREC>::load(src, g.h, cb, s);
  if (g5) apply_g5(s);
  store_canon(dst + lex_of_cb(g, cb, p) * 24, s);
}

template <int PIN, int POUT>
__global__ void convert_kernel(int h, const char* __restrict__ src, char* __restrict__ dst) {
  const int cb = blockIdx.x * FNT + threadIdx.x;
  if (cb >= h) return;
  typedef typename SpinorFmt<PIN>::real R;
  cpx<R> s[12];
  SpinorFmt<PIN>::load(src, h, cb, s);
  SpinorFmt<POUT>::store(dst, h, cb, s);
}

// out = diag(Du, Du, Dl, Dl) in, site by site (in == out allowed)
template <int PREC>
__global__ void diag_kernel(int h, const char* in, size_t istride, char* out, size_t ostride, double dur,
                            double dui, double dlr, double dli) {
  const int cb = blockIdx.x * FNT + threadIdx.x, r = blockIdx.y;
  if (cb >= h) return;
  typedef typename SpinorFmt<PREC>::real R;
  cpx<R> s[12];
  SpinorFmt<PREC>::load(in + r * istride, h, cb, s);
  const cpx<R> Du = mk<R>((R)dur, (R)dui), Dl = mk<R>((R)dlr, (R)dli);
#pragma unroll
  for (int k = 0; k < 12; ++k) s[k] = ((k < 6) ? Du : Dl) * s[k];
  SpinorFmt<PREC>::store(out + r * ostride, h, cb, s);
}

#define TM_PREC_SWITCH(prec, F)        \
  switch (prec) {                      \
    case TM_F64: {                     \
      constexpr int P = TM_F64;        \
      F;                               \
    } break;                           \
    case TM_F32: {                     \
      constexpr int P = TM_F32;        \
      F;                               \
    } break;                           \
    case TM_DF64: {                    \
      constexpr int P = TM_DF64;       \
      F;                               \
    } break;                           \
    default: {                         \
      constexpr int P = TM_F16;        \
      F;                               \
    } break;                           \
  }

tm_status pack_full_parity(tm_lattice lat, int prec, void* dst, const double* src_full, int parity, int g5,
                           cudaStream_t s) {
  const Geom& g = lat->geom;
  const unsigned nb = (unsigned)((g.h + FNT - 1) / FNT);
  TM_PREC_SWITCH(prec, (pack_full_kernel<P><<<nb, FNT, 0, s>>>(g, src_full, static_cast<char*>(dst), parity, g5)));
  count_launch();
  return cuda_check(cudaGetLastError(), "pack kernel");
}

tm_status unpack_full_parity(tm_lattice lat, int prec, double* dst_full, const void* src, int parity, int g5,
                             cudaStream_t s) {
  const Geom& g = lat->geom;
  const unsigned nb = (unsigned)((g.h + FNT - 1) / FNT);
  TM_PREC_SWITCH(prec,
                 (unpack_full_kernel<P><<<nb, FNT, 0, s>>>(g, static_cast<const char*>(src), dst_full, parity, g5)));
  count_launch();
  return cuda_check(cudaGetLastError(), "unpack kernel");
}

tm_status convert_half(tm_lattice lat, int prec_out, void* dst, int prec_in, const void* src, cudaStream_t s) {
  const int h = lat->geom.h;
  const unsigned nb = (unsigned)((h + FNT - 1) / FNT);
  const char* in = static_cast<const char*>(src);
  char* out = static_cast<char*>(dst);
#define TM_CONV(A, B) \
  if (prec_in == A && prec_out == B) convert_kernel<A, B><<<nb, FNT, 0, s>>>(h, in, out);
  TM_CONV(TM_F64, TM_F64)
  TM_CONV(TM_F64, TM_F32)
  TM_CONV(TM_F64, TM_F16)
  TM_CONV(TM_F32, TM_F64)
  TM_CONV(TM_F32, TM_F32)
  TM_CONV(TM_F32, TM_F16)
  TM_CONV(TM_F16, TM_F64)
  TM_CONV(TM_F16, TM_F32)
  TM_CONV(TM_F16, TM_F16)
  TM_CONV(TM_F64, TM_DF64)
  TM_CONV(TM_DF64, TM_F64)
  TM_CONV(TM_DF64, TM_F32)
  TM_CONV(TM_F32, TM_DF64)
  TM_CONV(TM_DF64, TM_DF64)
#undef TM_CONV
  count_launch();
  return cuda_check(cudaGetLastError(), "convert kernel");
}

tm_status diag_apply(tm_lattice lat, int prec, void* out, const void* in, int nrhs, double dur, double dui,
                     double dlr, double dli, cudaStream_t s) {
  const int h = lat->geom.h;
  const size_t stride = spinor_bytes_per_site(prec) * lat->h;
  dim3 grid((h + FNT - 1) / FNT, nrhs);
  TM_PREC_SWITCH(prec, (diag_kernel<P><<<grid, FNT, 0, s>>>(h, static_cast<const char*>(in), stride,
                                                              static_cast<char*>(out), stride, dur, dui, dlr,
                                                              dli)));
  count_launch();
  return cuda_check(cudaGetLastError(), "diagonal kernel");
}

// Staging of host buffers: returns a device pointer holding (or receiving) `bytes`.
const void* stage_in(tm_lattice lat, int slot, const void* src, size_t bytes, cudaStream_t s, tm_status* st) {
  *st = TM_OK;
  if (is_device_pointer(src)) return src;
  void* d = workspace(lat, slot, bytes, st);
  if (*st != TM_OK) return nullptr;
  *st = cuda_check(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s), "host-to-device copy");
  return d;
}
void* stage_out(tm_lattice lat, int slot, void* dst, size_t bytes, tm_status* st) {
  *st = TM_OK;
  if (is_device_pointer(dst)) return dst;
  return workspace(lat, slot, bytes, st);
}
tm_status stage_out_finish(void* dst, const void* dev, size_t bytes, cudaStream_t s) {
  if (dst == dev) return TM_OK;
  return cuda_check(cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToHost, s), "device-to-host copy");
}

}  // namespace tmq

using namespace tmq;

extern "C" {

tm_status tm_pack_half(tm_lattice lat, tm_prec prec, void* dst, const double* src, int nrhs, void* stream) {
  if (!lat || !dst || !src || nrhs < 1) return set_error(TM_ERR_ARG, "tm_pack_half: bad argument");
  if (prec < TM_F64 || prec > TM_DF64) return set_error(TM_ERR_ARG, "tm_pack_half: precision %d", (int)prec);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tm_status st;
  const void* d = stage_in(lat, WS_STAGE_IN, src, (size_t)nrhs * lat->h * 24 * sizeof(double), s, &st);
  if (st != TM_OK) return st;
  const int h = lat->geom.h;
  dim3 grid((h + FNT - 1) / FNT, nrhs);
  const size_t stride = spinor_bytes_per_site(prec) * lat->h;
  TM_PREC_SWITCH(prec, (pack_half_kernel<P><<<grid, FNT, 0, s>>>(h, static_cast<const double*>(d),
                                                                   static_cast<char*>(dst), stride)));
  count_launch();
  return cuda_check(cudaGetLastError(), "tm_pack_half");
}

tm_status tm_unpack_half(tm_lattice lat, tm_prec prec, double* dst, const void* src, int nrhs, void* stream) {
  if (!lat || !dst || !src || nrhs < 1) return set_error(TM_ERR_ARG, "tm_unpack_half: bad argument");
  if (prec < TM_F64 || prec > TM_DF64) return set_error(TM_ERR_ARG, "tm_unpack_half: precision %d", (int)prec);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tm_status st;
  const size_t bytes = (size_t)nrhs * lat->h * 24 * sizeof(double);
  void* d = stage_out(lat, WS_STAGE_OUT, dst, bytes, &st);
  if (st != TM_OK) return st;
  const int h = lat->geom.h;
  dim3 grid((h + FNT - 1) / FNT, nrhs);
  const size_t stride = spinor_bytes_per_site(prec) * lat->h;
  TM_PREC_SWITCH(prec, (unpack_half_kernel<P><<<grid, FNT, 0, s>>>(h, static_cast<const char*>(src), stride,
                                                                     static_cast<double*>(d))));
  count_launch();
  st = cuda_check(cudaGetLastError(), "tm_unpack_half");
  if (st != TM_OK) return st;
  return stage_out_finish(dst, d, bytes, s);
}

tm_status tm_apply_Mee_inv(tm_lattice lat, void* out, const void* in, int flavour, tm_prec prec, int nrhs,
                           void* stream) {
  if (!lat || !out || !in || nrhs < 1) return set_error(TM_ERR_ARG, "tm_apply_Mee_inv: bad argument");
  if (flavour != 1 && flavour != -1) return set_error(TM_ERR_ARG, "tm_apply_Mee_inv: flavour must be +1 or -1");
  if (prec < TM_F64 || prec > TM_DF64) return set_error(TM_ERR_ARG, "tm_apply_Mee_inv: precision %d", (int)prec);
  const double mut = 2.0 * lat->kappa * lat->mu;
  const double n = 1.0 / (1.0 + mut * mut);
  return diag_apply(lat, prec, out, in, nrhs, n, -flavour * mut * n, n, flavour * mut * n,
                    static_cast<cudaStream_t>(stream));
}

}  // extern "C"
