// tm_internal.cuh -- types and device helpers shared by the library's translation units.
//
// Layouts (see include/tm.h for the public part):
//   half spinor field  per precision, blocks of 16 bytes, block-major ("SoA"): block k of
//                      site cb at byte offset (k * h + cb) * 16, so a warp reading block k of
//                      32 consecutive sites issues one fully coalesced 512-byte request.
//   gauge copy         per parity p (2), per direction mu (4): the link U_mu(x) of every
//                      site x of parity p, per 16-byte block, per site cb (the backward hop
//                      of a site reads its neighbour's link from the other parity's slabs
//                      and applies the adjoint); a link of R reals in storage type S takes
//                      R * sizeof(S) bytes = NB full 16-byte blocks plus a tail of 0, 4 or 8
//                      bytes stored in its own block-major array after the full blocks.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "tm.h"

namespace tmq {

// ------------------------------------------------------------------ complex ---
template <typename R>
struct cpx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cpx<R> mk(R a, R b) {
  return {a, b};
}
template <typename R>
__device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) {
  return {a.re + b.re, a.im + b.im};
}
template <typename R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) {
  return {a.re - b.re, a.im - b.im};
}
template <typename R>
__device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) {
  return {s * a.re, s * a.im};
}
template <typename R>
__device__ __forceinline__ cpx<R> cj(cpx<R> a) {
  return {a.re, -a.im};
}
// conj(a) * b
template <typename R>
__device__ __forceinline__ cpx<R> cjmul(cpx<R> a, cpx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cpx<R> times_i(cpx<R> a) {
  return {-a.im, a.re};
}
template <typename R>
__device__ __forceinline__ cpx<R> times_mi(cpx<R> a) {
  return {a.im, -a.re};
}
template <typename R>
__device__ __forceinline__ R norm2(cpx<R> a) {
  return a.re * a.re + a.im * a.im;
}

// Fused multiply-add a * b + c with one rounding, per arithmetic type.
template <typename R>
__device__ __forceinline__ R fmadd(R a, R b, R c);
template <>
__device__ __forceinline__ float fmadd<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fmadd<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// ------------------------------------------------------------ two-lane FP32 ---
// A pair of FP32 numbers, one per lattice site, for kernels in which a thread computes two
// output sites: every operation acts on both lanes with one packed FP32 instruction (sm_100 and
// later), so the FP32 arithmetic of two sites costs the issue slots of one.  Each lane rounds as
// the scalar operation would (IEEE round to nearest).
struct f2 {
  float2 v;
  f2() = default;
  __device__ __forceinline__ f2(float2 a) : v(a) {}
  __device__ __forceinline__ f2(float a) : v(make_float2(a, a)) {}
  __device__ __forceinline__ f2(int a) : v(make_float2((float)a, (float)a)) {}
  __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
};
__device__ __forceinline__ f2 operator-(f2 a) { return f2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return f2(__fadd2_rn(a.v, (-b).v)); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
template <>
__device__ __forceinline__ f2 fmadd<f2>(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }
// complex products of pairs as FMA chains (the scalar types get them from FMA contraction)
__device__ __forceinline__ cpx<f2> operator*(cpx<f2> a, cpx<f2> b) {
  return {fmadd(a.re, b.re, -(a.im * b.im)), fmadd(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ cpx<f2> cjmul(cpx<f2> a, cpx<f2> b) {
  return {fmadd(a.re, b.re, a.im * b.im), fmadd(a.re, b.im, -(a.im * b.re))};
}
__device__ __forceinline__ f2 norm2(cpx<f2> a) { return fmadd(a.re, a.re, a.im * a.im); }

// ------------------------------------------------------------- double-float ---
// A real number held as the unevaluated sum hi + lo of two FP32 numbers ("double-word"
// arithmetic, Dekker 1971).  The building blocks are the error-free transformations TwoSum
// (Knuth; exact: s + e = a + b) and TwoProd via FMA (exact: p + e = a * b), and the addition
// and multiplication of double-word numbers as analysed by Joldes, Muller and Popescu (ACM
// TOMS 2017): relative error about 3 * 2^-48 and 5 * 2^-48, so about 48 significant bits,
// with the FP32 exponent range.  All of it runs on the FP32 pipes, which on GB300 issue
// about 58 times the FP64 rate.
struct dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  __device__ dd(float f) : hi(f), lo(0.f) {}
  __device__ dd(int i) : hi((float)i), lo(0.f) {}
  __device__ dd(double d) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
  }
  __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __device__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ float dd_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}
__device__ __forceinline__ float dd_fast_two_sum(float a, float b, float& e) {  // needs |a| >= |b|
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}
__device__ __forceinline__ dd operator+(dd x, dd y) {
  float e, f;
  float s = dd_two_sum(x.hi, y.hi, e);
  const float t = dd_two_sum(x.lo, y.lo, f);
  e = __fadd_rn(e, t);
  float g;
  s = dd_fast_two_sum(s, e, g);
  g = __fadd_rn(g, f);
  float lo;
  s = dd_fast_two_sum(s, g, lo);
  return dd(s, lo);
}
__device__ __forceinline__ dd operator-(dd x) { return dd(-x.hi, -x.lo); }
__device__ __forceinline__ dd operator-(dd x, dd y) { return x + (-y); }
__device__ __forceinline__ dd operator*(dd x, dd y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  float lo;
  const float s = dd_fast_two_sum(p, e, lo);
  return dd(s, lo);
}

// ------------------------------------------------------------------ geometry ---
// T x L^3 lattice, checkerboard index cb = lex / 2 within one parity.
struct Geom {
  int T, L, Lh;      // Lh = L / 2
  int h;             // sites per parity
  int sy, sz, st;    // cb strides of y, z, t: Lh, L*Lh, L*L*Lh
};

struct SiteCoord {
  int t, z, y, x;
};

__device__ __forceinline__ SiteCoord site_of(const Geom& g, int cb, int parity) {
  SiteCoord c;
  int xh = cb % g.Lh;
  int r = cb / g.Lh;
  c.y = r % g.L;
  r /= g.L;
  c.z = r % g.L;
  c.t = r / g.L;
  c.x = 2 * xh + ((c.t + c.z + c.y + parity) & 1);
  return c;
}

// cb indices of the 8 neighbours: nb[mu] = x + mu^, nb[4 + mu] = x - mu^ (periodic wrap).
__device__ __forceinline__ void neighbours(const Geom& g, int cb, const SiteCoord& c, int nb[8]) {
  const int row = cb - (c.x >> 1);  // cb of (t, z, y, x = 0 or 1)
  // t
  nb[0] = (c.t == g.T - 1) ? cb - (g.T - 1) * g.st : cb + g.st;
  nb[4] = (c.t == 0) ? cb + (g.T - 1) * g.st : cb - g.st;
  // x
  const int xp = (c.x == g.L - 1) ? 0 : c.x + 1;
  const int xm = (c.x == 0) ? g.L - 1 : c.x - 1;
  nb[1] = row + (xp >> 1);
  nb[5] = row + (xm >> 1);
  // y
  nb[2] = (c.y == g.L - 1) ? cb - (g.L - 1) * g.sy : cb + g.sy;
  nb[6] = (c.y == 0) ? cb + (g.L - 1) * g.sy : cb - g.sy;
  // z
  nb[3] = (c.z == g.L - 1) ? cb - (g.L - 1) * g.sz : cb + g.sz;
  nb[7] = (c.z == 0) ? cb + (g.L - 1) * g.sz : cb - g.sz;
}

// --------------------------------------------------------------- precisions ---
template <int PREC>
struct SpinorFmt;

// Each format provides load/store of the 12 complex components of site i, and
// load_unscaled(), which leaves out the FP16 per-site norm (returned in `scale`, 1 for the
// other formats) so that a caller can apply it after a linear map that halves the data.
// FP64: double2 blocks [12][h]
template <>
struct SpinorFmt<TM_F64> {
  typedef double real;
  static constexpr bool has_norm = false;
  static constexpr size_t bytes_per_site = 192;
  template <typename R>
  __device__ static __forceinline__ void load_unscaled(const void* base, int h, int i, cpx<R> s[12], R& scale) {
    load(base, h, i, s);
    scale = R(1);
  }
  template <typename R>
  __device__ static __forceinline__ void load(const void* base, int h, int i, cpx<R> s[12]) {
    const double2* p = static_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 v = __ldg(p + (size_t)k * h + i);
      s[k] = mk<R>((R)v.x, (R)v.y);
    }
  }
  template <typename R>
  __device__ static __forceinline__ void store(void* base, int h, int i, const cpx<R> s[12]) {
    double2* p = static_cast<double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k) p[(size_t)k * h + i] = make_double2((double)s[k].re, (double)s[k].im);
  }
  // components [kb, ke) only (block-aligned)
  static constexpr int NBLK = 12, CPB = 1;
  template <typename R>
  __device__ static __forceinline__ void load_range(const void* base, int h, int i, cpx<R> s[12], int kb, int ke) {
    const double2* p = static_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k)
      if (k >= kb && k < ke) {
        double2 v = __ldg(p + (size_t)k * h + i);
        s[k] = mk<R>((R)v.x, (R)v.y);
      }
  }
  template <typename R>
  __device__ static __forceinline__ void store_range(void* base, int h, int i, const cpx<R> s[12], int kb, int ke,
                                                     float, bool) {
    double2* p = static_cast<double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k)
      if (k >= kb && k < ke) p[(size_t)k * h + i] = make_double2((double)s[k].re, (double)s[k].im);
  }
};

// FP32: float4 blocks [6][h]
template <>
struct SpinorFmt<TM_F32> {
  typedef float real;
  static constexpr bool has_norm = false;
  static constexpr size_t bytes_per_site = 96;
  template <typename R>
  __device__ static __forceinline__ void load_unscaled(const void* base, int h, int i, cpx<R> s[12], R& scale) {
    load(base, h, i, s);
    scale = R(1);
  }
  template <typename R>
  __device__ static __forceinline__ void load(const void* base, int h, int i, cpx<R> s[12]) {
    const float4* p = static_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float4 v = __ldg(p + (size_t)k * h + i);
      s[2 * k] = mk<R>((R)v.x, (R)v.y);
      s[2 * k + 1] = mk<R>((R)v.z, (R)v.w);
    }
  }
  template <typename R>
  __device__ static __forceinline__ void store(void* base, int h, int i, const cpx<R> s[12]) {
    float4* p = static_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; ++k)
      p[(size_t)k * h + i] = make_float4((float)s[2 * k].re, (float)s[2 * k].im,
                                         (float)s[2 * k + 1].re, (float)s[2 * k + 1].im);
  }
  static constexpr int NBLK = 6, CPB = 2;
  // The site's 24 words as loaded (software-pipelined hopping kernel), and their unpacking.
  __device__ static __forceinline__ void load_words(const void* base, int h, int i, unsigned int w[24]) {
    const uint4* p = static_cast<const uint4*>(base);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const uint4 v = __ldg(p + (size_t)k * h + i);
      w[4 * k] = v.x;
      w[4 * k + 1] = v.y;
      w[4 * k + 2] = v.z;
      w[4 * k + 3] = v.w;
    }
  }
  template <typename R>
  __device__ static __forceinline__ void unpack_words(const unsigned int w[24], cpx<R> s[12], R& scale) {
#pragma unroll
    for (int k = 0; k < 12; ++k) s[k] = mk<R>((R)__uint_as_float(w[2 * k]), (R)__uint_as_float(w[2 * k + 1]));
    scale = R(1);
  }
  template <typename R>
  __device__ static __forceinline__ void load_range(const void* base, int h, int i, cpx<R> s[12], int kb, int ke) {
    const float4* p = static_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (2 * k >= kb && 2 * k < ke) {
        float4 v = __ldg(p + (size_t)k * h + i);
        s[2 * k] = mk<R>((R)v.x, (R)v.y);
        s[2 * k + 1] = mk<R>((R)v.z, (R)v.w);
      }
  }
  template <typename R>
  __device__ static __forceinline__ void store_range(void* base, int h, int i, const cpx<R> s[12], int kb, int ke,
                                                     float, bool) {
    float4* p = static_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (2 * k >= kb && 2 * k < ke)
        p[(size_t)k * h + i] = make_float4((float)s[2 * k].re, (float)s[2 * k].im, (float)s[2 * k + 1].re,
                                           (float)s[2 * k + 1].im);
  }
};

// FP16 + per-site FP32 norm: uint4 blocks [3][h] (8 halves each), then float norm[h].
template <>
struct SpinorFmt<TM_F16> {
  typedef float real;
  static constexpr bool has_norm = true;
  static constexpr size_t bytes_per_site = 52;
  template <typename R>
  __device__ static __forceinline__ void load_unscaled(const void* base, int h, int i, cpx<R> s[12], R& scale) {
    const uint4* p = static_cast<const uint4*>(base);
    const float* nrm = reinterpret_cast<const float*>(p + (size_t)3 * h);
    scale = (R)__ldg(nrm + i);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 v = __ldg(p + (size_t)k * h + i);
      float2 a = h2f(v.x), b = h2f(v.y), c = h2f(v.z), d = h2f(v.w);
      s[4 * k + 0] = mk<R>((R)a.x, (R)a.y);
      s[4 * k + 1] = mk<R>((R)b.x, (R)b.y);
      s[4 * k + 2] = mk<R>((R)c.x, (R)c.y);
      s[4 * k + 3] = mk<R>((R)d.x, (R)d.y);
    }
  }
  // The site's 12 words of halves and its norm as loaded (software-pipelined hopping kernel).
  __device__ static __forceinline__ void load_words(const void* base, int h, int i, unsigned int w[13]) {
    const uint4* p = static_cast<const uint4*>(base);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const uint4 v = __ldg(p + (size_t)k * h + i);
      w[4 * k] = v.x;
      w[4 * k + 1] = v.y;
      w[4 * k + 2] = v.z;
      w[4 * k + 3] = v.w;
    }
    w[12] = __ldg(reinterpret_cast<const unsigned int*>(p + (size_t)3 * h) + i);
  }
  template <typename R>
  __device__ static __forceinline__ void unpack_words(const unsigned int w[13], cpx<R> s[12], R& scale) {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float2 a = h2f(w[k]);
      s[k] = mk<R>((R)a.x, (R)a.y);
    }
    scale = (R)__uint_as_float(w[12]);
  }
  __device__ static __forceinline__ float2 h2f(unsigned int w) {
    __half2 hv = *reinterpret_cast<__half2*>(&w);
    return __half22float2(hv);
  }
  __device__ static __forceinline__ unsigned int f2h(float a, float b) {
    __half2 hv = __floats2half2_rn(a, b);
    return *reinterpret_cast<unsigned int*>(&hv);
  }
  template <typename R>
  __device__ static __forceinline__ void load(const void* base, int h, int i, cpx<R> s[12]) {
    const uint4* p = static_cast<const uint4*>(base);
    const float* nrm = reinterpret_cast<const float*>(p + (size_t)3 * h);
    const float n = __ldg(nrm + i);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 v = __ldg(p + (size_t)k * h + i);
      float2 a = h2f(v.x), b = h2f(v.y), c = h2f(v.z), d = h2f(v.w);
      s[4 * k + 0] = mk<R>((R)(a.x * n), (R)(a.y * n));
      s[4 * k + 1] = mk<R>((R)(b.x * n), (R)(b.y * n));
      s[4 * k + 2] = mk<R>((R)(c.x * n), (R)(c.y * n));
      s[4 * k + 3] = mk<R>((R)(d.x * n), (R)(d.y * n));
    }
  }
  template <typename R>
  __device__ static __forceinline__ void store(void* base, int h, int i, const cpx<R> s[12]) {
    uint4* p = static_cast<uint4*>(base);
    float* nrm = reinterpret_cast<float*>(p + (size_t)3 * h);
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf((float)s[k].re), fabsf((float)s[k].im)));
    const float inv = (m > 0.f) ? 1.0f / m : 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 v;
      v.x = f2h((float)s[4 * k + 0].re * inv, (float)s[4 * k + 0].im * inv);
      v.y = f2h((float)s[4 * k + 1].re * inv, (float)s[4 * k + 1].im * inv);
      v.z = f2h((float)s[4 * k + 2].re * inv, (float)s[4 * k + 2].im * inv);
      v.w = f2h((float)s[4 * k + 3].re * inv, (float)s[4 * k + 3].im * inv);
      p[(size_t)k * h + i] = v;
    }
    nrm[i] = m;
  }
  static constexpr int NBLK = 3, CPB = 4;
  template <typename R>
  __device__ static __forceinline__ void load_range(const void* base, int h, int i, cpx<R> s[12], int kb, int ke) {
    const uint4* p = static_cast<const uint4*>(base);
    const float* nrm = reinterpret_cast<const float*>(p + (size_t)3 * h);
    const float n = __ldg(nrm + i);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (4 * k >= kb && 4 * k < ke) {
        uint4 v = __ldg(p + (size_t)k * h + i);
        float2 a = h2f(v.x), b = h2f(v.y), c = h2f(v.z), d = h2f(v.w);
        s[4 * k + 0] = mk<R>((R)(a.x * n), (R)(a.y * n));
        s[4 * k + 1] = mk<R>((R)(b.x * n), (R)(b.y * n));
        s[4 * k + 2] = mk<R>((R)(c.x * n), (R)(c.y * n));
        s[4 * k + 3] = mk<R>((R)(d.x * n), (R)(d.y * n));
      }
  }
  // m: the site's norm (largest |re| or |im| over all 12 components), computed by the caller
  template <typename R>
  __device__ static __forceinline__ void store_range(void* base, int h, int i, const cpx<R> s[12], int kb, int ke,
                                                     float m, bool write_norm) {
    uint4* p = static_cast<uint4*>(base);
    float* nrm = reinterpret_cast<float*>(p + (size_t)3 * h);
    const float inv = (m > 0.f) ? 1.0f / m : 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (4 * k >= kb && 4 * k < ke) {
        uint4 v;
        v.x = f2h((float)s[4 * k + 0].re * inv, (float)s[4 * k + 0].im * inv);
        v.y = f2h((float)s[4 * k + 1].re * inv, (float)s[4 * k + 1].im * inv);
        v.z = f2h((float)s[4 * k + 2].re * inv, (float)s[4 * k + 2].im * inv);
        v.w = f2h((float)s[4 * k + 3].re * inv, (float)s[4 * k + 3].im * inv);
        p[(size_t)k * h + i] = v;
      }
    if (write_norm) nrm[i] = m;
  }
};

// Precision of the iterated residual that goes with an operator storage precision.
template <int PREC>
struct ResidPrec {
  static constexpr int value = (PREC == TM_F64 || PREC == TM_DF64) ? PREC : TM_F32;
};

// Double-float (TM_DF64): float4 blocks [12][h], block k = (re.hi, re.lo, im.hi, im.lo) of
// complex component k.  Same footprint as FP64, double-float arithmetic.
template <>
struct SpinorFmt<TM_DF64> {
  typedef dd real;
  static constexpr bool has_norm = false;
  static constexpr size_t bytes_per_site = 192;
  static constexpr int NBLK = 12, CPB = 1;
  template <typename R>
  __device__ static __forceinline__ void load(const void* base, int h, int i, cpx<R> s[12]) {
    const float4* p = static_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k) s[k] = conv<R>(__ldg(p + (size_t)k * h + i));
  }
  template <typename R>
  __device__ static __forceinline__ void load_unscaled(const void* base, int h, int i, cpx<R> s[12], R& scale) {
    load(base, h, i, s);
    scale = R(1);
  }
  template <typename R>
  __device__ static __forceinline__ void store(void* base, int h, int i, const cpx<R> s[12]) {
    float4* p = static_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k) p[(size_t)k * h + i] = pack(s[k]);
  }
  template <typename R>
  __device__ static __forceinline__ void load_range(const void* base, int h, int i, cpx<R> s[12], int kb, int ke) {
    const float4* p = static_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k)
      if (k >= kb && k < ke) s[k] = conv<R>(__ldg(p + (size_t)k * h + i));
  }
  template <typename R>
  __device__ static __forceinline__ void store_range(void* base, int h, int i, const cpx<R> s[12], int kb, int ke,
                                                     float, bool) {
    float4* p = static_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k)
      if (k >= kb && k < ke) p[(size_t)k * h + i] = pack(s[k]);
  }
  // conversions: the (hi, lo) pair to the arithmetic type R, and any R to a (hi, lo) pair
  template <typename R>
  __device__ static __forceinline__ cpx<R> conv(float4 v) {
    return mk<R>(R(dd(v.x, v.y)), R(dd(v.z, v.w)));
  }
  __device__ static __forceinline__ float4 pack(const cpx<dd>& z) { return make_float4(z.re.hi, z.re.lo, z.im.hi, z.im.lo); }
  __device__ static __forceinline__ float4 pack(const cpx<double>& z) {
    const dd a(z.re), b(z.im);
    return make_float4(a.hi, a.lo, b.hi, b.lo);
  }
  __device__ static __forceinline__ float4 pack(const cpx<float>& z) { return make_float4(z.re, 0.f, z.im, 0.f); }
};

__host__ __device__ inline size_t spinor_bytes_per_site(int prec) {
  return prec == TM_F64 ? 192 : (prec == TM_F32 ? 96 : (prec == TM_F16 ? 52 : 192));
}

// -------------------------------------------------------------------- links ---
// Storage type per spinor precision: FP64 -> double, FP32 -> float, FP16 -> half.
template <int PREC>
struct LinkStore;
template <>
struct LinkStore<TM_F64> {
  typedef double type;
  static constexpr int size = 8;
};
template <>
struct LinkStore<TM_F32> {
  typedef float type;
  static constexpr int size = 4;
};
template <>
struct LinkStore<TM_F16> {
  typedef __half type;
  static constexpr int size = 2;
};
template <>
struct LinkStore<TM_DF64> {
  typedef dd type;
  static constexpr int size = 8;
};

__host__ __device__ inline int link_elem_size(int prec) {
  return (prec == TM_F64 || prec == TM_DF64) ? 8 : (prec == TM_F32 ? 4 : 2);
}
__host__ __device__ inline size_t link_bytes(int prec, int nreal) {
  return (size_t)nreal * link_elem_size(prec);
}
// byte offset of the (parity, mu) slab inside a gauge copy
__host__ __device__ inline size_t link_slab_offset(int prec, int nreal, int h, int parity, int mu) {
  return (size_t)(parity * 4 + mu) * link_bytes(prec, nreal) * (size_t)h;
}

// Load the R raw reals (as 32-bit words) of link (slab, i).
template <int BYTES>
struct RawWords {
  unsigned int w[BYTES / 4];
};

template <int BYTES>
__device__ __forceinline__ RawWords<BYTES> load_raw(const char* slab, int h, int i) {
  RawWords<BYTES> r;
  constexpr int NB = BYTES / 16;
  constexpr int TAIL = BYTES % 16;
  const uint4* blk = reinterpret_cast<const uint4*>(slab);
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    uint4 q = __ldg(blk + (size_t)j * h + i);
    r.w[4 * j + 0] = q.x;
    r.w[4 * j + 1] = q.y;
    r.w[4 * j + 2] = q.z;
    r.w[4 * j + 3] = q.w;
  }
  if (TAIL == 8) {
    const uint2* t = reinterpret_cast<const uint2*>(slab + (size_t)NB * 16 * h);
    uint2 q = __ldg(t + i);
    r.w[4 * NB + 0] = q.x;
    r.w[4 * NB + 1] = q.y;
  } else if (TAIL == 4) {
    const unsigned int* t = reinterpret_cast<const unsigned int*>(slab + (size_t)NB * 16 * h);
    r.w[4 * NB] = __ldg(t + i);
  }
  return r;
}

template <int BYTES>
__device__ __forceinline__ void store_raw(char* slab, int h, int i, const RawWords<BYTES>& r) {
  constexpr int NB = BYTES / 16;
  constexpr int TAIL = BYTES % 16;
  uint4* blk = reinterpret_cast<uint4*>(slab);
#pragma unroll
  for (int j = 0; j < NB; ++j)
    blk[(size_t)j * h + i] = make_uint4(r.w[4 * j], r.w[4 * j + 1], r.w[4 * j + 2], r.w[4 * j + 3]);
  if (TAIL == 8) {
    uint2* t = reinterpret_cast<uint2*>(slab + (size_t)NB * 16 * h);
    t[i] = make_uint2(r.w[4 * NB], r.w[4 * NB + 1]);
  } else if (TAIL == 4) {
    unsigned int* t = reinterpret_cast<unsigned int*>(slab + (size_t)NB * 16 * h);
    t[i] = r.w[4 * NB];
  }
}

// real number k of a raw link in storage type S
template <typename S, int BYTES>
struct RawGet;
template <int BYTES>
struct RawGet<double, BYTES> {
  __device__ static __forceinline__ double get(const RawWords<BYTES>& r, int k) {
    return __hiloint2double((int)r.w[2 * k + 1], (int)r.w[2 * k]);
  }
  __device__ static __forceinline__ void put(RawWords<BYTES>& r, int k, double v) {
    r.w[2 * k] = (unsigned)__double2loint(v);
    r.w[2 * k + 1] = (unsigned)__double2hiint(v);
  }
};
template <int BYTES>
struct RawGet<float, BYTES> {
  __device__ static __forceinline__ float get(const RawWords<BYTES>& r, int k) {
    return __uint_as_float(r.w[k]);
  }
  __device__ static __forceinline__ void put(RawWords<BYTES>& r, int k, float v) {
    r.w[k] = __float_as_uint(v);
  }
};
template <int BYTES>
struct RawGet<dd, BYTES> {
  __device__ static __forceinline__ dd get(const RawWords<BYTES>& r, int k) {
    return dd(__uint_as_float(r.w[2 * k]), __uint_as_float(r.w[2 * k + 1]));
  }
  __device__ static __forceinline__ void put(RawWords<BYTES>& r, int k, dd v) {
    r.w[2 * k] = __float_as_uint(v.hi);
    r.w[2 * k + 1] = __float_as_uint(v.lo);
  }
};
template <int BYTES>
struct RawGet<__half, BYTES> {
  __device__ static __forceinline__ float get(const RawWords<BYTES>& r, int k) {
    unsigned short bits = (unsigned short)((r.w[k >> 1] >> (16 * (k & 1))) & 0xffffu);
    return __half2float(__ushort_as_half(bits));
  }
  __device__ static __forceinline__ void put(RawWords<BYTES>& r, int k, float v) {
    unsigned int bits = (unsigned int)__half_as_ushort(__float2half_rn(v));
    unsigned int sh = 16 * (k & 1);
    r.w[k >> 1] = (r.w[k >> 1] & ~(0xffffu << sh)) | (bits << sh);
  }
};

// 3x3 complex matrix in registers, row-major
template <typename R>
struct Mat3 {
  cpx<R> m[3][3];
};

// Reconstruct a link from its stored reals.
//  18: all 9 entries, row-major (re, im).
//  12: rows 0 and 1; row 2 = conj(row0 x row1) (det = 1).
//   8: a1, a2 (row 0, columns 1, 2), b0 (row 1, column 0), arg(a0)/pi, arg(c0)/pi, where
//      a, b, c are rows 0, 1, 2.  |a0| follows from the unit norm of row 0, |c0| from the
//      unit norm of column 0, b1 and b2 from orthogonality of rows 0 and 1 together with
//      c0 = conj(a1 b2 - a2 b1), and row 2 from c = conj(a x b).
template <typename R, typename S, int NREAL>
struct LinkRecon;

template <typename R, typename S>
struct LinkRecon<R, S, 18> {
  static constexpr int BYTES = 18 * (int)sizeof(S);
  __device__ static __forceinline__ void unpack(const RawWords<BYTES>& r, Mat3<R>& U) {
    from_reals([&](int k) { return (R)RawGet<S, BYTES>::get(r, k); }, U);
  }
  // the matrix from its stored reals, get(k) = real number k (one site, or a pair of sites)
  template <class Get>
  __device__ static __forceinline__ void from_reals(Get get, Mat3<R>& U) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) U.m[a][b] = mk<R>(get(2 * (3 * a + b)), get(2 * (3 * a + b) + 1));
  }
  __device__ static __forceinline__ void pack(RawWords<BYTES>& r, const Mat3<double>& U) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        RawGet<S, BYTES>::put(r, 2 * (3 * a + b), (S)U.m[a][b].re);
        RawGet<S, BYTES>::put(r, 2 * (3 * a + b) + 1, (S)U.m[a][b].im);
      }
  }
};

// conj(a b - c d) as two FMA chains (the entries of row 3 = conj(row 1 x row 2))
template <typename R>
__device__ __forceinline__ cpx<R> cross_conj(cpx<R> a, cpx<R> b, cpx<R> c, cpx<R> d) {
  R re = a.re * b.re;
  re = fmadd(-a.im, b.im, re);
  re = fmadd(-c.re, d.re, re);
  re = fmadd(c.im, d.im, re);
  R im = c.re * d.im;
  im = fmadd(c.im, d.re, im);
  im = fmadd(-a.re, b.im, im);
  im = fmadd(-a.im, b.re, im);
  return mk<R>(re, im);
}
template <>
__device__ __forceinline__ cpx<dd> cross_conj<dd>(cpx<dd> a, cpx<dd> b, cpx<dd> c, cpx<dd> d) {
  return cj(a * b - c * d);
}

template <typename R>
__device__ __forceinline__ void third_row(Mat3<R>& U) {
  U.m[2][0] = cross_conj(U.m[0][1], U.m[1][2], U.m[0][2], U.m[1][1]);
  U.m[2][1] = cross_conj(U.m[0][2], U.m[1][0], U.m[0][0], U.m[1][2]);
  U.m[2][2] = cross_conj(U.m[0][0], U.m[1][1], U.m[0][1], U.m[1][0]);
}

template <typename R, typename S>
struct LinkRecon<R, S, 12> {
  static constexpr int BYTES = 12 * (int)sizeof(S);
  __device__ static __forceinline__ void unpack(const RawWords<BYTES>& r, Mat3<R>& U) {
    from_reals([&](int k) { return (R)RawGet<S, BYTES>::get(r, k); }, U);
  }
  template <class Get>
  __device__ static __forceinline__ void from_reals(Get get, Mat3<R>& U) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) U.m[a][b] = mk<R>(get(2 * (3 * a + b)), get(2 * (3 * a + b) + 1));
    third_row(U);
  }
  __device__ static __forceinline__ void pack(RawWords<BYTES>& r, const Mat3<double>& U) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        RawGet<S, BYTES>::put(r, 2 * (3 * a + b), (S)U.m[a][b].re);
        RawGet<S, BYTES>::put(r, 2 * (3 * a + b) + 1, (S)U.m[a][b].im);
      }
  }
};

// Square root of a non-negative number (0 for a negative rounding residue), reciprocal and
// sin/cos of pi v for the 8-real reconstruction.  FP64 uses the accurate library functions.  The
// reduced-precision operators (FP32 arithmetic) use the hardware approximations: reciprocal
// square root (v * rsqrt(v), a few ulp), reciprocal (2 ulp), sine/cosine (absolute error ~4e-7
// on |x| <= pi), all far below FP16 storage and within the FP32 8-real parity bound; the IEEE
// square root and reciprocal carry range checks and a slow path that cost ~190 instructions per
// output site.
__device__ __forceinline__ double sqrt_nn(double v) { return sqrt(v > 0.0 ? v : 0.0); }
__device__ __forceinline__ float sqrt_nn(float v) { return v > 0.f ? v * rsqrtf(v) : 0.f; }
__device__ __forceinline__ f2 sqrt_nn(f2 v) { return f2(sqrt_nn(v.v.x), sqrt_nn(v.v.y)); }
__device__ __forceinline__ double recip_(double v) { return 1.0 / v; }
__device__ __forceinline__ float recip_(float v) { return __fdividef(1.0f, v); }
__device__ __forceinline__ f2 recip_(f2 v) { return f2(recip_(v.v.x), recip_(v.v.y)); }
__device__ __forceinline__ void sincospi_(double v, double* s, double* c) { sincospi(v, s, c); }
__device__ __forceinline__ void sincospi_(float v, float* s, float* c) { __sincosf(v * 3.14159265358979323846f, s, c); }
__device__ __forceinline__ void sincospi_(f2 v, f2* s, f2* c) {
  sincospi_(v.v.x, &s->v.x, &c->v.x);
  sincospi_(v.v.y, &s->v.y, &c->v.y);
}

template <typename R, typename S>
struct LinkRecon<R, S, 8> {
  static constexpr int BYTES = 8 * (int)sizeof(S);
  __device__ static __forceinline__ void unpack(const RawWords<BYTES>& r, Mat3<R>& U) {
    from_reals([&](int k) { return (R)RawGet<S, BYTES>::get(r, k); }, U);
  }
  template <class Get>
  __device__ static __forceinline__ void from_reals(Get get, Mat3<R>& U) {
    const cpx<R> a1 = mk<R>(get(0), get(1));
    const cpx<R> a2 = mk<R>(get(2), get(3));
    const cpx<R> b0 = mk<R>(get(4), get(5));
    const R tha = get(6), thc = get(7);    // phases / pi
    const R N = norm2(a1) + norm2(a2);       // = 1 - |a0|^2
    const R ma0 = sqrt_nn(R(1) - N);
    const R mc0 = sqrt_nn(N - norm2(b0));    // = 1 - |a0|^2 - |b0|^2
    R sa, ca, sc, cc;
    sincospi_(tha, &sa, &ca);
    sincospi_(thc, &sc, &cc);
    const cpx<R> a0 = mk<R>(ma0 * ca, ma0 * sa);
    const cpx<R> c0 = mk<R>(mc0 * cc, mc0 * sc);
    const R invN = recip_(N);
    // b1 = -(b0 conj(a0) a1 + conj(a2) conj(c0)) / N ;  b2 = (conj(a1) conj(c0) - a2 b0 conj(a0)) / N
    const cpx<R> b0ca0 = cjmul(a0, b0);  // conj(a0) b0
    const cpx<R> b1 = (-invN) * (b0ca0 * a1 + cj(a2 * c0));
    const cpx<R> b2 = invN * (cj(a1 * c0) - a2 * b0ca0);
    U.m[0][0] = a0;
    U.m[0][1] = a1;
    U.m[0][2] = a2;
    U.m[1][0] = b0;
    U.m[1][1] = b1;
    U.m[1][2] = b2;
    // row 3 = conj(row 1 x row 2); its first entry is c0 itself
    U.m[2][0] = c0;
    U.m[2][1] = cross_conj(a2, b0, a0, b2);
    U.m[2][2] = cross_conj(a0, b1, a1, b0);
  }
  __device__ static __forceinline__ void pack(RawWords<BYTES>& r, const Mat3<double>& U) {
    typedef RawGet<S, BYTES> G;
    G::put(r, 0, (S)U.m[0][1].re);
    G::put(r, 1, (S)U.m[0][1].im);
    G::put(r, 2, (S)U.m[0][2].re);
    G::put(r, 3, (S)U.m[0][2].im);
    G::put(r, 4, (S)U.m[1][0].re);
    G::put(r, 5, (S)U.m[1][0].im);
    G::put(r, 6, (S)(atan2(U.m[0][0].im, U.m[0][0].re) / 3.14159265358979323846));
    G::put(r, 7, (S)(atan2(U.m[2][0].im, U.m[2][0].re) / 3.14159265358979323846));
  }
};

// ---------------------------------------------------------------- epilogue ---
// out_s = D_s (c * hop_s + E_s * y_s), D and E complex per chirality (s = 0, 1 upper; 2, 3 lower).
struct EpiCoef {
  double c;
  double d_up_re, d_up_im, d_lo_re, d_lo_im;
  double e_up_re, e_up_im, e_lo_re, e_lo_im;
  double m_up_re, m_up_im, m_lo_re, m_lo_im;  // the inverse of D (residual epilogue, mode 3)
  // For the FP32 arithmetic of the FP32 / FP16 kernels: D c and D E formed in FP64 and rounded
  // once, on the host (epi_finish).  GB300 runs FP64 and FP64 -> FP32 conversions at ~1/64 of the
  // FP32 rate; forming these per thread kept the FP64 pipe 44% busy in the hopping launches with
  // a y input (FP16/12 on 32^3 x 64).
  float f_dcu_re, f_dcu_im, f_dcl_re, f_dcl_im;
  float f_deu_re, f_deu_im, f_del_re, f_del_im;
};
EpiCoef epi_finish(EpiCoef e);  // fills the FP32 fields from the FP64 ones

// Epilogue coefficient sets used by the operators (eq. eo0, eo2, eo3, App. B.2).
EpiCoef epi_plain();                                    // out = H in
EpiCoef epi_mdiag_inv_hop(double mut, int f);           // out = (M_ee^f)^-1 H in
EpiCoef epi_scaled_minv(double mut, int f, double c);   // out = (M_ee^f)^-1 (c H in + y); m = M_ee^f
EpiCoef epi_full_M(double kappa, double mut, int f);    // out = (1 + i f mut g5) y - kappa H in
EpiCoef epi_schur_q(double kappa, double mut, int f);   // out = g5 [(1 + i f mut g5) y - kappa^2 H in]
EpiCoef epi_g5_y_plus(double c);                        // out = g5 (y + c H in)

// ----------------------------------------------------------------- CG state ---
// Scalars of one CG system, kept in device memory so that the iteration never
// needs the host.  Written only by the last block of the kernel that finishes a
// reduction ("last block done" pattern), read by the following kernels.
struct CGState {
  double rr;        // ||r||^2 of the iterated residual
  double pAp;       // <p, A p> = ||Qhat^-f p||^2
  double alpha, beta;
  double stop2;     // stop when rr < stop2 (= tol^2 ||b||^2 for the active stage)
  double rr_ref;    // reliable updates: ||r||^2 at the last update
  double delta2;    // reliable updates: trigger when rr < delta2 * rr_ref
  double rr_min;    // smallest ||r||^2 of this stage
  double grow2;     // divergence guard: stop the stage when rr > grow2 * rr_min (0: off)
  int iter;         // iterations done in this stage
  int max_iter;
  int done;         // iteration loop finished (converged, out of iterations, or failed)
  int applied;      // iteration count whose solution/direction update has been applied
  int converged;
  int nonfinite;
  int want_update;  // reliable updates: the sloppy residual fell below the trigger
  int diverged;     // the stage ended because the iterated residual grew (restart p)
  int loops;        // graph loop: iteration bodies executed in this stage
  int loop_cap;     // graph loop: hard bound on loops (the loop always ends)
  // batched solves, the FP64 service of a stopped system inside the solve's graph
  int finished;     // the system is done for good (converged, failed or out of iterations)
  int ok;           // converged: the FP64 residual met the tolerance
  int serv_iter;    // iteration count at the last service (no progress since: breakdown)
  int updates;      // FP64 residual recomputations
  int missed;       // sloppy stages that reported convergence the FP64 residual did not confirm
  int bad;          // stages dropped for a non-finite value
  int rearm;        // set by the service for the systems it resumed (the conversions follow)
  int restart;      // ... whose search direction restarts from the FP64 residual
  double rr64;      // the last FP64 residual ||b' - A X||^2
};

// What the last block does with the sum of a reduction.
enum FinKind : int {
  FIN_STORE = 0,     // result[sys] = sum
  FIN_CG_ALPHA = 1,  // st.pAp = sum; st.alpha = st.rr / sum
  FIN_CG_RR = 2      // st.beta = sum / st.rr; st.rr = sum; st.iter++; convergence / trigger tests
};

struct Reduce {
  double* partials;    // [nsys][nblocks]
  unsigned* counters;  // [nsys], zero between uses
  double* result;      // [nsys] (FIN_STORE)
  CGState* st;         // [nsys] (FIN_CG_*)
  int kind;
  // optional: [nsys][ceil(nblocks / NT)] group counters, zero between uses, for grids of many
  // blocks (two-level sum, grid_reduce2)
  unsigned* gcounters = nullptr;
};

__device__ __forceinline__ void fin_apply(const Reduce& red, int sys, double sum) {
  if (red.kind == FIN_STORE) {
    red.result[sys] = sum;
  } else if (red.kind == FIN_CG_ALPHA) {
    CGState& s = red.st[sys];
    s.pAp = sum;
    if (!(sum > 0.0) || !isfinite(sum) || !isfinite(s.rr)) {
      s.nonfinite = (!isfinite(sum) || !isfinite(s.rr)) ? 1 : s.nonfinite;
      s.alpha = 0.0;
      s.done = 1;
    } else {
      s.alpha = s.rr / sum;
    }
  } else if (red.kind == FIN_CG_RR) {
    CGState& s = red.st[sys];
    if (!isfinite(sum)) {
      s.nonfinite = 1;
      s.done = 1;
      s.beta = 0.0;
      return;
    }
    s.beta = sum / s.rr;
    s.rr = sum;
    s.iter += 1;
    if (sum < s.rr_min) s.rr_min = sum;
    if (sum < s.stop2) {
      s.converged = 1;
      s.done = 1;
    } else if (s.iter >= s.max_iter) {
      s.done = 1;
    } else if (s.delta2 > 0.0 && sum < s.delta2 * s.rr_ref) {
      s.want_update = 1;
      s.done = 1;
    } else if (s.grow2 > 0.0 && sum > s.grow2 * s.rr_min) {
      s.want_update = 1;
      s.diverged = 1;
      s.done = 1;
    }
  }
}

// A thread's own sum over its site's components, before the FP64 sum across threads and
// blocks: FP32 when the terms are FP32 numbers (FP32 / FP16 storage), FP64 otherwise.  GB300
// retires FP64 adds at ~1/60 of the FP32 rate; converting and adding a site's 24 terms in
// FP64 cost more than the kernel's memory traffic (a 6 MB copy kernel with such a norm:
// 8.9 us per launch against 2.8 us with the per-thread sum in FP32).
template <typename R>
struct SiteSum {
  typedef double type;
};
template <>
struct SiteSum<float> {
  typedef float type;
};

// Arrival at a grid-wide counter: a device-scope atomic increment with release semantics (the
// caller's earlier writes are visible to whoever observes the increment) and acquire semantics
// (the caller sees the writes released by the increments before it).  Returns the old value.
__device__ __forceinline__ unsigned arrive_acq_rel(unsigned* counter) {
  unsigned prev;
  asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(prev) : "l"(counter) : "memory");
  return prev;
}

// Deterministic block sum of a double (fixed shuffle tree, then warps in order).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) s += sh[w];
  }
  return s;  // valid in thread 0
}

// The same for FP32 per-thread sums (FP32 / FP16 storage): the warp's shuffle tree in FP32, the
// warps and everything after in FP64.  GB300 runs FP64 adds at ~1/64 of the FP32 rate; the FP64
// tree cost 5 of them per thread.
template <int NT>
__device__ __forceinline__ double block_sum(float v, double* sh) {
#ifdef TM_WARP_SUM_F64
  return block_sum<NT>((double)v, sh);
#else
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) s += sh[w];
  }
  return s;  // valid in thread 0
#endif
}

// Two levels, for grids of many blocks: the blocks form groups of NT (blocks g NT .. g NT + NT - 1);
// the last block of a group to arrive sums its group's partials (one per thread) in fixed order,
// writes the sum over the group's first partial and arrives at the system's counter; the last
// group sums the group sums in fixed order and finalises.  A single last block summing 83 k
// partials (one hopping launch on 48^3 x 96) waits out ~80 rounds of L2 loads.
template <int NT>
__device__ __forceinline__ void grid_reduce2(const Reduce& red, int sys, int nblocks, int bid, double bsum,
                                             double* sh) {
  __shared__ bool lastg, lasttop;
  const size_t base = (size_t)sys * nblocks;
  const int ngroups = (nblocks + NT - 1) / NT;
  const int g = bid / NT;
  const int gsize = min(NT, nblocks - g * NT);
  unsigned* gctr = red.gcounters + (size_t)sys * ngroups + g;
  if (threadIdx.x == 0) {
    red.partials[base + bid] = bsum;
    lastg = (arrive_acq_rel(gctr) == (unsigned)gsize - 1);
  }
  __syncthreads();
  if (!lastg) return;
  // every partial of the group is visible, as in grid_reduce: through the counter's acquire
  const double v = (int)threadIdx.x < gsize ? __ldcg(red.partials + base + (size_t)g * NT + threadIdx.x) : 0.0;
  const double gs = block_sum<NT>(v, sh);
  if (threadIdx.x == 0) {
    *gctr = 0u;
    red.partials[base + (size_t)g * NT] = gs;
    lasttop = (arrive_acq_rel(red.counters + sys) == (unsigned)ngroups - 1);
  }
  __syncthreads();
  if (!lasttop) return;
  double w = 0.0;
  for (int b0 = threadIdx.x; b0 < ngroups; b0 += 8 * NT) {
    double t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = b0 + u * NT;
      t[u] = k < ngroups ? __ldcg(red.partials + base + (size_t)k * NT) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) w += t[u];
  }
  __syncthreads();
  const double tot = block_sum<NT>(w, sh);
  if (threadIdx.x == 0) {
    fin_apply(red, sys, tot);
    red.counters[sys] = 0u;
  }
}

// Called by every thread of every block with the block's contribution (valid in thread 0).
// The last block of system `sys` to arrive sums the partials in fixed order and finalises (two
// levels when the caller provides group counters and the grid has more than 64 NT blocks: below
// that the single tail's few rounds of loads cost less than the second arrival -- 16^3 x 32, 1024
// blocks: 199 mixed solves/s with one level, 185 with two; 48^3 x 96, 83 k blocks: 0.76 -> 0.80).
template <int NT>
__device__ __forceinline__ void grid_reduce(const Reduce& red, int sys, int nblocks, int bid, double bsum,
                                            double* sh) {
  if (red.gcounters != nullptr && nblocks > 64 * NT) {
    grid_reduce2<NT>(red, sys, nblocks, bid, bsum, sh);
    return;
  }
  __shared__ bool last;
  if (threadIdx.x == 0) {
    red.partials[(size_t)sys * nblocks + bid] = bsum;
    last = (arrive_acq_rel(red.counters + sys) == (unsigned)nblocks - 1);
  }
  __syncthreads();
  if (!last) return;
  // thread t adds partials t, t + NT, t + 2 NT, ... in that order; the loads of a group of 16
  // are issued together (L2, bypassing L1) so the tail pays one round trip per group.  Every
  // other block's partial is visible here: its release increment precedes this block's
  // acquiring one in the counter's modification order, and the barrier orders this block's
  // threads after that acquire.
  double v = 0.0;
  const double* parts = red.partials + (size_t)sys * nblocks;
  for (int base = threadIdx.x; base < nblocks; base += 16 * NT) {
    double t[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int k = base + u * NT;
      t[u] = k < nblocks ? __ldcg(parts + k) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) v += t[u];
  }
  __syncthreads();
  double tot = block_sum<NT>(v, sh);
  if (threadIdx.x == 0) {
    fin_apply(red, sys, tot);
    red.counters[sys] = 0u;
  }
}

// ------------------------------------------------ programmatic dependent launch ---
// A kernel launched with the programmatic-stream-serialization attribute may be scheduled while
// its predecessor in the stream is still running: pdl_wait() holds its threads until the
// predecessor has completed and its writes are visible, pdl_allow() lets the next kernel be
// scheduled once every block of this one has called it.  Both are no-ops when the kernel was
// launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_allow() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// -------------------------------------------------------------- host side ---
void count_launch(unsigned n = 1);
bool use_pdl();  // programmatic dependent launch of the iteration kernels (TM_PDL=1; off by default)

// Launches `kernel` on `s` with the programmatic-stream-serialization attribute when use_pdl().
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = use_pdl() ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
tm_status set_error(tm_status st, const char* fmt, ...);
tm_status cuda_check(cudaError_t e, const char* what);

}  // namespace tmq

// The lattice object (host side).
struct tm_lattice_s {
  int T, L;
  double kappa, mu;
  tmq::Geom geom;
  size_t V, h;
  int device;
  bool has_gauge;
  double* U_canon;          // 72 V doubles, canonical copy on the device
  void* links[4][3];        // gauge copies [prec][0:18, 1:12, 2:8], built on demand
  int hop_tps[4][3];        // hopping kernel per form (autotuned): threads per site 1, 2, 4, or TM_HOP_PIPELINED
  int hop_tps_forced[4][3]; // set by tm_set_hop_threads: the tuner keeps hands off
  // work space
  void* ws[32];             // half-field buffers, allocated on demand
  size_t ws_bytes[32];
  double* partials;         // reduction partials
  size_t partials_count;
  unsigned* counters;       // reduction counters (zeroed)
  size_t counters_count;
  unsigned* gcounters;      // group counters of two-level reductions (zeroed; allocated once, h / 1024 + 16)
  double* dscalars;         // small device scalar scratch
  tmq::CGState* cgstate;     // device CG state array
  size_t cgstate_count;
  tmq::CGState* cgstate_host;  // pinned host mirror
  double* stage;            // device staging buffer for host in/out of full fields
  size_t stage_bytes;
  int* flag_host;           // pinned host word
  struct StageGraph {       // instantiated CUDA graphs of one CG stage loop (see tm_solver.cu)
    bool valid;
    int prec, nreal, px, f;
    const void *x, *r, *p, *T, *W;
    double kappa, mu;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
  } graphs[8];
  int graph_next;           // round-robin replacement slot
  struct AuxGraph {         // graphs of the other solvers' stage loops, keyed by 16 words
    bool valid;
    unsigned long long key[16];
    cudaGraph_t graph;
    cudaGraphExec_t exec;
  } aux_graphs[8];
  int aux_next;
};

namespace tmq {
inline int link_index(int nreal) { return nreal == 18 ? 0 : (nreal == 12 ? 1 : 2); }
tm_status ensure_links(tm_lattice lat, int prec, int nreal, cudaStream_t s);
void* workspace(tm_lattice lat, int slot, size_t bytes, tm_status* st);
tm_status ensure_reduce(tm_lattice lat, size_t nparts, size_t ncounters);
tm_status ensure_cgstate(tm_lattice lat, size_t n);
bool is_device_pointer(const void* p);

// Hopping launch description (one parity, nrhs fields).
struct HopArgs {
  int out_parity;
  int prec;
  int nreal;
  int nrhs;
  const void* in;
  size_t in_stride;   // bytes between rhs fields
  void* out;
  size_t out_stride;
  const void* y;      // site-local input (same format as out), or null
  size_t y_stride;
  EpiCoef coef;
  int mode;           // 0 store, 1 store + norm, 2 r -= alpha * out (r = out buffer) + norm
  const CGState* alpha_src;  // mode 2: alpha = alpha_sign * st[sys].alpha (alpha_sign if null)
  double alpha_sign;
  Reduce red;         // modes 1, 2
  const int* skip;    // if non-null and *skip != 0 the kernel does nothing
};
tm_status hop_launch(tm_lattice lat, const HopArgs& a, cudaStream_t s);
tm_status hop_launch_dispatch(tm_lattice lat, const HopArgs& a, cudaStream_t s);  // no gauge-copy check
// blocks of a hopping launch with `tps` threads per site (128-thread blocks)
inline unsigned hop_grid_blocks(size_t h, int tps) { return (unsigned)((h + 128 / tps - 1) / (128 / tps)); }
void invalidate_graphs(tm_lattice lat);

// Field conversions (tm_fields.cu)
tm_status pack_full_parity(tm_lattice lat, int prec, void* dst, const double* src_full, int parity,
                           int g5, cudaStream_t s);
tm_status unpack_full_parity(tm_lattice lat, int prec, double* dst_full, const void* src, int parity,
                             int g5, cudaStream_t s);
tm_status convert_half(tm_lattice lat, int prec_out, void* dst, int prec_in, const void* src,
                       cudaStream_t s);
tm_status apply_M_halves(tm_lattice lat, void* out_e, void* out_o, const void* in_e, const void* in_o, int f,
                         cudaStream_t s);
tm_status diag_apply(tm_lattice lat, int prec, void* out, const void* in, int nrhs, double dur, double dui,
                     double dlr, double dli, cudaStream_t s);
// Workspace slots: 0..17 CG solver, 22..25 tm_apply_D, 26 staged input, 27 staged output,
// 28 initial-guess work space, 29 contraction partials, 30 chronological-guess scalars,
// 31 BiCGstab state; 18..20 BiCGstab vectors; 21 staged correlator matrices.
enum { WS_GAMMA = 21, WS_APPLY_D = 22, WS_STAGE_IN = 26, WS_STAGE_OUT = 27, WS_X0 = 28, WS_CHRONO = 30, WS_BISTATE = 31 };
// host-buffer staging through workspace slots
const void* stage_in(tm_lattice lat, int slot, const void* src, size_t bytes, cudaStream_t s, tm_status* st);
void* stage_out(tm_lattice lat, int slot, void* dst, size_t bytes, tm_status* st);
tm_status stage_out_finish(void* dst, const void* dev, size_t bytes, cudaStream_t s);
}  // namespace tmq
