// tm_lattice.cu -- lattice object, error reporting, device buffers, gauge field
// validation and the parity-split gauge copy (Sec. 4.1: links stored again in the
// order the operator reads them; here per output parity: 4 forward links U_mu(x)
// and 4 backward links U_mu(x - mu^)^dag per site, in FP64/FP32/FP16 and with
// 18, 12 or 8 stored reals).
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "tm_dslash.cuh"
#include "tm_internal.cuh"

namespace tmq {

static thread_local char g_err[1024] = "";
static std::atomic<unsigned long long> g_launches{0};

void count_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

tm_status set_error(tm_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

tm_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TM_OK;
  if (e == cudaErrorMemoryAllocation)
    return set_error(TM_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return set_error(TM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------- epilogue coefficients ---
EpiCoef epi_finish(EpiCoef e) {
  e.f_dcu_re = (float)(e.d_up_re * e.c);
  e.f_dcu_im = (float)(e.d_up_im * e.c);
  e.f_dcl_re = (float)(e.d_lo_re * e.c);
  e.f_dcl_im = (float)(e.d_lo_im * e.c);
  e.f_deu_re = (float)(e.d_up_re * e.e_up_re - e.d_up_im * e.e_up_im);
  e.f_deu_im = (float)(e.d_up_re * e.e_up_im + e.d_up_im * e.e_up_re);
  e.f_del_re = (float)(e.d_lo_re * e.e_lo_re - e.d_lo_im * e.e_lo_im);
  e.f_del_im = (float)(e.d_lo_re * e.e_lo_im + e.d_lo_im * e.e_lo_re);
  return e;
}
EpiCoef epi_plain() {
  EpiCoef e{};
  e.c = 1.0;
  e.d_up_re = e.d_lo_re = 1.0;
  return epi_finish(e);
}
EpiCoef epi_mdiag_inv_hop(double mut, int f) {  // (1 - i f mut g5) / (1 + mut^2) H
  EpiCoef e{};
  const double n = 1.0 / (1.0 + mut * mut);
  e.c = 1.0;
  e.d_up_re = n;
  e.d_up_im = -f * mut * n;
  e.d_lo_re = n;
  e.d_lo_im = f * mut * n;
  return epi_finish(e);
}
EpiCoef epi_scaled_minv(double mut, int f, double c) {  // (M_ee^f)^-1 (c H + y)
  EpiCoef e = epi_mdiag_inv_hop(mut, f);
  e.c = c;
  e.e_up_re = e.e_lo_re = 1.0;
  e.m_up_re = e.m_lo_re = 1.0;  // M_ee^f = 1 + i f mut gamma5
  e.m_up_im = f * mut;
  e.m_lo_im = -f * mut;
  return epi_finish(e);
}
EpiCoef epi_full_M(double kappa, double mut, int f) {  // (1 + i f mut g5) y - kappa H
  EpiCoef e{};
  e.c = -kappa;
  e.d_up_re = e.d_lo_re = 1.0;
  e.e_up_re = 1.0;
  e.e_up_im = f * mut;
  e.e_lo_re = 1.0;
  e.e_lo_im = -f * mut;
  return epi_finish(e);
}
EpiCoef epi_schur_q(double kappa, double mut, int f) {  // g5 [(1 + i f mut g5) y - kappa^2 H]
  EpiCoef e = epi_full_M(kappa * kappa, mut, f);
  e.c = -kappa * kappa;
  e.d_up_re = 1.0;
  e.d_lo_re = -1.0;
  return epi_finish(e);
}
EpiCoef epi_g5_y_plus(double c) {  // g5 (y + c H)
  EpiCoef e{};
  e.c = c;
  e.d_up_re = 1.0;
  e.d_lo_re = -1.0;
  e.e_up_re = e.e_lo_re = 1.0;
  return epi_finish(e);
}

// ------------------------------------------------------------------ buffers ---
void* workspace(tm_lattice lat, int slot, size_t bytes, tm_status* st) {
  *st = TM_OK;
  if (slot < 0 || slot >= 32) {
    *st = set_error(TM_ERR_ARG, "internal: workspace slot %d", slot);
    return nullptr;
  }
  if (lat->ws_bytes[slot] >= bytes && lat->ws[slot] != nullptr) return lat->ws[slot];
  if (lat->ws[slot]) cudaFree(lat->ws[slot]);
  lat->ws[slot] = nullptr;
  lat->ws_bytes[slot] = 0;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    *st = cuda_check(e, "workspace allocation");
    return nullptr;
  }
  lat->ws[slot] = p;
  lat->ws_bytes[slot] = bytes;
  return p;
}

tm_status ensure_reduce(tm_lattice lat, size_t nparts, size_t ncounters) {
  if (!lat->gcounters) {  // once per lattice, before any graph capture uses it
    const size_t n = lat->h / 1024 + 16;
    tm_status st = cuda_check(cudaMalloc(&lat->gcounters, n * sizeof(unsigned)), "reduction group counters");
    if (st == TM_OK) st = cuda_check(cudaMemset(lat->gcounters, 0, n * sizeof(unsigned)), "reduction group counters");
    if (st != TM_OK) return st;
  }
  if (nparts > lat->partials_count) {
    if (lat->partials) cudaFree(lat->partials);
    lat->partials = nullptr;
    lat->partials_count = 0;
    tm_status st = cuda_check(cudaMalloc(&lat->partials, nparts * sizeof(double)), "reduction buffer");
    if (st != TM_OK) return st;
    lat->partials_count = nparts;
  }
  if (ncounters > lat->counters_count) {
    if (lat->counters) cudaFree(lat->counters);
    lat->counters = nullptr;
    lat->counters_count = 0;
    tm_status st = cuda_check(cudaMalloc(&lat->counters, ncounters * sizeof(unsigned)), "reduction counters");
    if (st != TM_OK) return st;
    st = cuda_check(cudaMemset(lat->counters, 0, ncounters * sizeof(unsigned)), "reduction counters");
    if (st != TM_OK) return st;
    lat->counters_count = ncounters;
  }
  return TM_OK;
}

tm_status ensure_cgstate(tm_lattice lat, size_t n) {
  if (n <= lat->cgstate_count) return TM_OK;
  if (lat->cgstate) cudaFree(lat->cgstate);
  if (lat->cgstate_host) cudaFreeHost(lat->cgstate_host);
  lat->cgstate = nullptr;
  lat->cgstate_host = nullptr;
  lat->cgstate_count = 0;
  tm_status st = cuda_check(cudaMalloc(&lat->cgstate, n * sizeof(CGState)), "CG state");
  if (st != TM_OK) return st;
  st = cuda_check(cudaMallocHost(&lat->cgstate_host, n * sizeof(CGState)), "CG state (host)");
  if (st != TM_OK) return st;
  lat->cgstate_count = n;
  return TM_OK;
}

// --------------------------------------------------------- gauge validation ---
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// dev[0] = max |U^dag U - 1|, dev[1] = max |det U - 1|, dev[2] = number of non-finite entries
__global__ void check_su3_kernel(const double* __restrict__ U, size_t nlinks, unsigned long long* dev) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nlinks) return;
  Mat3<double> m;
  bool finite = true;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double re = U[18 * i + 6 * a + 2 * b], im = U[18 * i + 6 * a + 2 * b + 1];
      finite = finite && isfinite(re) && isfinite(im);
      m.m[a][b] = mk(re, im);
    }
  if (!finite) {
    atomicAdd(dev + 2, 1ull);
    return;
  }
  double du = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cpx<double> s = mk(0.0, 0.0);
      for (int k = 0; k < 3; ++k) s = s + cjmul(m.m[k][a], m.m[k][b]);
      s.re -= (a == b) ? 1.0 : 0.0;
      du = fmax(du, fmax(fabs(s.re), fabs(s.im)));
    }
  cpx<double> det = m.m[0][0] * (m.m[1][1] * m.m[2][2] - m.m[1][2] * m.m[2][1]) -
                    m.m[0][1] * (m.m[1][0] * m.m[2][2] - m.m[1][2] * m.m[2][0]) +
                    m.m[0][2] * (m.m[1][0] * m.m[2][1] - m.m[1][1] * m.m[2][0]);
  det.re -= 1.0;
  atomic_max_nonneg(dev + 0, du);
  atomic_max_nonneg(dev + 1, sqrt(norm2(det)));
}

// ------------------------------------------------------------ gauge copies ---
// The 8-real form in half precision.  Its reconstruction obtains |c0| = sqrt(N - |b0|^2) and divides
// by N = |a1|^2 + |a2|^2, which amplifies the rounding of the stored halves on some links: rounding
// each of the 8 reals to nearest leaves a largest entry error of the reconstructed matrix up to
// ~3e-2 (mean 4e-4 on an eps = 0.6 field), against 6e-4 (mean 2e-4) for the 12-real form.  The
// halves are therefore chosen by a local search instead: from the rounded values, each of the 8 is
// moved by 4, 2 and 1 units in the last place up or down while that lowers the largest entry
// error |U_rec - U| of the matrix the hopping kernel reconstructs from them (its own FP32
// arithmetic), in two passes (96 reconstructions per link, once per gauge field).  On the eps = 0.6
// field this gives mean 1.9e-4 and 99th percentile 4.7e-4 (1 - 3e-2 remain on 6 of 98304 links,
// where |c0|^2 ~ 1e-5 << N).
__device__ __forceinline__ unsigned short half_ulp_step(unsigned short b, bool up) {
  const bool neg = (b & 0x8000u) != 0;
  if (up) {
    if (!neg) return b < 0x7bffu ? (unsigned short)(b + 1) : b;
    return b == 0x8000u ? (unsigned short)0x0001u : (unsigned short)(b - 1);
  }
  if (neg) return b < 0xfbffu ? (unsigned short)(b + 1) : b;
  return b == 0x0000u ? (unsigned short)0x8001u : (unsigned short)(b - 1);
}

__device__ __forceinline__ double recon8_half_error(const RawWords<16>& r, const Mat3<double>& F) {
  Mat3<float> R;
  LinkRecon<float, __half, 8>::unpack(r, R);
  double e = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      e = fmax(e, fmax(fabs((double)R.m[a][b].re - F.m[a][b].re), fabs((double)R.m[a][b].im - F.m[a][b].im)));
  return e;
}

__device__ void refine_half8(RawWords<16>& r, const Mat3<double>& F) {
  double best = recon8_half_error(r, F);
  for (int pass = 0; pass < 2; ++pass)
    for (int n = 4; n >= 1; n >>= 1)
      for (int k = 0; k < 8; ++k)
        for (int d = 0; d < 2; ++d) {
          RawWords<16> q = r;
          const int sh = 16 * (k & 1);
          unsigned short b = (unsigned short)((q.w[k >> 1] >> sh) & 0xffffu);
          for (int j = 0; j < n; ++j) b = half_ulp_step(b, d == 0);
          q.w[k >> 1] = (q.w[k >> 1] & ~(0xffffu << sh)) | ((unsigned int)b << sh);
          const double e = recon8_half_error(q, F);
          if (e < best) {
            best = e;
            r = q;
          }
        }
}

// Per parity p and site cb of that parity, slab mu holds U_mu(x) compressed to NREAL reals of
// type S.  The hopping kernel reads the forward link of an output site from its own parity's
// slab and the backward link U_mu(x - mu^) from the other parity's slab at the neighbour.
template <typename S, int NREAL>
__global__ void build_links_kernel(Geom g, const double* __restrict__ U, char* __restrict__ out) {
  const int p = blockIdx.y;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= g.h) return;
  constexpr int BYTES = NREAL * (int)sizeof(S);
  const SiteCoord c = site_of(g, cb, p);
  const size_t lex = (((size_t)c.t * g.L + c.z) * g.L + c.y) * g.L + c.x;
  const size_t slab = (size_t)BYTES * g.h;
  for (int mu = 0; mu < 4; ++mu) {
    Mat3<double> F;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const double* uf = U + 72 * lex + 18 * mu + 6 * a + 2 * b;
        F.m[a][b] = mk(uf[0], uf[1]);
      }
    RawWords<BYTES> rf;
    LinkRecon<double, S, NREAL>::pack(rf, F);
    if constexpr (NREAL == 8 && sizeof(S) == 2) refine_half8(rf, F);
    store_raw<BYTES>(out + (size_t)(p * 4 + mu) * slab, g.h, cb, rf);
  }
}

static tm_status tune_hop(tm_lattice lat, int prec, int nreal, cudaStream_t s, bool retime = false);

template <typename S, int NREAL>
static void launch_build(tm_lattice lat, char* out, cudaStream_t s) {
  dim3 grid((lat->geom.h + 127) / 128, 2);
  build_links_kernel<S, NREAL><<<grid, 128, 0, s>>>(lat->geom, lat->U_canon, out);
  count_launch();
}

tm_status ensure_links(tm_lattice lat, int prec, int nreal, cudaStream_t s) {
  if (!lat->has_gauge) return set_error(TM_ERR_NO_GAUGE, "no gauge field: call tm_set_gauge first");
  if (prec < 0 || prec > 3) return set_error(TM_ERR_ARG, "precision %d not one of TM_F64/F32/F16/DF64", prec);
  if (nreal != 18 && nreal != 12 && nreal != 8)
    return set_error(TM_ERR_ARG, "link format %d not one of 18, 12, 8", nreal);
  if (prec == TM_DF64 && nreal != 18)
    return set_error(TM_ERR_UNSUPPORTED, "double-float storage supports 18-real links only");
  void*& slot = lat->links[prec][link_index(nreal)];
  if (slot) return TM_OK;
  const size_t bytes = 8 * link_bytes(prec, nreal) * lat->h;  // 2 parities x 4 directions
  tm_status st = cuda_check(cudaMalloc(&slot, bytes), "gauge copy allocation");
  if (st != TM_OK) {
    slot = nullptr;
    return st;
  }
  char* out = static_cast<char*>(slot);
  if (prec == TM_F64) {
    if (nreal == 18) launch_build<double, 18>(lat, out, s);
    if (nreal == 12) launch_build<double, 12>(lat, out, s);
    if (nreal == 8) launch_build<double, 8>(lat, out, s);
  } else if (prec == TM_F32) {
    if (nreal == 18) launch_build<float, 18>(lat, out, s);
    if (nreal == 12) launch_build<float, 12>(lat, out, s);
    if (nreal == 8) launch_build<float, 8>(lat, out, s);
  } else if (prec == TM_DF64) {
    launch_build<dd, 18>(lat, out, s);
  } else {
    if (nreal == 18) launch_build<__half, 18>(lat, out, s);
    if (nreal == 12) launch_build<__half, 12>(lat, out, s);
    if (nreal == 8) launch_build<__half, 8>(lat, out, s);
  }
  if ((st = cuda_check(cudaGetLastError(), "gauge copy build")) != TM_OK) return st;
  return tune_hop(lat, prec, nreal, s);
}

// ---------------------------------------------------------------- autotuner ---
// Picks the hopping kernel for one storage form of this lattice -- 1, 2 or 4 threads per site,
// or one thread per site with software-pipelined loads (TM_HOP_PIPELINED) -- by timing each
// choice (CUDA events, fastest of several timed groups, candidates interleaved) on scratch
// buffers.  TM_HOP_TPS=1|2|3|4 in the environment fixes the choice for every form (3: the
// pipelined kernel, FP64 falls back to 1); tm_set_hop_threads fixes it for one form.  Runs
// when the form's gauge copy is built.  A choice is kept for the rest of the process by device,
// extents and storage form (it depends on the launch shape, not on the field's values): a later
// lattice of the same shape takes it without timing again, and tm_set_hop_threads(..., 0) times
// again and replaces it.
static int env_tps() {
  const char* e = getenv("TM_HOP_TPS");
  if (!e) return 0;
  const int v = atoi(e);
  return (v == 1 || v == 2 || v == 4 || v == TM_HOP_PIPELINED || v == TM_HOP_PAIRED) ? v : 0;
}

// The choices made so far in this process.
struct TuneChoice {
  int device, T, L, prec, nreal, tps;
};
static std::mutex g_tune_mu;
static std::vector<TuneChoice> g_tune_choices;

// Times the kernel choices of one storage form on this lattice and keeps the best.  The score
// is one CG iteration's mix: two plain launches (K1, K3) and two launches with a site-local
// input, the residual update and the fused reduction (K2, K4).  More threads per site must
// win by 10%: measured at 16^3 x 32, FP32 kernels with 2 threads per site ran at their
// stand-alone speed in a host loop but 2.3x slower inside the CG stage graphs.  (They need
// 116-144 registers a thread, so only 3-4 of their 128-thread blocks fit on an SM.)
static tm_status tune_hop(tm_lattice lat, int prec, int nreal, cudaStream_t s, bool retime) {
  const int li = link_index(nreal);
  if (lat->hop_tps_forced[prec][li]) return TM_OK;
  if (prec == TM_DF64) {  // built with one thread per site only
    lat->hop_tps[prec][li] = 1;
    return TM_OK;
  }
  if (const int e = env_tps()) {
    lat->hop_tps[prec][li] = ((e == TM_HOP_PIPELINED || e == TM_HOP_PAIRED) && prec == TM_F64) ? 1 : e;
    return TM_OK;
  }
  if (!retime) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const TuneChoice& c : g_tune_choices)
      if (c.device == lat->device && c.T == lat->T && c.L == lat->L && c.prec == prec && c.nreal == nreal) {
        lat->hop_tps[prec][li] = c.tps;
        return TM_OK;
      }
  }
  const size_t hb = spinor_bytes_per_site(prec) * lat->h;
  const int pr = (prec == TM_F64) ? TM_F64 : TM_F32;
  const size_t rb = spinor_bytes_per_site(pr) * lat->h;
  void *din = nullptr, *dout = nullptr, *dy = nullptr, *dr = nullptr;
  tm_status st = cuda_check(cudaMalloc(&din, hb), "tuner buffer");
  if (st == TM_OK) st = cuda_check(cudaMalloc(&dout, hb), "tuner buffer");
  if (st == TM_OK) st = cuda_check(cudaMalloc(&dy, hb), "tuner buffer");
  if (st == TM_OK) st = cuda_check(cudaMalloc(&dr, rb), "tuner buffer");
  if (st == TM_OK) st = cuda_check(cudaMemsetAsync(din, 0, hb, s), "tuner buffer");
  if (st == TM_OK) st = cuda_check(cudaMemsetAsync(dy, 0, hb, s), "tuner buffer");
  if (st == TM_OK) st = cuda_check(cudaMemsetAsync(dr, 0, rb, s), "tuner buffer");
  if (st == TM_OK) st = ensure_reduce(lat, hop_grid_blocks(lat->h, 4), 4);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == TM_OK) st = cuda_check(cudaEventCreate(&e0), "event");
  if (st == TM_OK) st = cuda_check(cudaEventCreate(&e1), "event");
  HopArgs plain{};
  plain.prec = prec;
  plain.nreal = nreal;
  plain.nrhs = 1;
  plain.in = din;
  plain.out = dout;
  plain.coef = epi_plain();
  HopArgs upd = plain;  // r -= 1 * (y + H in), sum ||r||^2
  upd.y = dy;
  upd.out = dr;
  upd.coef = epi_g5_y_plus(1.0);
  upd.mode = 2;
  upd.alpha_sign = 1.0;
  upd.red = Reduce{lat->partials, lat->counters, lat->dscalars, nullptr, FIN_STORE};
  // Passes interleave the candidates so that a clock still ramping up after the gauge copy
  // was built (or any other drift) slows every candidate alike; pass 0 is the warm-up.  A
  // group is two iterations' mix (8 launches); each candidate's score is its fastest group
  // (five groups, three for FP64 storage, whose launches are ~10x longer).  Candidates: one
  // thread per site, its software-pipelined form (FP32 / FP16 storage), 2 and 4 threads per site,
  // and two sites per thread with packed FP32 pairs (FP32 / FP16 storage).
  const int cands[5] = {1, TM_HOP_PIPELINED, 2, 4, TM_HOP_PAIRED};
  const bool has_pipe = (prec == TM_F32 || prec == TM_F16);
  const int rounds = (prec == TM_F64) ? 4 : 6;
  float score[5] = {1e30f, 1e30f, 1e30f, 1e30f, 1e30f};
  for (int k = 0; k < rounds && st == TM_OK; ++k) {
    for (int c = 0; c < 5 && st == TM_OK; ++c) {
      if ((c == 1 || c == 4) && !has_pipe) continue;
      lat->hop_tps[prec][li] = cands[c];
      st = cuda_check(cudaEventRecord(e0, s), "event");
      for (int q = 0; q < 8 && st == TM_OK; ++q) {
        HopArgs a = (q & 1) ? upd : plain;
        a.out_parity = (q >> 1) & 1;
        st = hop_launch_dispatch(lat, a, s);
      }
      if (st == TM_OK) st = cuda_check(cudaEventRecord(e1, s), "event");
      if (st == TM_OK) st = cuda_check(cudaEventSynchronize(e1), "tuner");
      float ms = 0.f;
      if (st == TM_OK) st = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "event");
      if (k > 0 && ms < score[c]) score[c] = ms;
    }
  }
  // Plain or pipelined: a difference above 3% decides; within 3% (the scores' repeat-to-repeat
  // spread) the rule does, so that the choice is reproducible: the pipelined kernel where the
  // plain one's grid fits in one wave (each thread's load latencies set the launch time there:
  // 16^3 x 32 FP32/12 1.9% faster inside the mixed solve, 13% per cold launch), else the plain
  // one.  The paired kernel must beat the better of the two by 3%; more threads per site must
  // be 10% faster than the best so far.
  int bi = 0;
  if (has_pipe) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    const bool one_wave = lat->h <= (size_t)sms * HOP_BLOCKS_12 * hop_spb(1);
    const float ratio = score[1] / score[0];
    bi = ratio < 0.97f ? 1 : (ratio > 1.03f ? 0 : (one_wave ? 1 : 0));
    if (score[4] < 0.97f * score[bi]) bi = 4;
  }
  const float base = score[bi];
  for (int c = 2; c < 4; ++c)
    if (score[c] < 0.9f * base && score[c] < score[bi]) bi = c;
  lat->hop_tps[prec][li] = cands[bi];
  if (st == TM_OK) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    bool found = false;
    for (TuneChoice& c : g_tune_choices)
      if (c.device == lat->device && c.T == lat->T && c.L == lat->L && c.prec == prec && c.nreal == nreal) {
        c.tps = cands[bi];
        found = true;
      }
    if (!found) g_tune_choices.push_back(TuneChoice{lat->device, lat->T, lat->L, prec, nreal, cands[bi]});
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(din);
  cudaFree(dout);
  cudaFree(dy);
  cudaFree(dr);
  return st;
}

// Off by default: measured on the 16^3 x 32 mixed solve, programmatic dependent launch of the
// iteration kernels made the solve slower (123 vs 140 solves/s); TM_PDL=1 turns it on.
bool use_pdl() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("TM_PDL");
    v = (e && *e == '1') ? 1 : 0;
  }
  return v == 1;
}

void invalidate_graphs(tm_lattice lat) {
  for (int k = 0; k < 8; ++k) {
    if (lat->graphs[k].valid) {
      cudaGraphExecDestroy(lat->graphs[k].exec);
      cudaGraphDestroy(lat->graphs[k].graph);
      lat->graphs[k].valid = false;
    }
    if (lat->aux_graphs[k].valid) {
      cudaGraphExecDestroy(lat->aux_graphs[k].exec);
      cudaGraphDestroy(lat->aux_graphs[k].graph);
      lat->aux_graphs[k].valid = false;
    }
  }
}

tm_status hop_launch(tm_lattice lat, const HopArgs& a, cudaStream_t s) {
  tm_status st = ensure_links(lat, a.prec, a.nreal, s);
  if (st != TM_OK) return st;
  return hop_launch_dispatch(lat, a, s);
}

tm_status hop_launch_dispatch(tm_lattice lat, const HopArgs& a, cudaStream_t s) {
  switch (a.prec) {
    case TM_F64:
      return hop_launch_f64(lat, a, s);
    case TM_F32:
      return hop_launch_f32(lat, a, s);
    case TM_F16:
      return hop_launch_f16(lat, a, s);
    case TM_DF64:
      return hop_launch_df64(lat, a, s);
    default:
      return set_error(TM_ERR_ARG, "precision %d", a.prec);
  }
}

}  // namespace tmq

using namespace tmq;

// ================================================================== C ABI ===
extern "C" {

const char* tm_last_error(void) { return tmq::g_err; }

unsigned long long tm_launch_count(void) { return tmq::g_launches.load(); }
void tm_reset_launch_count(void) { tmq::g_launches.store(0); }

tm_status tm_lattice_create(int T, int L, double kappa, double mu, tm_lattice* out) {
  tmq::g_err[0] = 0;
  if (!out) return set_error(TM_ERR_ARG, "tm_lattice_create: out is NULL");
  *out = nullptr;
  if (T < 2 || L < 2 || (T & 1) || (L & 1))
    return set_error(TM_ERR_ODD_EXTENT, "tm_lattice_create: T=%d, L=%d must be even and >= 2", T, L);
  if (!std::isfinite(kappa) || !std::isfinite(mu))
    return set_error(TM_ERR_ARG, "tm_lattice_create: kappa and mu must be finite");
  const double Vd = (double)T * L * L * L;
  if (Vd / 2 > 2.0e9) return set_error(TM_ERR_ARG, "tm_lattice_create: lattice too large");
  tm_lattice lat = static_cast<tm_lattice>(calloc(1, sizeof(tm_lattice_s)));
  if (!lat) return set_error(TM_ERR_OOM, "tm_lattice_create: host allocation");
  lat->T = T;
  lat->L = L;
  lat->kappa = kappa;
  lat->mu = mu;
  lat->V = (size_t)T * L * L * L;
  lat->h = lat->V / 2;
  lat->geom.T = T;
  lat->geom.L = L;
  lat->geom.Lh = L / 2;
  lat->geom.h = (int)lat->h;
  lat->geom.sy = L / 2;
  lat->geom.sz = L * (L / 2);
  lat->geom.st = L * L * (L / 2);
  tm_status st = cuda_check(cudaGetDevice(&lat->device), "cudaGetDevice");
  if (st == TM_OK) st = cuda_check(cudaMalloc(&lat->dscalars, 64 * sizeof(double)), "scalar scratch");
  if (st == TM_OK) st = cuda_check(cudaMallocHost(&lat->flag_host, 64 * sizeof(int)), "host flag");
  // reduction buffers sized once for every kernel of the library (a hopping launch uses at
  // most ceil(h / 32) blocks, the vector kernels at most 152 * 16), so nothing is reallocated
  // while kernels that use them may be in flight
  if (st == TM_OK) st = ensure_reduce(lat, hop_grid_blocks(lat->h, 4) + 152 * 16, 64);
  if (st == TM_OK) st = ensure_cgstate(lat, 2);
  if (st != TM_OK) {
    tm_lattice_destroy(lat);
    return st;
  }
  *out = lat;
  return TM_OK;
}

tm_status tm_lattice_destroy(tm_lattice lat) {
  if (!lat) return TM_OK;
  cudaDeviceSynchronize();
  cudaFree(lat->U_canon);
  for (int p = 0; p < 4; ++p)
    for (int l = 0; l < 3; ++l) cudaFree(lat->links[p][l]);
  for (int k = 0; k < 32; ++k) cudaFree(lat->ws[k]);
  cudaFree(lat->partials);
  cudaFree(lat->counters);
  cudaFree(lat->gcounters);
  cudaFree(lat->dscalars);
  cudaFree(lat->cgstate);
  cudaFree(lat->stage);
  if (lat->cgstate_host) cudaFreeHost(lat->cgstate_host);
  if (lat->flag_host) cudaFreeHost(lat->flag_host);
  invalidate_graphs(lat);
  free(lat);
  return TM_OK;
}

tm_status tm_lattice_set_params(tm_lattice lat, double kappa, double mu) {
  if (!lat) return set_error(TM_ERR_ARG, "tm_lattice_set_params: lattice is NULL");
  if (!std::isfinite(kappa) || !std::isfinite(mu))
    return set_error(TM_ERR_ARG, "tm_lattice_set_params: kappa and mu must be finite");
  lat->kappa = kappa;
  lat->mu = mu;
  return TM_OK;
}

size_t tm_volume(tm_lattice lat) { return lat ? lat->V : 0; }

tm_status tm_set_hop_threads(tm_lattice lat, tm_prec prec, tm_link link, int threads_per_site) {
  if (!lat || prec < TM_F64 || prec > TM_DF64 || (link != 18 && link != 12 && link != 8))
    return set_error(TM_ERR_ARG, "tm_set_hop_threads: bad argument");
  if (threads_per_site != 0 && threads_per_site != 1 && threads_per_site != 2 && threads_per_site != 4 &&
      threads_per_site != TM_HOP_PIPELINED && threads_per_site != TM_HOP_PAIRED)
    return set_error(TM_ERR_ARG,
                     "tm_set_hop_threads: threads_per_site must be 0 (tune), 1, 2, 4, 3 (pipelined) or 5 (paired)");
  if ((threads_per_site == TM_HOP_PIPELINED || threads_per_site == TM_HOP_PAIRED) && prec != TM_F32 &&
      prec != TM_F16)
    return set_error(TM_ERR_UNSUPPORTED,
                     "tm_set_hop_threads: the pipelined and paired kernels exist for FP32 and FP16 storage");
  const int li = link_index(link);
  invalidate_graphs(lat);  // captured graphs hold the previous kernel choice
  if (threads_per_site == 0) {
    lat->hop_tps_forced[prec][li] = 0;
    if (lat->links[prec][li]) return tune_hop(lat, prec, link, nullptr, true);
    return TM_OK;
  }
  if (prec == TM_DF64 && threads_per_site != 1)
    return set_error(TM_ERR_UNSUPPORTED, "tm_set_hop_threads: double-float runs with one thread per site");
  lat->hop_tps_forced[prec][li] = 1;
  lat->hop_tps[prec][li] = threads_per_site;
  return TM_OK;
}

int tm_get_hop_threads(tm_lattice lat, tm_prec prec, tm_link link) {
  if (!lat || prec < TM_F64 || prec > TM_DF64 || (link != 18 && link != 12 && link != 8)) return 0;
  const int v = lat->hop_tps[prec][link_index(link)];
  return v == 0 ? 1 : v;
}

size_t tm_half_field_bytes(tm_lattice lat, tm_prec prec) {
  if (!lat || prec < 0 || prec > 3) return 0;
  return spinor_bytes_per_site(prec) * lat->h;
}

tm_status tm_set_gauge(tm_lattice lat, const double* U, void* stream) {
  tmq::g_err[0] = 0;
  if (!lat || !U) return set_error(TM_ERR_ARG, "tm_set_gauge: NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n = 72 * lat->V;
  double* tmp = nullptr;
  tm_status st = cuda_check(cudaMalloc(&tmp, n * sizeof(double)), "tm_set_gauge: allocation");
  if (st != TM_OK) return st;
  st = cuda_check(cudaMemcpyAsync(tmp, U, n * sizeof(double), cudaMemcpyDefault, s), "tm_set_gauge: copy");
  unsigned long long* dev = reinterpret_cast<unsigned long long*>(lat->dscalars);
  if (st == TM_OK) st = cuda_check(cudaMemsetAsync(dev, 0, 3 * sizeof(unsigned long long), s), "memset");
  if (st == TM_OK) {
    const size_t nl = 4 * lat->V;
    check_su3_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, s>>>(tmp, nl, dev);
    count_launch();
    st = cuda_check(cudaGetLastError(), "tm_set_gauge: check kernel");
  }
  unsigned long long hv[3] = {0, 0, 0};
  if (st == TM_OK) st = cuda_check(cudaMemcpyAsync(hv, dev, sizeof(hv), cudaMemcpyDeviceToHost, s), "readback");
  if (st == TM_OK) st = cuda_check(cudaStreamSynchronize(s), "tm_set_gauge: synchronise");
  if (st != TM_OK) {
    cudaFree(tmp);
    return st;
  }
  double du, dd;
  memcpy(&du, &hv[0], sizeof(double));
  memcpy(&dd, &hv[1], sizeof(double));
  if (hv[2] != 0) {
    cudaFree(tmp);
    return set_error(TM_ERR_NONFINITE, "tm_set_gauge: %llu links have non-finite entries", hv[2]);
  }
  if (du > 1e-10 || dd > 1e-10) {
    cudaFree(tmp);
    return set_error(TM_ERR_NOT_SU3, "tm_set_gauge: max |U^dag U - 1| = %.3e, max |det U - 1| = %.3e", du, dd);
  }
  // accept: replace the canonical copy and drop every derived copy
  cudaFree(lat->U_canon);
  lat->U_canon = tmp;
  for (int p = 0; p < 4; ++p)
    for (int l = 0; l < 3; ++l) {
      cudaFree(lat->links[p][l]);
      lat->links[p][l] = nullptr;
    }
  lat->has_gauge = true;
  st = ensure_links(lat, TM_F64, 18, s);
  if (st != TM_OK) return st;
  return cuda_check(cudaStreamSynchronize(s), "tm_set_gauge: build");
}

}  // extern "C"
