// tm_operator.cu -- the operator entry points: the hopping matrix H_{p,1-p} between half
// fields (eq. eo2 blocks) and the full operator M of eq. eo0 on canonical fields.
#include "tm_internal.cuh"

namespace tmq {

static bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + nb && y < x + na;
}

// out_p = (1 + i f mut g5) in_p - kappa H_{p,1-p} in_{1-p} for both parities, FP64, one field.
tm_status apply_M_halves(tm_lattice lat, void* out_e, void* out_o, const void* in_e, const void* in_o, int f,
                         cudaStream_t s) {
  const double mut = 2.0 * lat->kappa * lat->mu;
  HopArgs a{};
  a.prec = TM_F64;
  a.nreal = 18;
  a.nrhs = 1;
  a.coef = epi_full_M(lat->kappa, mut, f);
  a.mode = 0;
  a.out_parity = 0;
  a.in = in_o;
  a.y = in_e;
  a.out = out_e;
  tm_status st = hop_launch(lat, a, s);
  if (st != TM_OK) return st;
  a.out_parity = 1;
  a.in = in_e;
  a.y = in_o;
  a.out = out_o;
  return hop_launch(lat, a, s);
}

}  // namespace tmq

using namespace tmq;

extern "C" {

tm_status tm_apply_hopping_eo(tm_lattice lat, int out_parity, void* out, const void* in, tm_prec prec,
                              tm_link link, int nrhs, void* stream) {
  if (!lat || !out || !in || nrhs < 1) return set_error(TM_ERR_ARG, "tm_apply_hopping_eo: bad argument");
  if (out_parity != 0 && out_parity != 1)
    return set_error(TM_ERR_ARG, "tm_apply_hopping_eo: out_parity must be 0 or 1");
  if (prec < TM_F64 || prec > TM_DF64) return set_error(TM_ERR_ARG, "tm_apply_hopping_eo: precision %d", (int)prec);
  if (link != TM_LINK18 && link != TM_LINK12 && link != TM_LINK8)
    return set_error(TM_ERR_ARG, "tm_apply_hopping_eo: link format %d", (int)link);
  const size_t fb = tm_half_field_bytes(lat, prec);
  if (overlap(out, fb * nrhs, in, fb * nrhs)) return set_error(TM_ERR_ARG, "tm_apply_hopping_eo: out overlaps in");
  HopArgs a{};
  a.out_parity = out_parity;
  a.prec = prec;
  a.nreal = (int)link;
  a.nrhs = nrhs;
  a.in = in;
  a.in_stride = fb;
  a.out = out;
  a.out_stride = fb;
  a.coef = epi_plain();
  a.mode = 0;
  return hop_launch(lat, a, static_cast<cudaStream_t>(stream));
}

tm_status tm_apply_D(tm_lattice lat, double* out, const double* in, int flavour, int dagger, int nrhs,
                     void* stream) {
  if (!lat || !out || !in || nrhs < 1) return set_error(TM_ERR_ARG, "tm_apply_D: bad argument");
  if (flavour != 1 && flavour != -1) return set_error(TM_ERR_ARG, "tm_apply_D: flavour must be +1 or -1");
  if (!lat->has_gauge) return set_error(TM_ERR_NO_GAUGE, "tm_apply_D: no gauge field");
  const size_t fbytes = lat->V * 24 * sizeof(double);
  if (overlap(out, fbytes * nrhs, in, fbytes * nrhs)) return set_error(TM_ERR_ARG, "tm_apply_D: out overlaps in");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tm_status st;
  const double* din = static_cast<const double*>(stage_in(lat, WS_STAGE_IN, in, fbytes * nrhs, s, &st));
  if (st != TM_OK) return st;
  double* dout = static_cast<double*>(stage_out(lat, WS_STAGE_OUT, out, fbytes * nrhs, &st));
  if (st != TM_OK) return st;
  const size_t hb = tm_half_field_bytes(lat, TM_F64);
  void* w[4];
  for (int k = 0; k < 4; ++k) {
    w[k] = workspace(lat, WS_APPLY_D + k, hb, &st);
    if (st != TM_OK) return st;
  }
  // M^dag = g5 M(-f) g5
  const int f = dagger ? -flavour : flavour;
  const int g5 = dagger ? 1 : 0;
  for (int r = 0; r < nrhs; ++r) {
    const double* src = din + (size_t)r * lat->V * 24;
    double* dst = dout + (size_t)r * lat->V * 24;
    if ((st = pack_full_parity(lat, TM_F64, w[0], src, 0, g5, s)) != TM_OK) return st;
    if ((st = pack_full_parity(lat, TM_F64, w[1], src, 1, g5, s)) != TM_OK) return st;
    if ((st = apply_M_halves(lat, w[2], w[3], w[0], w[1], f, s)) != TM_OK) return st;
    if ((st = unpack_full_parity(lat, TM_F64, dst, w[2], 0, g5, s)) != TM_OK) return st;
    if ((st = unpack_full_parity(lat, TM_F64, dst, w[3], 1, g5, s)) != TM_OK) return st;
  }
  return stage_out_finish(out, dout, fbytes * nrhs, s);
}

}  // extern "C"
