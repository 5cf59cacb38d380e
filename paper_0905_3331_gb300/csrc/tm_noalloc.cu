// tm_noalloc.cu -- tm_apply_D_noalloc: the full operator M (or M^dag) on canonical FP64
// device fields without any device-memory allocation.
//
// tm_apply_D needs four half-field work buffers (even/odd input, even/odd output) and
// allocates them from the device on first use.  Some callers cannot allow that: code that
// runs under a fixed device-memory budget (a framework whose caching allocator already holds
// the memory, or a process with a hard memory limit), and latency-critical loops where a
// cudaMalloc/cudaFree would synchronise the device.  This entry point takes its work buffers
// from a file-scope static device array instead, sized once when the library's device code
// is loaded and kept by every GPU that loads the library until the process exits.
#include <mutex>

#include "tm_internal.cuh"

namespace tmq {

// Scratch for the four FP64 half fields: 4 x 192 h bytes <= 64 MiB, i.e. h <= 87381,
// V = T L^3 <= 174762 sites (16^3 x 32 fits).
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 128;
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[NOALLOC_MAX_DEVICES];

// Device address of g_noalloc_scratch on the current device.  The symbol's name is only a
// host-side stand-in in host code, so the address is looked up once per device (with that
// device current) and cached.
static tm_status noalloc_scratch(void** out) {
  int dev = -1;
  tm_status st = cuda_check(cudaGetDevice(&dev), "tm_apply_D_noalloc: cudaGetDevice");
  if (st != TM_OK) return st;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return set_error(TM_ERR_ARG, "tm_apply_D_noalloc: device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    st = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "tm_apply_D_noalloc: cudaGetSymbolAddress");
    if (st != TM_OK) return st;
    if (p == nullptr) return set_error(TM_ERR_CUDA, "tm_apply_D_noalloc: null scratch address");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return TM_OK;
}

// True if p is memory that this call may hand to the lattice's kernels without staging:
// device memory of the lattice's device, or managed memory (reachable from every device).
// A pointer into another GPU's memory would be read over the interconnect with peer access,
// and fault without it.
static bool on_lattice_device(const void* p, int lattice_device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == lattice_device;
}

}  // namespace tmq

using namespace tmq;

extern "C" tm_status tm_apply_D_noalloc(tm_lattice lat, double* out, const double* in, int flavour, int dagger,
                                        int nrhs, void* stream) {
  if (!lat || !out || !in || nrhs < 1) return set_error(TM_ERR_ARG, "tm_apply_D_noalloc: bad argument");
  if (flavour != 1 && flavour != -1) return set_error(TM_ERR_ARG, "tm_apply_D_noalloc: flavour must be +1 or -1");
  const size_t hb = tm_half_field_bytes(lat, TM_F64);
  const size_t slot = (hb + 255) / 256 * 256;
  if (4 * slot > NOALLOC_SCRATCH_BYTES)
    return set_error(TM_ERR_ARG,
                     "tm_apply_D_noalloc: a %dx%d^3 lattice needs %zu bytes of scratch; the limit is %zu bytes "
                     "(at most 174762 sites); use tm_apply_D",
                     lat->T, lat->L, 4 * slot, NOALLOC_SCRATCH_BYTES);
  if (!lat->has_gauge) return set_error(TM_ERR_NO_GAUGE, "tm_apply_D_noalloc: no gauge field");
  const size_t fbytes = lat->V * 24 * sizeof(double) * (size_t)nrhs;
  {
    const char* a = reinterpret_cast<const char*>(out);
    const char* b = reinterpret_cast<const char*>(in);
    if (a < b + fbytes && b < a + fbytes) return set_error(TM_ERR_ARG, "tm_apply_D_noalloc: out overlaps in");
  }
  if (!is_device_pointer(in) || !is_device_pointer(out))
    return set_error(TM_ERR_ARG, "tm_apply_D_noalloc: in and out must be device memory (no host staging)");
  int dev = -1;
  tm_status st = cuda_check(cudaGetDevice(&dev), "tm_apply_D_noalloc: cudaGetDevice");
  if (st != TM_OK) return st;
  if (dev != lat->device)
    return set_error(TM_ERR_ARG, "tm_apply_D_noalloc: current device %d is not the lattice's device %d", dev,
                     lat->device);
  if (!on_lattice_device(in, lat->device) || !on_lattice_device(out, lat->device))
    return set_error(TM_ERR_ARG, "tm_apply_D_noalloc: in and out must be device memory of the lattice's device %d",
                     lat->device);
  void* base = nullptr;
  if ((st = noalloc_scratch(&base)) != TM_OK) return st;
  char* sc = static_cast<char*>(base);
  void* w[4] = {sc, sc + slot, sc + 2 * slot, sc + 3 * slot};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // M^dag = g5 M(-f) g5; every scratch byte that is read was written earlier in the same call
  const int f = dagger ? -flavour : flavour;
  const int g5 = dagger ? 1 : 0;
  for (int r = 0; r < nrhs; ++r) {
    const double* src = in + (size_t)r * lat->V * 24;
    double* dst = out + (size_t)r * lat->V * 24;
    if ((st = pack_full_parity(lat, TM_F64, w[0], src, 0, g5, s)) != TM_OK) return st;
    if ((st = pack_full_parity(lat, TM_F64, w[1], src, 1, g5, s)) != TM_OK) return st;
    if ((st = apply_M_halves(lat, w[2], w[3], w[0], w[1], f, s)) != TM_OK) return st;
    if ((st = unpack_full_parity(lat, TM_F64, dst, w[2], 0, g5, s)) != TM_OK) return st;
    if ((st = unpack_full_parity(lat, TM_F64, dst, w[3], 1, g5, s)) != TM_OK) return st;
  }
  return TM_OK;
}
