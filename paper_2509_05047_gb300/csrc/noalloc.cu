// noalloc.cu -- a finalize entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: processes whose device memory is
// reserved up front by another allocator (a serving framework's memory
// pool, a host application that owns the device), code under a strict
// device-memory cap, or real-time reconstruction loops that must not
// allocate (cudaMalloc can synchronise the device and can fail) once they
// are running.  psc_finalize_static gives them the smoothed scatter estimate
// from buffers they already own: every input and the output are the
// caller's device pointers, and the smoothing's working memory is the
// fixed array below, which lives in the library's image on every device
// that loads it, until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>
#include <tuple>
#include <utility>

#include "psc.h"
#include "psc_internal.h"

using namespace psc;

namespace {

// Working memory of psc_finalize_static: the FP32 smoothing buffer (4 bytes
// per sinogram bin) followed by the reciprocal of the normalisation
// sinogram (8 bytes per element).  Shared by every call on a device.
constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" int psc_finalize_static(const int64_t* acc, int32_t n_rings, int32_t n_crystals,
                                   int32_t n_rad, int32_t n_tof, const double* sens,
                                   int32_t sens_per_lor, const double* norm, int32_t norm_per_lor,
                                   const double* sigma, double scale, int32_t sens_first,
                                   double* out, psc_stream stream) {
  if (!acc || !out) return psc_set_error(PSC_EINVAL, "acc and out must be device pointers");
  // the sinogram shapes psc_load_scanner accepts: an even crystal count, the
  // radial bins a centred clip of the n_crystals - 1 (same parity)
  if (n_crystals < 4 || (n_crystals & 1) || n_rings < 1 || n_tof < 1 || n_rad < 1 ||
      n_rad > n_crystals - 1 || ((n_crystals - 1 - n_rad) & 1))
    return psc_set_error(PSC_EINVAL,
                         "bad sinogram dimensions (n_crystals even and >= 4, n_rings and n_tof >= 1, "
                         "n_rad in [1, n_crystals - 1] with n_crystals - 1 - n_rad even)");
  if (!std::isfinite(scale)) return psc_set_error(PSC_EINVAL, "scale must be finite");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return psc_set_error(PSC_EDEVICE, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return psc_set_error(PSC_EINVAL, "device %d not supported", dev);

  FinParams p;
  std::memset(&p, 0, sizeof p);
  p.acc = (const long long*)acc;
  p.out = out;
  p.sens = sens;
  p.sens_per_lor = sens_per_lor ? 1 : 0;
  p.c = std::ldexp(scale, -32);
  p.n_rings = n_rings;
  p.V = n_crystals / 2;
  p.R = n_rad;
  p.T = n_tof;
  p.n_bins = (long long)n_rings * n_rings * p.V * p.R * p.T;
  p.smooth = sigma ? 1 : 0;
  p.sens_first = sens_first ? 1 : 0;
  p.magic_T = p.T == 1 ? 0u : (unsigned)(((1ULL << 32) + p.T - 1) / p.T);
  const long long J = (long long)p.V * p.R * p.T;
  if (J * p.T >= (1LL << 32)) return psc_set_error(PSC_EOVERFLOW, "a sinogram plane is too large");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t s = (cudaStream_t)stream;
  if (!p.smooth) {
    e = launch_finalize(p, sms, s);
    return e == cudaSuccess ? PSC_OK : psc_set_error(PSC_EDEVICE, "finalize: %s", cudaGetErrorString(e));
  }

  // working memory needed: FP32 sinogram + FP64 reciprocal of norm
  const long long n_norm = norm ? (norm_per_lor ? p.n_bins / p.T : p.n_bins) : 0;
  const size_t scr = sizeof(float) * (size_t)p.n_bins;
  const size_t norm_off = (scr + 255) / 256 * 256;
  const size_t need = norm ? norm_off + sizeof(double) * (size_t)n_norm : scr;
  if (need > kStaticScratchBytes)
    return psc_set_error(PSC_EOVERFLOW,
                         "sinogram needs %zu bytes of working memory; the allocation-free entry "
                         "point holds %zu (4 bytes per bin + 8 per normalisation value)",
                         need, kStaticScratchBytes);
  {
    const int rc = finalize_plan(p, sigma);
    if (rc) return rc;
  }

  // set-up, once per device with that device current: the device address
  // of the working array (its name in host code is only a host stand-in).
  // Under lazy module loading (CUDA's default) this lookup is also what
  // loads this file's module and so maps the 64 MiB array on the device.
  // The address is cached per device ordinal for the life of the process:
  // a device reset (cudaDeviceReset) unloads the module and is not
  // supported between calls.
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      e = cudaGetSymbolAddress(&g_scratch_ptr[dev], g_scratch);
      if (e != cudaSuccess) {
        g_scratch_ptr[dev] = nullptr;
        return psc_set_error(PSC_EDEVICE, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      }
    }
    base = g_scratch_ptr[dev];
  }
  p.scratch = (float*)base;
  if (norm) {
    double* rnorm = (double*)((unsigned char*)base + norm_off);
    p.norm = norm;
    p.norm_per_lor = norm_per_lor ? 1 : 0;
    p.rnorm = rnorm;
    e = launch_reciprocal(norm, rnorm, nullptr, n_norm, sms, s);
    if (e != cudaSuccess) return psc_set_error(PSC_EDEVICE, "reciprocal: %s", cudaGetErrorString(e));
  }
  e = launch_finalize(p, sms, s);
  return e == cudaSuccess ? PSC_OK : psc_set_error(PSC_EDEVICE, "finalize: %s", cudaGetErrorString(e));
}
