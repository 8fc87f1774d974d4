// check.cu -- device self-checks of the transport's random numbers: the
// kernel's own Philox4x32-10 (Salmon et al., SC'11) on given counters and
// keys, and cuRAND's Philox4_32_10 generator (called, through its device
// API) on a seed and subsequence, so tests can hold the two against each
// other and against the published known-answer vectors.
#include <curand_kernel.h>

#include <vector>

#include "psc_check.h"
#include "psc_internal.h"

namespace {

__global__ void philox_kernel(const uint32_t* __restrict__ in, long long n, uint32_t* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t* a = in + 6 * i;
  const uint4 r = psc::philox4x32_10(make_uint4(a[0], a[1], a[2], a[3]), make_uint2(a[4], a[5]));
  out[4 * i + 0] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

__global__ void curand_philox_kernel(unsigned long long seed, unsigned long long subsequence, int n_blocks,
                                     uint32_t* __restrict__ out) {
  curandStatePhilox4_32_10_t st;
  curand_init(seed, subsequence, 0, &st);
  for (int b = 0; b < n_blocks; ++b) {
    const uint4 r = curand4(&st);
    out[4 * b + 0] = r.x;
    out[4 * b + 1] = r.y;
    out[4 * b + 2] = r.z;
    out[4 * b + 3] = r.w;
  }
}

// run fn on device copies of in (n_in words) into out (n_out words), synchronously
template <class F>
int on_device(const uint32_t* in, size_t n_in, uint32_t* out, size_t n_out, F fn) {
  uint32_t *d_in = nullptr, *d_out = nullptr;
  cudaError_t e = cudaSuccess;
  if (n_in) e = cudaMalloc(&d_in, n_in * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, n_out * sizeof(uint32_t));
  if (e == cudaSuccess && n_in) e = cudaMemcpy(d_in, in, n_in * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    fn(d_in, d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, n_out * sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (d_in) cudaFree(d_in);
  if (d_out) cudaFree(d_out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return psc::set_error(PSC_EDEVICE, cudaGetErrorString(e));
  }
  return PSC_OK;
}

}  // namespace

extern "C" {

int psc_check_philox(const uint32_t* in, int64_t n, uint32_t* out) {
  if (!in || !out || n < 1 || n > (1 << 24)) return psc::set_error(PSC_EINVAL, "need 1 <= n <= 2^24 and buffers");
  return on_device(in, (size_t)n * 6, out, (size_t)n * 4, [n](const uint32_t* d_in, uint32_t* d_out) {
    philox_kernel<<<(unsigned)((n + 255) / 256), 256>>>(d_in, n, d_out);
  });
}

int psc_check_curand_philox(uint64_t seed, uint64_t subsequence, int32_t n_blocks, uint32_t* out) {
  if (!out || n_blocks < 1 || n_blocks > (1 << 20)) return psc::set_error(PSC_EINVAL, "need 1 <= n_blocks <= 2^20");
  return on_device(nullptr, 0, out, (size_t)n_blocks * 4, [=](const uint32_t*, uint32_t* d_out) {
    curand_philox_kernel<<<1, 1>>>(seed, subsequence, n_blocks, d_out);
  });
}

}  // extern "C"
