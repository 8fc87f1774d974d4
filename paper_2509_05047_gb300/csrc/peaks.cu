// peaks.cu -- measurement kernels for the transport's roofline (not on the
// simulation path): the rate of random int64 atomic adds into a large
// buffer, and the rate of random 4-byte gathers from an L2-sized table.
// The transport kernel's own rates (atomics and gathers per second, from
// its device counters) are reported as fractions of these.
#include "psc_peaks.h"

#include <cuda_runtime.h>

#include "psc_internal.h"

namespace {

// Knuth's MMIX linear congruential generator; the index is taken from the
// high bits (the best-mixed ones) by a 64 x 64 -> high-64 multiply
__device__ __forceinline__ unsigned long long lcg64(unsigned long long x) {
  return x * 6364136223846793005ull + 1442695040888963407ull;
}

__global__ void random_atomics_kernel(unsigned long long* __restrict__ buf, unsigned long long n, int per_thread,
                                      unsigned long long seed) {
  unsigned long long x = lcg64(seed ^ ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B97F4A7C15ull);
  for (int i = 0; i < per_thread; ++i) {
    x = lcg64(x);
    atomicAdd(buf + __umul64hi(x, n), 1ull);
  }
}

__global__ void random_gather_kernel(const float* __restrict__ table, unsigned n, int per_thread,
                                     unsigned long long seed, float* __restrict__ sink) {
  unsigned long long x = lcg64(seed ^ ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B97F4A7C15ull);
  float acc = 0.0f;
  for (int i = 0; i < per_thread; i += 8) {
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // eight independent loads in flight
      x = lcg64(x);
      v[j] = __ldg(table + __umulhi((unsigned)(x >> 32), n));
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) acc += v[j];
  }
  if (acc == -1.0f) sink[0] = acc;  // never true for a table of non-negative values: keeps the loads
}

int launch_ok(cudaError_t e) {
  if (e == cudaSuccess) return PSC_OK;
  cudaGetLastError();
  return psc::set_error(PSC_EDEVICE, cudaGetErrorString(e));
}

}  // namespace

extern "C" {

int psc_peak_random_atomics(int64_t* buf, uint64_t n_slots, int32_t grid, int32_t block, int32_t per_thread,
                            uint64_t seed, psc_stream stream) {
  if (!buf || n_slots == 0 || grid < 1 || block < 32 || block > 1024 || block % 32 || per_thread < 1)
    return psc::set_error(PSC_EINVAL, "bad buffer, size or launch shape");
  random_atomics_kernel<<<grid, block, 0, (cudaStream_t)stream>>>((unsigned long long*)buf, n_slots, per_thread,
                                                                  seed);
  return launch_ok(cudaGetLastError());
}

int psc_peak_random_gather(const float* table, uint32_t n, int32_t grid, int32_t block, int32_t per_thread,
                           uint64_t seed, float* sink, psc_stream stream) {
  if (!table || !sink || n == 0 || grid < 1 || block < 32 || block > 1024 || block % 32 || per_thread < 8 ||
      per_thread % 8)
    return psc::set_error(PSC_EINVAL, "bad table, sink, size or launch shape");
  random_gather_kernel<<<grid, block, 0, (cudaStream_t)stream>>>(table, n, per_thread, seed, sink);
  return launch_ok(cudaGetLastError());
}

}  // extern "C"
