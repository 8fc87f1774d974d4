// finalize.cu -- scatter estimate from the int64 fixed-point accumulator
// (Sec. 2.2.4: multiply by the scatter-sensitivity sinogram; Sec. 2.3.2:
// multiply by the smoothing-normalisation sinogram, Gaussian-smooth, divide
// by it again).
//
// Without smoothing one FP64 elementwise pass: out = ((double)acc * c) * s,
// c = scale * 2^-32.
//
// With smoothing three passes, each reading and writing every bin once
// through a shared-memory tile that holds whole lines of the smoothed axis
// (so no halo is re-read):
//   A  radial: acc (int64) -> FP32 tile per (plane, view) line -> scratch
//   B  view:   scratch in place, tile (all views) x (inner chunk)
//   C  axial:  scratch -> tile (planes of one ring-difference segment) x
//              (inner chunk) -> FP64 epilogue (x 1/norm, x sens) -> out
// The smoothing arithmetic is FP32 (the FP64 part of the path is the final
// normalisation / sensitivity multiply).  Kernels are truncated at
// ceil(4 sigma) with weights normalised to 1; edges reflect half-sample
// symmetrically; the axial neighbours of a plane are the planes of the same
// ring difference.
#include "psc_internal.h"

namespace psc {

__device__ __forceinline__ int reflect(int m, int n) {
  const int p = 2 * n;
  m %= p;
  if (m < 0) m += p;
  return m >= n ? p - 1 - m : m;
}

__device__ __forceinline__ double lor_or_bin(const double* a, int per_lor, long long bin, int n_tof) {
  return per_lor ? __ldg(a + bin / n_tof) : __ldg(a + bin);
}

// ---------------------------------------------------------------------------
// no smoothing: out = (acc * c) * sens  (FP64, same operation order as the
// definition so the product is exact to the last bit)
// ---------------------------------------------------------------------------
__global__ void finalize_plain_kernel(const __grid_constant__ FinParams P) {
  const long long n = P.n_bins;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double x = (double)__ldg(P.acc + i) * P.c;
    if (P.sens) x = x * lor_or_bin(P.sens, P.sens_per_lor, i, P.T);
    P.out[i] = x;
  }
}

// 1D convolution of a smem column: out_k = sum_j g_j x[reflect(k + j - K)]
// for k in [k0, k0 + cnt), column stride `ld`.
__device__ __forceinline__ float conv_at(const float* col, int ld, int n, int k, const float* g, int K) {
  float acc = 0.0f;
  if (k - K >= 0 && k + K < n) {
    const float* x = col + (long long)(k - K) * ld;
    for (int j = 0; j <= 2 * K; ++j) acc = fmaf(g[j], x[(long long)j * ld], acc);
  } else {
    for (int j = 0; j <= 2 * K; ++j) acc = fmaf(g[j], col[(long long)reflect(k + j - K, n) * ld], acc);
  }
  return acc;
}

// ---------------------------------------------------------------------------
// pass A: radial.  One CTA per (plane, view) line of n_rad x T values.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) smooth_radial_kernel(const __grid_constant__ FinParams P) {
  extern __shared__ float tile[];          // [n_rad][T]
  __shared__ float g[2 * kMaxSmoothRadius + 1];
  const int K = P.K[0];
  for (int j = threadIdx.x; j <= 2 * K; j += blockDim.x) g[j] = P.g[0][j];
  const long long line = blockIdx.x;       // plane * V + view
  const int R = P.R, T = P.T, RT = R * T;
  const long long base = line * RT;
  const float cf = (float)P.c;
  for (int i = threadIdx.x; i < RT; i += blockDim.x) {
    const long long bin = base + i;
    float x = __ll2float_rn(__ldg(P.acc + bin)) * cf;
    if (P.sens_first && P.sens) x *= (float)lor_or_bin(P.sens, P.sens_per_lor, bin, T);
    if (P.norm) x *= (float)lor_or_bin(P.norm, P.norm_per_lor, bin, T);
    tile[i] = x;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < RT; i += blockDim.x) {
    const int r = i / T, t = i - r * T;
    P.scratch[base + i] = K == 0 ? tile[i] : conv_at(tile + t, T, R, r, g, K);
  }
}

// ---------------------------------------------------------------------------
// pass B: view.  CTA per (plane, chunk of CH inner (rad, tof) values); the
// tile holds every view of that chunk.  In place on the scratch buffer: a
// CTA reads its whole tile before writing, and tiles are disjoint.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) smooth_view_kernel(const __grid_constant__ FinParams P) {
  extern __shared__ float tile[];          // [V][CH]
  __shared__ float g[2 * kMaxSmoothRadius + 1];
  const int K = P.K[1];
  for (int j = threadIdx.x; j <= 2 * K; j += blockDim.x) g[j] = P.g[1][j];
  const int V = P.V, I = P.R * P.T, CH = P.chunk_view;
  const int n_chunks = (I + CH - 1) / CH;
  const long long plane = blockIdx.x / n_chunks;
  const int j0 = (blockIdx.x % n_chunks) * CH;
  const int cw = min(CH, I - j0);
  const long long base = plane * V * (long long)I + j0;
  for (int i = threadIdx.x; i < V * CH; i += blockDim.x) {
    const int v = i / CH, j = i - v * CH;
    if (j < cw) tile[i] = P.scratch[base + (long long)v * I + j];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < V * CH; i += blockDim.x) {
    const int v = i / CH, j = i - v * CH;
    if (j < cw) P.scratch[base + (long long)v * I + j] = conv_at(tile + j, CH, V, v, g, K);
  }
}

// ---------------------------------------------------------------------------
// pass C: axial within a ring-difference segment, then the FP64 epilogue.
// CTA per (segment, chunk of CH inner (view, rad, tof) values).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) smooth_axial_kernel(const __grid_constant__ FinParams P) {
  extern __shared__ float tile[];          // [seg_len][CH]
  __shared__ float g[2 * kMaxSmoothRadius + 1];
  const int K = P.K[2];
  for (int j = threadIdx.x; j <= 2 * K; j += blockDim.x) g[j] = P.g[2][j];
  const int nr = P.n_rings;
  const long long J = (long long)P.V * P.R * P.T;
  const int CH = P.chunk_axial;
  const long long n_chunks = (J + CH - 1) / CH;
  const int seg = (int)(blockIdx.x / n_chunks);      // 0 .. 2 nr - 2
  const long long j0 = (blockIdx.x % n_chunks) * (long long)CH;
  const int cw = (int)min((long long)CH, J - j0);
  const int d = seg - (nr - 1);                       // ring difference rb - ra
  const int ra0 = max(0, -d);
  const int L = nr - abs(d);
  for (int i = threadIdx.x; i < L * CH; i += blockDim.x) {
    const int k = i / CH, j = i - k * CH;
    const long long plane = (long long)(ra0 + k) * nr + (ra0 + k + d);
    if (j < cw) tile[i] = P.scratch[plane * J + j0 + j];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < L * CH; i += blockDim.x) {
    const int k = i / CH, j = i - k * CH;
    if (j >= cw) continue;
    const long long plane = (long long)(ra0 + k) * nr + (ra0 + k + d);
    const long long bin = plane * J + j0 + j;
    double y = (double)conv_at(tile + j, CH, L, k, g, K);
    if (P.rnorm) y = y * lor_or_bin(P.rnorm, P.norm_per_lor, bin, P.T);
    if (!P.sens_first && P.sens) y = y * lor_or_bin(P.sens, P.sens_per_lor, bin, P.T);
    P.out[bin] = y;
  }
}

// reciprocal of a normalisation sinogram, 0 where it is 0
__global__ void reciprocal_kernel(const double* __restrict__ a, double* __restrict__ r, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double v = a[i];
    r[i] = v != 0.0 ? 1.0 / v : 0.0;
  }
}

static int grid_for(long long n, int block, int sms) {
  long long g = (n + block - 1) / block;
  const long long cap = (long long)sms * 32;
  return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

cudaError_t launch_reciprocal(const double* a, double* r, long long n, int sms, cudaStream_t s) {
  reciprocal_kernel<<<grid_for(n, 256, sms), 256, 0, s>>>(a, r, n);
  return cudaGetLastError();
}

size_t finalize_smem_radial(const FinParams& p) { return sizeof(float) * (size_t)p.R * p.T; }
size_t finalize_smem_view(const FinParams& p) { return sizeof(float) * (size_t)p.V * p.chunk_view; }
size_t finalize_smem_axial(const FinParams& p) { return sizeof(float) * (size_t)p.n_rings * p.chunk_axial; }

cudaError_t launch_finalize(const FinParams& p, int sms, cudaStream_t s) {
  cudaError_t e;
  if (!p.smooth) {
    finalize_plain_kernel<<<grid_for(p.n_bins, 256, sms), 256, 0, s>>>(p);
    return cudaGetLastError();
  }
  const long long n_lines = (long long)p.n_rings * p.n_rings * p.V;
  size_t sm = finalize_smem_radial(p);
  if ((e = cudaFuncSetAttribute(smooth_radial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess) return e;
  smooth_radial_kernel<<<(unsigned)n_lines, 256, sm, s>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  const long long I = (long long)p.R * p.T;
  const long long nb = (long long)p.n_rings * p.n_rings * ((I + p.chunk_view - 1) / p.chunk_view);
  sm = finalize_smem_view(p);
  if ((e = cudaFuncSetAttribute(smooth_view_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess) return e;
  smooth_view_kernel<<<(unsigned)nb, 256, sm, s>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  const long long J = (long long)p.V * I;
  const long long na = (long long)(2 * p.n_rings - 1) * ((J + p.chunk_axial - 1) / p.chunk_axial);
  sm = finalize_smem_axial(p);
  if ((e = cudaFuncSetAttribute(smooth_axial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess) return e;
  smooth_axial_kernel<<<(unsigned)na, 256, sm, s>>>(p);
  return cudaGetLastError();
}

}  // namespace psc
