// finalize.cu -- scatter estimate from the int64 fixed-point accumulator
// (Sec. 2.2.4: multiply by the scatter-sensitivity sinogram; Sec. 2.3.2:
// multiply by the smoothing-normalisation sinogram, Gaussian-smooth, divide
// by it again).
//
// Without smoothing one FP64 elementwise pass: out = ((double)acc * c) * s,
// c = scale * 2^-32 (the operation order of the definition, so the product
// is exact to the last bit).
//
// With smoothing three passes, each reading and writing every bin once
// through a shared-memory tile that holds whole lines of the smoothed axis
// plus a reflected halo of K rows on each side (so the inner loop has no
// boundary logic and no halo is re-read from HBM):
//   A  radial: acc (int64) -> FP32 tile per (plane, view) line -> scratch
//   B  view:   scratch in place, tile (all views) x (column chunk)
//   C  axial:  scratch -> tile (planes of one ring-difference segment) x
//              (column chunk) -> FP64 epilogue (x 1/norm, x sens) -> out
// Each thread produces NB consecutive outputs along the smoothed axis from a
// register sliding window (NB + 2K shared-memory loads for NB outputs), with
// the truncation radius K a template parameter for K <= kMaxTemplK.
// Kernels are truncated at ceil(4 sigma) with weights normalised to 1; edges
// reflect half-sample symmetrically; a plane's axial neighbours are the
// planes of the same ring difference.
#include <algorithm>

#include "psc_internal.h"

namespace psc {

constexpr int NB = 8;            // outputs per thread along the smoothed axis
constexpr int kMaxTemplK = 12;   // template-specialised truncation radii 1..12

__device__ __forceinline__ int reflect(int m, int n) {
  const int p = 2 * n;
  m %= p;
  if (m < 0) m += p;
  return m >= n ? p - 1 - m : m;
}

// exact i / d for i * d < 2^32 with magic = ceil(2^32 / d) (magic 0: d = 1)
__device__ __forceinline__ unsigned fdiv(unsigned i, unsigned magic) {
  return magic ? __umulhi(i, magic) : i;
}

__device__ __forceinline__ double at(const double* a, long long i) { return __ldg(a + i); }

// ---------------------------------------------------------------------------
// no smoothing: out = (acc * c) * sens (FP64)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) finalize_plain_kernel(const __grid_constant__ FinParams P) {
  // grid.y = plane, grid.x strides over the plane's J = V * R * T bins
  const long long plane = blockIdx.y;
  const int J = P.V * P.R * P.T;
  const long long base = plane * J;
  const long long lor0 = plane * (long long)P.V * P.R;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < J; j += gridDim.x * blockDim.x) {
    const long long i = base + j;
    double x = (double)__ldg(P.acc + i) * P.c;
    if (P.sens) x = x * at(P.sens, P.sens_per_lor ? lor0 + fdiv((unsigned)j, P.magic_T) : i);
    P.out[i] = x;
  }
}

// ---------------------------------------------------------------------------
// the convolution of one thread's NB outputs along a tile column
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void conv_slide(const float* col, int ld, const float* gs, float (&o)[NB]) {
  float g[2 * K + 1];
#pragma unroll
  for (int j = 0; j <= 2 * K; ++j) g[j] = gs[j];
#pragma unroll
  for (int b = 0; b < NB; ++b) o[b] = 0.0f;
#pragma unroll
  for (int m = 0; m < NB + 2 * K; ++m) {
    const float x = col[m * ld];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = m - b;
      if (j >= 0 && j <= 2 * K) o[b] = fmaf(g[j], x, o[b]);
    }
  }
}

__device__ __forceinline__ void conv_generic(const float* col, int ld, const float* gs, int K, float (&o)[NB]) {
#pragma unroll
  for (int b = 0; b < NB; ++b) o[b] = 0.0f;
  for (int j = 0; j <= 2 * K; ++j) {
    const float gj = gs[j];
#pragma unroll
    for (int b = 0; b < NB; ++b) o[b] = fmaf(gj, col[(b + j) * ld], o[b]);
  }
}

template <int K>
__device__ __forceinline__ void conv(const float* col, int ld, const float* gs, int Kr, float (&o)[NB]) {
  if (K >= 0) conv_slide<(K >= 0 ? K : 0)>(col, ld, gs, o);
  else conv_generic(col, ld, gs, Kr, o);
}

// rows of a tile: core n rounded up to NB, plus K halo rows on each side
__host__ __device__ inline int tile_rows(int n, int K) { return (n + NB - 1) / NB * NB + 2 * K; }

// ---------------------------------------------------------------------------
// pass A: radial.  One CTA per (plane, view) line of R x T values.
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(256) smooth_radial_kernel(const __grid_constant__ FinParams P) {
  extern __shared__ float ext[];           // [tile_rows(R, K)][T]
  __shared__ float gs[2 * kMaxSmoothRadius + 1];
  const int Kr = K >= 0 ? K : P.K[0];
  for (int j = threadIdx.x; j <= 2 * Kr; j += blockDim.x) gs[j] = P.g[0][j];
  const long long line = blockIdx.x;       // plane * V + view
  const int R = P.R, T = P.T;
  const int rows = tile_rows(R, Kr);
  const long long base = line * (long long)R * T;
  const float cf = (float)P.c;
  for (int i = threadIdx.x; i < rows * T; i += blockDim.x) {
    const int e = (int)fdiv((unsigned)i, P.magic_T), t = i - e * T;
    const int s = e - Kr;
    float x = 0.0f;
    if (s < R + Kr) {
      const int r = (s >= 0 && s < R) ? s : reflect(s, R);
      const long long bin = base + (long long)r * T + t;
      x = __ll2float_rn(__ldg(P.acc + bin)) * cf;
      if (P.sens_first && P.sens) x *= (float)at(P.sens, P.sens_per_lor ? line * R + r : bin);
      if (P.norm) x *= (float)at(P.norm, P.norm_per_lor ? line * R + r : bin);
    }
    ext[i] = x;
  }
  __syncthreads();
  const int nrb = (R + NB - 1) / NB;
  for (int i = threadIdx.x; i < nrb * T; i += blockDim.x) {
    const int rb = (int)fdiv((unsigned)i, P.magic_T), t = i - rb * T;
    float o[NB];
    conv<K>(ext + rb * NB * T + t, T, gs, Kr, o);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int r = rb * NB + b;
      if (r < R) P.scratch[base + (long long)r * T + t] = o[b];
    }
  }
}

// ---------------------------------------------------------------------------
// pass B: view.  CTA per (plane, chunk of CH columns of the (rad, tof)
// plane); the tile holds every view of that chunk.  In place on the scratch
// buffer: a CTA reads its whole tile before writing, and tiles are disjoint.
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(256) smooth_view_kernel(const __grid_constant__ FinParams P) {
  extern __shared__ float ext[];           // [tile_rows(V, K)][CH]
  __shared__ float gs[2 * kMaxSmoothRadius + 1];
  const int Kr = K >= 0 ? K : P.K[1];
  for (int j = threadIdx.x; j <= 2 * Kr; j += blockDim.x) gs[j] = P.g[1][j];
  const int V = P.V, I = P.R * P.T, CH = P.chunk_view, sh = P.chunk_view_log2;
  const int n_chunks = (I + CH - 1) / CH;
  const long long plane = blockIdx.x / n_chunks;
  const int j0 = (blockIdx.x % n_chunks) * CH;
  const int cw = min(CH, I - j0);
  const int rows = tile_rows(V, Kr);
  const long long base = plane * V * (long long)I + j0;
  for (int i = threadIdx.x; i < rows * CH; i += blockDim.x) {
    const int e = i >> sh, c = i & (CH - 1);
    const int s = e - Kr;
    float x = 0.0f;
    if (c < cw && s < V + Kr) {
      const int v = (s >= 0 && s < V) ? s : reflect(s, V);
      x = P.scratch[base + (long long)v * I + c];
    }
    ext[i] = x;
  }
  __syncthreads();
  const int nvb = (V + NB - 1) / NB;
  for (int i = threadIdx.x; i < nvb * CH; i += blockDim.x) {
    const int vb = i >> sh, c = i & (CH - 1);
    if (c >= cw) continue;
    float o[NB];
    conv<K>(ext + vb * NB * CH + c, CH, gs, Kr, o);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int v = vb * NB + b;
      if (v < V) P.scratch[base + (long long)v * I + c] = o[b];
    }
  }
}

// ---------------------------------------------------------------------------
// pass C: axial within a ring-difference segment, then the FP64 epilogue.
// CTA per (segment, chunk of CH columns of the (view, rad, tof) volume).
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(256) smooth_axial_kernel(const __grid_constant__ FinParams P) {
  extern __shared__ float ext[];           // [tile_rows(L, K)][CH]
  __shared__ float gs[2 * kMaxSmoothRadius + 1];
  const int Kr = K >= 0 ? K : P.K[2];
  for (int j = threadIdx.x; j <= 2 * Kr; j += blockDim.x) gs[j] = P.g[2][j];
  const int nr = P.n_rings;
  const int J = P.V * P.R * P.T;
  const int CH = P.chunk_axial, sh = P.chunk_axial_log2;
  const int n_chunks = (J + CH - 1) / CH;
  const int seg = blockIdx.x / n_chunks;             // 0 .. 2 nr - 2
  const int j0 = (blockIdx.x % n_chunks) * CH;
  const int cw = min(CH, J - j0);
  const int d = seg - (nr - 1);                      // ring difference rb - ra
  const int ra0 = max(0, -d);
  const int L = nr - abs(d);
  const int rows = tile_rows(L, Kr);
  for (int i = threadIdx.x; i < rows * CH; i += blockDim.x) {
    const int e = i >> sh, c = i & (CH - 1);
    const int s = e - Kr;
    float x = 0.0f;
    if (c < cw && s < L + Kr) {
      const int k = (s >= 0 && s < L) ? s : reflect(s, L);
      const long long plane = (long long)(ra0 + k) * nr + (ra0 + k + d);
      x = P.scratch[plane * J + j0 + c];
    }
    ext[i] = x;
  }
  __syncthreads();
  const long long lors = (long long)P.V * P.R;
  const int nkb = (L + NB - 1) / NB;
  for (int i = threadIdx.x; i < nkb * CH; i += blockDim.x) {
    const int kb = i >> sh, c = i & (CH - 1);
    if (c >= cw) continue;
    float o[NB];
    conv<K>(ext + kb * NB * CH + c, CH, gs, Kr, o);
    const int lor_in_plane = (int)fdiv((unsigned)(j0 + c), P.magic_T);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int k = kb * NB + b;
      if (k >= L) break;
      const long long plane = (long long)(ra0 + k) * nr + (ra0 + k + d);
      const long long bin = plane * J + j0 + c;
      const long long lor = plane * lors + lor_in_plane;
      double y = (double)o[b];
      if (P.rnorm) y = y * at(P.rnorm, P.norm_per_lor ? lor : bin);
      if (!P.sens_first && P.sens) y = y * at(P.sens, P.sens_per_lor ? lor : bin);
      P.out[bin] = y;
    }
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

size_t finalize_smem_radial(const FinParams& p) { return sizeof(float) * (size_t)tile_rows(p.R, p.K[0]) * p.T; }
size_t finalize_smem_view(const FinParams& p) { return sizeof(float) * (size_t)tile_rows(p.V, p.K[1]) * p.chunk_view; }
size_t finalize_smem_axial(const FinParams& p) { return sizeof(float) * (size_t)tile_rows(p.n_rings, p.K[2]) * p.chunk_axial; }

template <template <int> class Launcher, int K>
static cudaError_t dispatch_k(int k, const FinParams& p, size_t smem, unsigned grid, cudaStream_t s) {
  if constexpr (K > kMaxTemplK) {
    return Launcher<-1>::run(p, smem, grid, s);
  } else {
    if (k == K) return Launcher<K>::run(p, smem, grid, s);
    return dispatch_k<Launcher, K + 1>(k, p, smem, grid, s);
  }
}

#define PSC_LAUNCHER(NAME, KERNEL)                                                             \
  template <int K>                                                                             \
  struct NAME {                                                                                \
    static cudaError_t run(const FinParams& p, size_t smem, unsigned grid, cudaStream_t s) {    \
      cudaError_t e = cudaFuncSetAttribute(KERNEL<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
      if (e != cudaSuccess) return e;                                                          \
      KERNEL<K><<<grid, 256, smem, s>>>(p);                                                    \
      return cudaGetLastError();                                                               \
    }                                                                                          \
  };
PSC_LAUNCHER(RadialL, smooth_radial_kernel)
PSC_LAUNCHER(ViewL, smooth_view_kernel)
PSC_LAUNCHER(AxialL, smooth_axial_kernel)

cudaError_t launch_finalize(const FinParams& p, int sms, cudaStream_t s) {
  cudaError_t e;
  if (!p.smooth) {
    const long long J = (long long)p.V * p.R * p.T;
    const unsigned planes = (unsigned)((long long)p.n_rings * p.n_rings);
    const long long per_plane = std::max(1LL, std::min((J + 255) / 256, 8LL * sms / (long long)planes + 1));
    finalize_plain_kernel<<<dim3((unsigned)per_plane, planes), 256, 0, s>>>(p);
    return cudaGetLastError();
  }
  const unsigned n_lines = (unsigned)((long long)p.n_rings * p.n_rings * p.V);
  if ((e = dispatch_k<RadialL, 1>(p.K[0] == 0 ? -1 : p.K[0], p, finalize_smem_radial(p), n_lines, s)) != cudaSuccess) return e;
  const long long I = (long long)p.R * p.T;
  const unsigned nb = (unsigned)((long long)p.n_rings * p.n_rings * ((I + p.chunk_view - 1) / p.chunk_view));
  if ((e = dispatch_k<ViewL, 1>(p.K[1] == 0 ? -1 : p.K[1], p, finalize_smem_view(p), nb, s)) != cudaSuccess) return e;
  const long long J = (long long)p.V * I;
  const unsigned na = (unsigned)((long long)(2 * p.n_rings - 1) * ((J + p.chunk_axial - 1) / p.chunk_axial));
  return dispatch_k<AxialL, 1>(p.K[2] == 0 ? -1 : p.K[2], p, finalize_smem_axial(p), na, s);
}

}  // namespace psc
