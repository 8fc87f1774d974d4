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
constexpr int kMaxRings = 128;   // rings per scanner for the axial pass

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
// Exact IEEE conversions and FP64 products on the integer pipes.
//
// The GB300 FP64 pipe retires about 2e11 operations per second (measured with
// ncu): one FP64 instruction per bin costs ~27 ms on a 5.5e9-bin sinogram.
// These helpers give the same round-to-nearest-even results as the FP64
// hardware from 32/64-bit integer instructions; zero is handled inline and
// the rare operands outside the normal range (subnormal, inf, NaN) fall back
// to the hardware instruction.
// ---------------------------------------------------------------------------
constexpr unsigned long long kMant52 = (1ull << 52) - 1;

// index of the highest / lowest set bit of a non-zero 64-bit value, from the
// 32-bit bit-scan instructions
__device__ __forceinline__ int msb64(unsigned long long u) {
  const unsigned hi = (unsigned)(u >> 32);
  return hi ? 63 - __clz(hi) : 31 - __clz((unsigned)u);
}
__device__ __forceinline__ int lsb64(unsigned long long u) {
  const unsigned lo = (unsigned)u;
  return lo ? __ffs(lo) - 1 : 31 + __ffs((unsigned)(u >> 32));
}

// round-to-nearest-even of m >> sh (sh >= 1), returning the carry-adjusted
// mantissa; e is bumped when rounding carries into a new bit
__device__ __forceinline__ unsigned long long rne_shift(unsigned long long m, int sh, bool sticky,
                                                        int width, int& e) {
  const unsigned long long q = m >> sh;
  const unsigned long long rem = m & ((1ull << sh) - 1);
  const unsigned long long half = 1ull << (sh - 1);
  unsigned long long r = q;
  if (rem > half || (rem == half && (sticky || (q & 1)))) r = q + 1;
  if (r >> width) {
    r >>= 1;
    ++e;
  }
  return r;
}

// non-negative int64 -> double (RNE)
__device__ __forceinline__ double i64_to_f64(long long v) {
  const unsigned long long u = (unsigned long long)v;
  if (u == 0) return 0.0;
  int e = msb64(u);
  unsigned long long m = e <= 52 ? u << (52 - e) : rne_shift(u, e - 52, false, 53, e);
  return __longlong_as_double(((unsigned long long)(e + 1023) << 52) | (m & kMant52));
}

// non-negative int64 -> float (RNE)
__device__ __forceinline__ float i64_to_f32(long long v) {
  const unsigned long long u = (unsigned long long)v;
  if (u == 0) return 0.0f;
  int e = msb64(u);
  unsigned long long m = e <= 23 ? u << (23 - e) : rne_shift(u, e - 23, false, 24, e);
  return __int_as_float((int)(((unsigned)(e + 127) << 23) | ((unsigned)m & 0x7fffffu)));
}

// float -> double (exact)
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = (unsigned)__float_as_int(f);
  const unsigned ef = (b >> 23) & 0xffu;
  if ((b & 0x7fffffffu) == 0) return (b >> 31) ? -0.0 : 0.0;
  if (ef == 0 || ef == 0xffu) return (double)f;
  return __longlong_as_double(((unsigned long long)(b >> 31) << 63) |
                              ((unsigned long long)(ef - 127 + 1023) << 52) |
                              ((unsigned long long)(b & 0x7fffffu) << 29));
}

// (double)x * b (RNE, one rounding of the exact product) for finite x, b
__device__ __forceinline__ double fmul_fd(float x, double b) {
  const unsigned xb = (unsigned)__float_as_int(x);
  const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
  const unsigned long long sign = ((unsigned long long)(xb >> 31) << 63) ^ (ub & (1ull << 63));
  const int ex = (int)((xb >> 23) & 0xffu), eb = (int)((ub >> 52) & 0x7ff);
  if ((xb << 1) == 0 || (ub << 1) == 0) return __longlong_as_double((long long)sign);
  if (ex == 0 || ex == 0xff || eb == 0 || eb == 0x7ff) return (double)x * b;
  const unsigned long long mx = (xb & 0x7fffffu) | 0x800000u;          // 24 bits
  const unsigned long long mb = (ub & kMant52) | (1ull << 52);         // 53 bits
  // P = mx * mb in [2^75, 2^77) = hi 2^32 + lo; T = P >> 13 in [2^62, 2^64)
  const unsigned long long lo = mx * (mb & 0xffffffffull);
  const unsigned long long hi = mx * (mb >> 32);
  const unsigned long long T = (hi << 19) + (lo >> 13);
  const bool sticky = (lo & 0x1fffull) != 0;
  const int top = (int)(T >> 63);
  int e = ex + eb - 127 + top;
  const unsigned long long m = rne_shift(T, 10 + top, sticky, 53, e);
  if (e <= 0 || e >= 0x7ff) return (double)x * b;
  return __longlong_as_double((long long)(sign | ((unsigned long long)e << 52) | (m & kMant52)));
}

// a * b (RNE) for finite doubles
__device__ __forceinline__ double dmul(double a, double b) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
  const unsigned long long sign = (ua ^ ub) & (1ull << 63);
  const int ea = (int)((ua >> 52) & 0x7ff), eb = (int)((ub >> 52) & 0x7ff);
  if (((ua << 1) == 0) || ((ub << 1) == 0)) return __longlong_as_double((long long)sign);
  if (ea == 0 || eb == 0 || ea == 0x7ff || eb == 0x7ff) return a * b;
  const unsigned long long ma = (ua & kMant52) | (1ull << 52), mb = (ub & kMant52) | (1ull << 52);
  // ma * mb in [2^104, 2^106): top 64 bits of (ma * mb) << 22, sticky below
  const unsigned long long hi = __umul64hi(ma << 11, mb << 11);
  const bool sticky = lsb64(ma) + lsb64(mb) < 42;
  int e = ea + eb - 1023;
  const int top = (int)(hi >> 63);
  e += top;
  const unsigned long long m = rne_shift(hi, 10 + top, sticky, 53, e);
  if (e <= 0 || e >= 0x7ff) return a * b;
  return __longlong_as_double((long long)(sign | ((unsigned long long)e << 52) | (m & kMant52)));
}

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
    double x = dmul(i64_to_f64(__ldg(P.acc + i)), P.c);
    if (P.sens) x = dmul(x, at(P.sens, P.sens_per_lor ? lor0 + fdiv((unsigned)j, P.magic_T) : i));
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
      x = i64_to_f32(__ldg(P.acc + bin)) * cf;
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
  __shared__ long long s_bin[kMaxRings];   // first bin of the segment's plane k
  __shared__ long long s_lor[kMaxRings];   // first LOR of the segment's plane k
  __shared__ int s_src[kMaxRings + 2 * kMaxSmoothRadius + NB];  // core row of tile row e (-1: pad)
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
  const long long lors = (long long)P.V * P.R;
  for (int k = threadIdx.x; k < L; k += blockDim.x) {
    const long long plane = (long long)(ra0 + k) * nr + (ra0 + k + d);
    s_bin[k] = plane * J;
    s_lor[k] = plane * lors;
  }
  for (int e = threadIdx.x; e < rows; e += blockDim.x) {
    const int s = e - Kr;
    s_src[e] = s < L + Kr ? ((s >= 0 && s < L) ? s : reflect(s, L)) : -1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < rows * CH; i += blockDim.x) {
    const int e = i >> sh, c = i & (CH - 1);
    const int k = s_src[e];
    ext[i] = (c < cw && k >= 0) ? P.scratch[s_bin[k] + j0 + c] : 0.0f;
  }
  __syncthreads();
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
      const long long bin = s_bin[k] + j0 + c;
      const long long lor = s_lor[k] + lor_in_plane;
      double y;
      if (P.rnorm) {
        y = fmul_fd(o[b], at(P.rnorm, P.norm_per_lor ? lor : bin));
        if (!P.sens_first && P.sens) y = dmul(y, at(P.sens, P.sens_per_lor ? lor : bin));
      } else if (!P.sens_first && P.sens) {
        y = fmul_fd(o[b], at(P.sens, P.sens_per_lor ? lor : bin));
      } else {
        y = f32_to_f64(o[b]);
      }
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
