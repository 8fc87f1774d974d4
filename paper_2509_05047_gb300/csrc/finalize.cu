// finalize.cu -- scatter estimate from the int64 fixed-point accumulator
// (Sec. 2.2.4: multiply by the scatter-sensitivity sinogram; Sec. 2.3.2:
// multiply by the smoothing-normalisation sinogram, Gaussian-smooth, divide
// by it again).
//
// Without smoothing one FP64 elementwise pass: out = ((double)acc * c) * s,
// c = scale * 2^-32 (the operation order of the definition, so the product
// is exact to the last bit).
//
// With smoothing three separable passes, each reading and writing every bin
// once.  A thread owns one column of the smoothed axis and slides down it
// with a register window: NB outputs per step from NB new loads, the 2K
// halo rows carried over in registers, the reflected edge rows loaded by
// index.  Loads and stores of a warp cover 32 consecutive bins of the
// innermost axes, so every access is coalesced; no shared memory and no
// barriers are needed, and enough warps are resident to keep HBM busy.
//   A  radial: acc (int64) -> FP32, columns (plane, view, tof) along rad,
//              into the first half of the output buffer (used as scratch)
//   B  view:   that -> FP32 working sinogram, columns (plane, rad, tof)
//   C  axial:  working sinogram -> epilogue (the FP32 value widened exactly,
//              x 1/norm, x sens in FP64, each product rounded to nearest)
//              -> out, columns (segment, view, rad, tof) along the
//              segment's planes
// No pass writes what it reads.  Kernels are truncated at ceil(4 sigma) with
// weights normalised to 1 and zero-padded to the instantiated radius KT
// (exact for K <= 8, then 10, 12, 16, 20, 24; a per-tap loop beyond), so the
// FMA chain is the same for every KT >= K; edges reflect half-sample
// symmetrically; a plane's axial neighbours are the planes of the same ring
// difference.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <type_traits>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "psc.h"
#include "psc_internal.h"

namespace psc {

constexpr int NB = 8;            // outputs per window step along the smoothed axis
// wide windows (radius 16 and up) take half the step: fewer registers, more warps
template <int KT>
constexpr int kNb = KT >= 16 ? 4 : NB;
constexpr int kSmoothThreads = 256;

// half-sample symmetric reflection of row m into [0, n), periodic beyond
// one reflection (only axes shorter than the kernel get there)
__device__ __forceinline__ int reflect(int m, int n) {
  if (m >= -n && m < 2 * n) return m < 0 ? -m - 1 : (m >= n ? 2 * n - 1 - m : m);
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

// the rare operands outside the normal range go to the FP64 hardware; kept
// out of line so the compiler never if-converts them into the common path
__device__ __noinline__ double hw_f32_to_f64(float f) { return (double)f; }
__device__ __noinline__ double hw_dmul(double a, double b) { return a * b; }
__device__ __noinline__ float hw_f64_to_f32(double d) { return (float)d; }

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
  if (ef == 0 || ef == 0xffu) return hw_f32_to_f64(f);
  return __longlong_as_double(((unsigned long long)(b >> 31) << 63) |
                              ((unsigned long long)(ef - 127 + 1023) << 52) |
                              ((unsigned long long)(b & 0x7fffffu) << 29));
}

// double -> float (RNE) from the two 32-bit halves: the 23 kept mantissa
// bits, then +1 on the rounding decision (a carry moves into the exponent,
// and past the largest finite value to infinity, as IEEE rounding does)
__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  if ((u << 1) == 0) return __uint_as_float(hi & 0x80000000u);
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  if (e < 1 || e > 254) return hw_f64_to_f32(d);
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
  return __uint_as_float(((hi & 0x80000000u) | ((unsigned)e << 23) | m) + up);
}

// a sinogram factor in FP32: from the FP32 copy when there is one, else
// rounded from the FP64 values
__device__ __forceinline__ float factor(const float* f32, const double* f64, long long i) {
  return f32 ? __ldg(f32 + i) : f64_to_f32(__ldg(f64 + i));
}

// a * b (RNE) for finite doubles
__device__ __forceinline__ double dmul(double a, double b) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
  const unsigned long long sign = (ua ^ ub) & (1ull << 63);
  const int ea = (int)((ua >> 52) & 0x7ff), eb = (int)((ub >> 52) & 0x7ff);
  // zero, subnormal, infinite and NaN operands: one range test on the exponent
  // fields first (a zero test on an FP64 operand's bits can be compiled to an
  // FP64 compare, which this keeps off the common path)
  if ((unsigned)(ea - 1) >= 0x7feu || (unsigned)(eb - 1) >= 0x7feu) {
    if (((ua << 1) == 0 && eb != 0x7ff) || ((ub << 1) == 0 && ea != 0x7ff))
      return __longlong_as_double((long long)sign);
    return hw_dmul(a, b);
  }
  const unsigned long long ma = (ua & kMant52) | (1ull << 52), mb = (ub & kMant52) | (1ull << 52);
  // ma * mb in [2^104, 2^106): top 64 bits of (ma * mb) << 22, sticky below
  const unsigned long long hi = __umul64hi(ma << 11, mb << 11);
  const bool sticky = lsb64(ma) + lsb64(mb) < 42;
  int e = ea + eb - 1023;
  const int top = (int)(hi >> 63);
  e += top;
  const unsigned long long m = rne_shift(hi, 10 + top, sticky, 53, e);
  if (e <= 0 || e >= 0x7ff) return hw_dmul(a, b);
  return __longlong_as_double((long long)(sign | ((unsigned long long)e << 52) | (m & kMant52)));
}

// (double)y * f, rounded to nearest even, for a float y and a double f, in
// 32-bit integer words: the 24-bit by 53-bit significand product, scaled by
// 2^8, from the low and high halves of four 32 x 32-bit products (fewer
// instructions than two 64-bit products, measured); the leading bit is normalised to bit
// 84 of the 96-bit value, the top 53 bits are the significand and the low
// word decides the rounding (ties to even); the rounded significand (hidden
// bit included) is added to the exponent field, so a rounding carry moves
// into the exponent (and past the largest finite value to infinity) as IEEE
// rounding does.  A zero y is handled inline; other zero, subnormal, infinite
// and NaN operands and results outside the normal range go to the FP64
// hardware.
__device__ __forceinline__ double mul_f32_f64(float y, double f) {
  const unsigned by = (unsigned)__float_as_int(y);
  const unsigned long long uf = (unsigned long long)__double_as_longlong(f);
  const unsigned fhi = (unsigned)(uf >> 32);
  const unsigned ey = (by >> 23) & 0xffu, ef = (fhi >> 20) & 0x7ffu;
  const unsigned long long sign = (unsigned long long)((by ^ fhi) & 0x80000000u) << 32;
  // zero, subnormal, infinite and NaN operands: one range test on the two
  // exponent fields (integer compares; a zero test on the FP64 operand's bits
  // can be compiled to an FP64 compare); y = 0 with a finite f is the common
  // case among them (bins the smoothing leaves empty)
  if (ey - 1u >= 254u || ef - 1u >= 0x7feu) {
    if ((by << 1) == 0u && ef != 0x7ffu) return __longlong_as_double((long long)sign);
    return hw_dmul(hw_f32_to_f64(y), f);
  }
  // P 2^8 = my 2^8 x (fh 2^32 + fl) as three 32-bit words w2:w1:w0 from 32 x 32-bit
  // products (low and high halves); P 2^8 in [2^83, 2^85), its leading bit at w2 bit 20
  // (top = 1) or 19 (shifted up by one).  The 53-bit significand is then w2:w1 and w0
  // holds the rounding bits.
  const unsigned m = (by << 8) | 0x80000000u;
  const unsigned fl = (unsigned)uf, fh = (fhi & 0xfffffu) | 0x100000u;
  const unsigned a0 = m * fl, a1 = __umulhi(m, fl), b0 = m * fh, b1 = __umulhi(m, fh);
  unsigned w1 = b0 + a1;
  unsigned w2 = b1 + (w1 < a1 ? 1u : 0u), w0 = a0;
  const unsigned top = w2 >> 20;
  if (!top) {
    w2 = __funnelshift_l(w1, w2, 1);
    w1 = __funnelshift_l(w0, w1, 1);
    w0 <<= 1;
  }
  const unsigned up = (w0 > 0x80000000u || (w0 == 0x80000000u && (w1 & 1u))) ? 1u : 0u;
  const int e = (int)ey - 127 + (int)ef + (int)top;  // (ey - 127) + (ef - 1023) + 1023, +1 when P >= 2^76
  if (e <= 0 || e >= 0x7ff) return hw_dmul(hw_f32_to_f64(y), f);
  const unsigned lo = w1 + up;
  const unsigned hiw = (((unsigned)(e - 1) << 20) + w2 + (lo < up ? 1u : 0u)) | (unsigned)(sign >> 32);
  return __hiloint2double((int)hiw, (int)lo);
}

// The j-th plane a launch covers: plane j itself, or, when the launch is
// restricted to ring-difference segments [seg_lo, seg_hi), the j-th plane of
// those segments in segment order and, within a segment, by ring a (plane
// ra (n_rings + 1) + d for d = s - n_rings + 1).  The host sizes the grid to
// the planes of the range, so the walk ends inside it.
__device__ __forceinline__ long long plane_at(const FinParams& P, long long j) {
  if (P.seg_hi <= P.seg_lo) return j;
  const int nr = P.n_rings;
  int sg = P.seg_lo;
  for (;;) {
    const int L = nr - abs(sg - (nr - 1));
    if (j < L || sg + 1 >= P.seg_hi) {
      const int d = sg - (nr - 1);
      return (long long)(max(0, -d) + (int)j) * (nr + 1) + d;
    }
    j -= L;
    ++sg;
  }
}

// ---------------------------------------------------------------------------
// no smoothing: out = (acc * c) * sens (FP64)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) finalize_plain_kernel(const __grid_constant__ FinParams P) {
  // grid.y = plane, grid.x strides over the plane's J = V * R * T bins
  const long long plane = plane_at(P, P.plane0 + (long long)blockIdx.y);
  const int J = P.V * P.R * P.T;
  const long long base = plane * J;
  const long long lor0 = plane * (long long)P.V * P.R;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < J; j += gridDim.x * blockDim.x) {
    const long long i = dbg_idx(P.dbg, kSiteFinBin, base + j, P.n_bins);
    double x = dmul(i64_to_f64(__ldg(P.acc + i)), P.c);
    if (P.sens)
      x = dmul(x, at(P.sens, P.sens_per_lor ? dbg_idx(P.dbg, kSiteFinLor, lor0 + fdiv((unsigned)j, P.magic_T),
                                                      P.n_bins / P.T)
                                            : i));
    P.out[i] = x;
  }
}



// ---------------------------------------------------------------------------
// the sliding window down one column of n rows; row r of the source is
// src[r * stride] (rows outside [0, n) reflect).  cvt(raw, r) -> float;
// store(o0, s[NB]) receives the outputs o0 .. o0 + NB - 1 of a step (those
// below n are real).  Each output is the FMA chain sum_j g[j] * x[o - KT + j],
// j = 0 .. 2 KT, in increasing j.  The NB loads of a step are issued before
// any of them is converted, and rows are reflected only in the edge steps.
// ---------------------------------------------------------------------------
using Weights = float[2 * kMaxSmoothRadius + 1];

template <int KT, int NBS, class In, class Cvt, class Store>
__device__ __forceinline__ void slide(const In* __restrict__ src, long long stride, int n, const Weights& g,
                                      Cvt cvt, Store store) {
  constexpr int NB = NBS;
  float w[NB + 2 * KT];
#pragma unroll
  for (int j = 0; j < 2 * KT; ++j) {
    const int r = reflect(j - KT, n);
    w[j] = cvt(__ldg(src + r * stride), r);
  }
  for (int o0 = 0; o0 < n; o0 += NB) {
    In raw[NB];
    int rr[NB];
    if (o0 + KT + NB <= n) {
      const In* p = src + (long long)(o0 + KT) * stride;
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        raw[q] = __ldg(p + q * stride);
        rr[q] = o0 + KT + q;
      }
    } else {
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        rr[q] = reflect(o0 + KT + q, n);
        raw[q] = __ldg(src + rr[q] * stride);
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) w[2 * KT + q] = cvt(raw[q], rr[q]);
    float s[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      s[q] = 0.0f;
#pragma unroll
      for (int j = 0; j <= 2 * KT; ++j) s[q] = fmaf(g[j], w[q + j], s[q]);
    }
    store(o0, s);
#pragma unroll
    for (int j = 0; j < 2 * KT; ++j) w[j] = w[NB + j];
  }
}

// radii above the largest instantiated window: one load per tap
template <class In, class Cvt, class Store>
__device__ __forceinline__ void slide_generic(const In* __restrict__ src, long long stride, int n, int K,
                                              const Weights& g, Cvt cvt, Store store) {
  for (int o0 = 0; o0 < n; o0 += NB) {
    float s[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      s[q] = 0.0f;
      for (int j = 0; j <= 2 * K; ++j) {
        const int r = reflect(o0 + q - K + j, n);
        s[q] = fmaf(g[j], cvt(__ldg(src + r * stride), r), s[q]);
      }
    }
    store(o0, s);
  }
}

template <int KT, int NBS = kNb<KT>, class In, class Cvt, class Store>
__device__ __forceinline__ void slide_any(const In* src, long long stride, int n, int K, const Weights& g, Cvt cvt,
                                          Store store) {
  if constexpr (KT >= 0) slide<KT, NBS>(src, stride, n, g, cvt, store);
  else slide_generic(src, stride, n, K, g, cvt, store);
}

// ---------------------------------------------------------------------------
// pass A: radial.  grid (ceil(V T / 256), planes); a thread owns the column
// (plane, view, tof) and slides along rad.  acc * c [x sens] [x norm] in
// FP32, written as FP32 into the first half of the output buffer.
// ---------------------------------------------------------------------------
template <int KT>
__global__ void __launch_bounds__(kSmoothThreads) smooth_radial_kernel(const __grid_constant__ FinParams P) {
  constexpr int NB = kNb<KT>;
  const int VT = P.V * P.T;
  const int c = blockIdx.x * kSmoothThreads + threadIdx.x;
  if (c >= VT) return;
  const int v = (int)fdiv((unsigned)c, P.magic_T), t = c - v * P.T;
  const long long line = plane_at(P, blockIdx.y) * P.V + v;
  const int R = P.R, T = P.T;
  const long long base = line * R * T + t;  // bin of (line, r = 0, t)
#if PSC_DEBUG
  // the column's rows 0 .. R - 1 (reflection stays inside them) and its LORs
  if (dbg_idx(P.dbg, kSiteFinColumn, base + (long long)(R - 1) * T, P.n_bins) != base + (long long)(R - 1) * T ||
      dbg_idx(P.dbg, kSiteFinLor, line * R + R - 1, P.n_bins / T) != line * R + R - 1)
    return;
#endif
  const float cf = (float)P.c;
  const bool per_bin_factor = (P.sens_first && P.sens) || P.norm;
  float* dst = reinterpret_cast<float*>(P.out) + base;
  auto cvt = [&](long long q, int r) {
    float x = i64_to_f32(q) * cf;
    if (per_bin_factor) {
      const long long bin = base + (long long)r * T, lor = line * R + r;
      if (P.sens_first && P.sens) x *= factor(P.sens32, P.sens, P.sens_per_lor ? lor : bin);
      if (P.norm) x *= factor(P.norm32, P.norm, P.norm_per_lor ? lor : bin);
    }
    return x;
  };
  auto store = [&](int r0, const float (&y)[NB]) {
#pragma unroll
    for (int q = 0; q < NB; ++q)
      if (r0 + q < R) dst[(r0 + q) * T] = y[q];
  };
  slide_any<KT>(P.acc + base, T, R, P.K[0], P.g[0], cvt, store);
}

// ---------------------------------------------------------------------------
// pass B: view.  grid (ceil(R T / 256), planes); a thread owns the column
// (plane, rad, tof) and slides along view.
// ---------------------------------------------------------------------------
template <int KT>
__global__ void __launch_bounds__(kSmoothThreads) smooth_view_kernel(const __grid_constant__ FinParams P) {
  constexpr int NB = KT >= 0 && KT < 16 ? 12 : kNb<KT>;
  const int I = P.R * P.T;
  const int i = blockIdx.x * kSmoothThreads + threadIdx.x;
  if (i >= I) return;
  const long long base = plane_at(P, blockIdx.y) * P.V * I + i;
#if PSC_DEBUG
  if (dbg_idx(P.dbg, kSiteFinColumn, base + (long long)(P.V - 1) * I, P.n_bins) != base + (long long)(P.V - 1) * I)
    return;
#endif
  const float* src = reinterpret_cast<const float*>(P.out) + base;
  float* dst = P.scratch + base;
  auto cvt = [](float x, int) { return x; };
  const int V = P.V;
  auto store = [&](int v0, const float (&y)[NB]) {
#pragma unroll
    for (int q = 0; q < NB; ++q)
      if (v0 + q < V) dst[(v0 + q) * I] = y[q];
  };
  slide_any<KT, NB>(src, I, V, P.K[1], P.g[1], cvt, store);
}

// The epilogue of one output: the FP32 smoothed value y in FP64 (exactly
// widened, times the FP64 reciprocal of the normalisation fr, times the FP64
// sensitivity fs, each product rounded to nearest, on the integer pipes), or
// for the normalisation sinogram (kDivide) y over the scaled input bin qa,
// 0 where qa is 0.
template <bool kDivide, bool kNorm>
__device__ __forceinline__ double axial_epilogue(float y, long long qa, double fr, double fs, bool use_sens,
                                                 float cf) {
  if (kDivide) return f32_to_f64(qa != 0 ? y / (i64_to_f32(qa) * cf) : 0.0f);
  if (kNorm) {
    const double x = mul_f32_f64(y, fr);
    return use_sens ? dmul(x, fs) : x;
  }
  return use_sens ? mul_f32_f64(y, fs) : f32_to_f64(y);
}

// The same epilogue on the FP64 hardware: y widened (exact) and multiplied by
// correctly rounded FP64 instructions, so the same bits as axial_epilogue.
// GB300's FP64 pipe retires about 2 operations per clock per SM; the axial
// pass sends one output of each 2-output step here and the other through the
// integer-pipe product, which splits the epilogue between the two pipes.
template <bool kDivide, bool kNorm>
__device__ __forceinline__ double axial_epilogue_fp64(float y, long long qa, double fr, double fs, bool use_sens,
                                                      float cf) {
  if (kDivide) return (double)(qa != 0 ? y / (i64_to_f32(qa) * cf) : 0.0f);
  if (kNorm) {
    const double x = (double)y * fr;
    return use_sens ? x * fs : x;
  }
  return use_sens ? (double)y * fs : (double)y;
}

// One axial column of an instantiated radius KT: the sliding window of slide
// with 2-output steps, written out for this pass.  The step's first output
// takes the integer-pipe epilogue and its second the FP64-pipe one.  Row,
// output and factor addresses advance by running pointers (one 64-bit add
// per step each); for
// columns of at least KT planes the first window's reflected rows are copies
// of rows 0 .. KT - 1, so it takes KT loads instead of 2 KT.  Same loads (up
// to those copies), same FMA chains and same outputs as slide.
template <int KT, bool kDivide, bool kNorm>
__device__ __forceinline__ void axial_column(const FinParams& P, long long bin0, long long lor0, long long bin_step,
                                             long long lor_step, int L) {
  constexpr int NB = 2;
  const Weights& g = P.g[2];
  const float* __restrict__ src = P.scratch + bin0;
  float w[2 * KT + NB];
  if (L >= KT) {
#pragma unroll
    for (int r = 0; r < KT; ++r) {  // row r, and row -1 - r reflected onto it
      const float x = __ldg(src + r * bin_step);
      w[KT + r] = x;
      w[KT - 1 - r] = x;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 2 * KT; ++j) w[j] = __ldg(src + reflect(j - KT, L) * bin_step);
  }
  const bool use_sens = !P.sens_first && P.sens;
  const float cf = (float)P.c;
  const long long step2 = NB * bin_step;
  const float* nxt = src + KT * bin_step;  // row o0 + KT
  double* dst = P.out + bin0;
  const long long* ap = P.acc + bin0;
  const long long rs = P.norm_per_lor ? lor_step : bin_step, ss = P.sens_per_lor ? lor_step : bin_step;
  const double* rp = kNorm ? P.rnorm + (P.norm_per_lor ? lor0 : bin0) : nullptr;
  const double* sp = use_sens ? P.sens + (P.sens_per_lor ? lor0 : bin0) : nullptr;
  for (int o0 = 0; o0 < L; o0 += NB) {
    float r0, r1;
    if (o0 + KT + NB <= L) {
      r0 = __ldg(nxt);
      r1 = __ldg(nxt + bin_step);
    } else {
      r0 = __ldg(src + reflect(o0 + KT, L) * bin_step);
      r1 = __ldg(src + reflect(o0 + KT + 1, L) * bin_step);
    }
    nxt += step2;
    w[2 * KT] = r0;
    w[2 * KT + 1] = r1;
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
    for (int j = 0; j <= 2 * KT; ++j) {
      s0 = fmaf(g[j], w[j], s0);
      s1 = fmaf(g[j], w[j + 1], s1);
    }
    const bool two = o0 + 1 < L;
    // the step's factors, loaded before its outputs are stored
    long long qa0 = 0, qa1 = 0;
    double fr0 = 1.0, fr1 = 1.0, fs0 = 1.0, fs1 = 1.0;
    if (kDivide) {
      qa0 = __ldg(ap);
      if (two) qa1 = __ldg(ap + bin_step);
      ap += step2;
    } else {
      if (kNorm) {
        fr0 = __ldg(rp);
        if (two) fr1 = __ldg(rp + rs);
        rp += NB * rs;
      }
      if (use_sens) {
        fs0 = __ldg(sp);
        if (two) fs1 = __ldg(sp + ss);
        sp += NB * ss;
      }
    }
    dst[0] = axial_epilogue<kDivide, kNorm>(s0, qa0, fr0, fs0, use_sens, cf);
    if (two) dst[bin_step] = axial_epilogue_fp64<kDivide, kNorm>(s1, qa1, fr1, fs1, use_sens, cf);
    dst += step2;
#pragma unroll
    for (int j = 0; j < 2 * KT; ++j) w[j] = w[NB + j];
  }
}

// ---------------------------------------------------------------------------
// pass C: axial within a ring-difference segment, then the epilogue.
// grid (ceil(R T / 256), segments x V); a thread owns the column (segment,
// view, rad, tof) and slides along the segment's planes p0 + k (n_rings + 1).
// ---------------------------------------------------------------------------
// kDivide: the output is the smoothed value over the (scaled) input bin,
// 0 where the input is 0 (the smoothing-normalisation sinogram)
// kNorm: a normalisation reciprocal multiplies the output (compiled in only
// where there is one: its factors would otherwise hold registers)
// resident CTAs per SM asked of the compiler for windows up to radius 8: the
// pass waits on memory, and 6 CTAs (48 warps) outweigh a 12-byte spill
// (measured); with a normalisation 4 (no spill); wider windows keep their
// registers
template <int KT, bool kNorm>
constexpr int kAxialMinCtas = KT >= 0 && KT <= 8 ? (kNorm ? 4 : 6) : 1;

// ---------------------------------------------------------------------------
// pass C with TMA-staged tiles.  The pass is bound by memory latency when
// each thread loads its column's rows one step at a time.  Here a CTA owns
// the tile of 256 consecutive bins of a plane (a chunk of the plane's J bins;
// the axial pass treats every bin alike) over the L planes of one segment:
// one thread issues L row copies (cp.async.bulk.tensor, 1 KB each) into
// shared memory at once, in groups of kTmaRows rows that complete on their
// own mbarrier, and every thread slides down its column in shared memory,
// waiting for a group only when its first row is needed.  Outputs, factors
// and arithmetic are those of axial_column (bit-identical results).
// grid (ceil(J / 256), segments); shared memory: the launch's longest segment, in KB.
// ---------------------------------------------------------------------------
constexpr int kTmaRows = 8;           // rows per mbarrier group
constexpr int kTmaMaxRings = 96;      // tiles of at most 96 rows (96 KB of shared memory)
constexpr int kTmaShortRows = 36;     // segments up to 36 planes: 6 CTAs of 36 KB tiles per SM
constexpr long kTmaSpinLimit = 1L << 24;  // a tile wait's bound, in polls: then the status word is set
constexpr long kTmaFaultSpins = 1L << 12;  // the injected wait's bound (tests)

__device__ __forceinline__ unsigned smem_u32(const void* q) { return (unsigned)__cvta_generic_to_shared(q); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_done(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// one box of the 2D map (x: bin in the plane, y: plane) into shared memory,
// completing on bar
__device__ __forceinline__ void tma_row(float* dst, const CUtensorMap* map, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// kFault (an instantiation for tests of the timeout path only): no copies are
// issued for a tile's first row group, whose wait runs out after
// kTmaFaultSpins polls; the other groups' copies run and are waited for.
// TW: the tile's width in bins, which is also the CTA's thread count.
template <int KT, bool kDivide, bool kNorm, bool kFault = false, int TW = kSmoothThreads>
__global__ void __launch_bounds__(TW, (kAxialMinCtas<KT, kNorm> * kSmoothThreads / TW))
    smooth_axial_tma_kernel(const __grid_constant__ FinParams P, const __grid_constant__ CUtensorMap map) {
  extern __shared__ __align__(128) float tile[];  // [L][TW]
  __shared__ __align__(8) unsigned long long bar[kTmaMaxRings / kTmaRows];
  constexpr int NB = 2;
  const int nr = P.n_rings;
  const int seg = P.seg0 + (int)blockIdx.y;
  const int d = seg - (nr - 1);  // ring difference rb - ra
  const int L = nr - abs(d);
  const long long p0 = (long long)max(0, -d) * (nr + 1) + d;
  const long long J = (long long)P.V * P.R * P.T;
  const int x0 = (int)blockIdx.x * TW;  // the chunk's first bin in a plane
  const int ng = (L + kTmaRows - 1) / kTmaRows;
  if (threadIdx.x == 0) {
    for (int g = 0; g < ng; ++g) mbar_init(&bar[g], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int g = 0; g < ng; ++g) {
      const int k0 = g * kTmaRows, k1 = min(L, k0 + kTmaRows);
      mbar_expect_tx(&bar[g], (unsigned)((k1 - k0) * TW * sizeof(float)));
      if (kFault && g == 0) continue;  // group 0 expects bytes no copy delivers
      for (int k = k0; k < k1; ++k) tma_row(tile + k * TW, &map, x0, (int)(p0 + (long long)k * (nr + 1)), &bar[g]);
    }
  }
  // groups known complete; a wait that runs out sets the status word, waits
  // once more (bounded) for the copies still in flight, and ends the thread
  int ready = 0;
  auto need = [&](int row) -> bool {
    const int g = row / kTmaRows;
    while (ready <= g) {
      long spins = 0;
      while (!mbar_done(&bar[ready], 0))
        if (++spins > (kFault ? kTmaFaultSpins : kTmaSpinLimit)) return false;
      ++ready;
    }
    return true;
  };
  auto give_up = [&]() {
    if (P.status) atomicExch(P.status, 1);
    for (int g = ready; g < ng; ++g) {
      if (kFault && g == 0) continue;  // nothing in flight there
      long spins = 0;
      while (!mbar_done(&bar[g], 0) && ++spins <= kTmaSpinLimit) {
      }
    }
  };
  const long long x = x0 + (long long)threadIdx.x;
  if (x >= J) {
    // a column past the plane's end (zero-filled by the copy): no output, but
    // the CTA's copies complete before any of its threads may end the CTA
    if (!need(L - 1)) give_up();
    return;
  }
  const long long bin0 = p0 * J + x;                   // bin of k = 0
  const long long bin_step = (long long)(nr + 1) * J;  // next plane of the segment
  const long long lors = (long long)P.V * P.R;
  const long long lor0 = p0 * lors + fdiv((unsigned)x, P.magic_T);  // x T < 2^32 (host check)
  const long long lor_step = (long long)(nr + 1) * lors;
#if PSC_DEBUG
  if (dbg_idx(P.dbg, kSiteFinColumn, bin0 + (L - 1) * bin_step, P.n_bins) != bin0 + (L - 1) * bin_step ||
      dbg_idx(P.dbg, kSiteFinLor, lor0 + (L - 1) * lor_step, P.n_bins / P.T) != lor0 + (L - 1) * lor_step) {
    if (!need(L - 1)) give_up();
    return;
  }
#endif
  const float* col = tile + threadIdx.x;  // row k at col[k * TW]
  const Weights& g = P.g[2];
  float w[2 * KT + NB];
  if (L >= KT) {
    if (KT > 0 && !need(KT - 1)) return give_up();
#pragma unroll
    for (int r = 0; r < KT; ++r) {  // row r, and row -1 - r reflected onto it
      const float v = col[r * TW];
      w[KT + r] = v;
      w[KT - 1 - r] = v;
    }
  } else {
    if (!need(L - 1)) return give_up();
#pragma unroll
    for (int j = 0; j < 2 * KT; ++j) w[j] = col[reflect(j - KT, L) * TW];
  }
  const bool use_sens = !P.sens_first && P.sens;
  const float cf = (float)P.c;
  const long long step2 = NB * bin_step;
  double* dst = P.out + bin0;
  const long long* ap = P.acc + bin0;
  const long long rs = P.norm_per_lor ? lor_step : bin_step, ss = P.sens_per_lor ? lor_step : bin_step;
  const double* rp = kNorm ? P.rnorm + (P.norm_per_lor ? lor0 : bin0) : nullptr;
  const double* sp = use_sens ? P.sens + (P.sens_per_lor ? lor0 : bin0) : nullptr;
  for (int o0 = 0; o0 < L; o0 += NB) {
    if (!need(min(o0 + KT + 1, L - 1))) return give_up();
    const int ra = o0 + KT < L ? o0 + KT : reflect(o0 + KT, L);
    const int rb = o0 + KT + 1 < L ? o0 + KT + 1 : reflect(o0 + KT + 1, L);
    w[2 * KT] = col[ra * TW];
    w[2 * KT + 1] = col[rb * TW];
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
    for (int j = 0; j <= 2 * KT; ++j) {
      s0 = fmaf(g[j], w[j], s0);
      s1 = fmaf(g[j], w[j + 1], s1);
    }
    const bool two = o0 + 1 < L;
    long long qa0 = 0, qa1 = 0;
    double fr0 = 1.0, fr1 = 1.0, fs0 = 1.0, fs1 = 1.0;
    if (kDivide) {
      qa0 = __ldg(ap);
      if (two) qa1 = __ldg(ap + bin_step);
      ap += step2;
    } else {
      if (kNorm) {
        fr0 = __ldg(rp);
        if (two) fr1 = __ldg(rp + rs);
        rp += NB * rs;
      }
      if (use_sens) {
        fs0 = __ldg(sp);
        if (two) fs1 = __ldg(sp + ss);
        sp += NB * ss;
      }
    }
    dst[0] = axial_epilogue<kDivide, kNorm>(s0, qa0, fr0, fs0, use_sens, cf);
    if (two) dst[bin_step] = axial_epilogue_fp64<kDivide, kNorm>(s1, qa1, fr1, fs1, use_sens, cf);
    dst += step2;
#pragma unroll
    for (int j = 0; j < 2 * KT; ++j) w[j] = w[NB + j];
  }
}


template <int KT, bool kDivide, bool kNorm>
__global__ void __launch_bounds__(kSmoothThreads, (kAxialMinCtas<KT, kNorm>)) smooth_axial_kernel(const __grid_constant__ FinParams P) {
  const int I = P.R * P.T;
  const int i = blockIdx.x * kSmoothThreads + threadIdx.x;
  if (i >= I) return;
  const int nr = P.n_rings;
  const int sl = blockIdx.y / P.V, v = blockIdx.y - sl * P.V;
  const int seg = P.seg0 + sl;
  const int d = seg - (nr - 1);  // ring difference rb - ra
  const int ra0 = max(0, -d);
  const int L = nr - abs(d);
  const long long J = (long long)P.V * I;
  const long long p0 = (long long)ra0 * (nr + 1) + d;
  const long long bin0 = p0 * J + (long long)v * I + i;       // bin of k = 0
  const long long bin_step = (long long)(nr + 1) * J;         // next plane of the segment
  const long long lors = (long long)P.V * P.R;
  const long long lor0 = p0 * lors + (long long)v * P.R + fdiv((unsigned)i, P.magic_T);
  const long long lor_step = (long long)(nr + 1) * lors;
#if PSC_DEBUG
  // the column's planes 0 .. L - 1 and their LORs
  if (dbg_idx(P.dbg, kSiteFinColumn, bin0 + (L - 1) * bin_step, P.n_bins) != bin0 + (L - 1) * bin_step ||
      dbg_idx(P.dbg, kSiteFinLor, lor0 + (L - 1) * lor_step, P.n_bins / P.T) != lor0 + (L - 1) * lor_step)
    return;
#endif
  if constexpr (KT >= 0) {
    axial_column<KT, kDivide, kNorm>(P, bin0, lor0, bin_step, lor_step, L);
  } else {
    // radii above the largest instantiated window: one load per tap
    constexpr int NB = kNb<KT>;
    const bool use_sens = !P.sens_first && P.sens;
    const float cf = (float)P.c;
    auto cvt = [](float x, int) { return x; };
    auto store = [&](int k0, const float (&o)[NB]) {
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        const int k = k0 + q;
        if (k >= L) break;
        const long long bin = bin0 + k * bin_step, lor = lor0 + k * lor_step;
        const long long qa = kDivide ? __ldg(P.acc + bin) : 0;
        const double fr = kNorm ? at(P.rnorm, P.norm_per_lor ? lor : bin) : 1.0;
        const double fs = use_sens && !kDivide ? at(P.sens, P.sens_per_lor ? lor : bin) : 1.0;
        P.out[bin] = axial_epilogue<kDivide, kNorm>(o[q], qa, fr, fs, use_sens, cf);
      }
    };
    slide_generic(P.scratch + bin0, bin_step, L, P.K[2], P.g[2], cvt, store);
  }
}

// reciprocal of a normalisation sinogram, 0 where it is 0: FP64 (r) and/or
// rounded to FP32 (r32)
__global__ void reciprocal_kernel(const double* __restrict__ a, double* __restrict__ r, float* __restrict__ r32,
                                  long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double v = a[i];
    const double x = v != 0.0 ? 1.0 / v : 0.0;
    if (r) r[i] = x;
    if (r32) r32[i] = f64_to_f32(x);
  }
}

// FP32 copy of a sinogram (round to nearest even)
__global__ void narrow_kernel(const double* __restrict__ a, float* __restrict__ b, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) b[i] = f64_to_f32(a[i]);
}

static int grid_for(long long n, int block, int sms) {
  long long g = (n + block - 1) / block;
  const long long cap = (long long)sms * 32;
  return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

cudaError_t launch_reciprocal(const double* a, double* r, float* r32, long long n, int sms, cudaStream_t s) {
  reciprocal_kernel<<<grid_for(n, 256, sms), 256, 0, s>>>(a, r, r32, n);
  return cudaGetLastError();
}

cudaError_t launch_narrow(const double* a, float* b, long long n, int sms, cudaStream_t s) {
  narrow_kernel<<<grid_for(n, 256, sms), 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host side: weights and window radii, launches
// ---------------------------------------------------------------------------
// instantiated window radii (ascending); larger K use the per-tap loop
constexpr int kWindowRadii[] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 16, 20, 24};

int finalize_plan(FinParams& p, const double sigma[3]) {
  if ((long long)p.n_rings * p.n_rings > 65535 || (2LL * p.n_rings - 1) * p.V > 65535)
    return psc_set_error(PSC_EINVAL, "smoothing supports at most 65535 planes and 65535 segment views");
  for (int ax = 0; ax < 3; ++ax) {
    const double sg = sigma[ax];
    if (!(sg >= 0.0) || !std::isfinite(sg)) return psc_set_error(PSC_EINVAL, "sigma[%d] must be finite and >= 0", ax);
    const int K = sg > 0.0 ? (int)std::ceil(4.0 * sg) : 0;
    if (K > kMaxSmoothRadius)
      return psc_set_error(PSC_EINVAL, "sigma[%d] too large (4 sigma > %d bins)", ax, kMaxSmoothRadius);
    double w[2 * kMaxSmoothRadius + 1], sum = 0.0;
    for (int k = -K; k <= K; ++k) {
      w[k + K] = K ? std::exp(-0.5 * (k / sg) * (k / sg)) : 1.0;
      sum += w[k + K];
    }
    int KT = -1;
    for (int r : kWindowRadii)
      if (r >= K) {
        KT = r;
        break;
      }
    const int c = KT >= 0 ? KT : K;  // centre of the stored weights
    p.K[ax] = K;
    p.KT[ax] = KT;
    for (int j = 0; j <= 2 * kMaxSmoothRadius; ++j) p.g[ax][j] = 0.0f;
    for (int k = -K; k <= K; ++k) p.g[ax][c + k] = (float)(w[k + K] / sum);
  }
  return PSC_OK;
}

template <template <int> class Launcher, int I = 0>
static cudaError_t dispatch_kt(int kt, const FinParams& p, dim3 grid, cudaStream_t s) {
  constexpr int n = (int)(sizeof(kWindowRadii) / sizeof(kWindowRadii[0]));
  if constexpr (I == n) {
    return Launcher<-1>::run(p, grid, s);
  } else {
    if (kt == kWindowRadii[I]) return Launcher<kWindowRadii[I]>::run(p, grid, s);
    return dispatch_kt<Launcher, I + 1>(kt, p, grid, s);
  }
}

#define PSC_LAUNCHER(NAME, KERNEL)                                          \
  template <int KT>                                                         \
  struct NAME {                                                             \
    static cudaError_t run(const FinParams& p, dim3 grid, cudaStream_t s) { \
      KERNEL<KT><<<grid, kSmoothThreads, 0, s>>>(p);                        \
      return cudaGetLastError();                                            \
    }                                                                       \
  };
PSC_LAUNCHER(RadialL, smooth_radial_kernel)
PSC_LAUNCHER(ViewL, smooth_view_kernel)
template <int KT>
struct AxialL {
  static cudaError_t run(const FinParams& p, dim3 grid, cudaStream_t s) {
    if (p.divide_acc) smooth_axial_kernel<KT, true, false><<<grid, kSmoothThreads, 0, s>>>(p);
    else if (p.rnorm) smooth_axial_kernel<KT, false, true><<<grid, kSmoothThreads, 0, s>>>(p);
    else smooth_axial_kernel<KT, false, false><<<grid, kSmoothThreads, 0, s>>>(p);
    return cudaGetLastError();
  }
};

cudaError_t launch_finalize_planes(const FinParams& p, int lo, int hi, int sms, cudaStream_t s) {
  if (hi <= lo) return cudaSuccess;
  const long long J = (long long)p.V * p.R * p.T;
  const long long n = hi - lo;
  const long long per_plane = std::max(1LL, std::min((J + 255) / 256, 8LL * sms / n + 1));
  FinParams q = p;
  q.plane0 = lo;
  finalize_plain_kernel<<<dim3((unsigned)per_plane, (unsigned)n), 256, 0, s>>>(q);
  return cudaGetLastError();
}

static unsigned smooth_blocks(long long n) { return (unsigned)((n + kSmoothThreads - 1) / kSmoothThreads); }

int finalize_planes(const FinParams& p) {
  if (p.seg_hi <= p.seg_lo) return p.n_rings * p.n_rings;
  int n = 0;
  for (int sg = p.seg_lo; sg < p.seg_hi; ++sg) n += p.n_rings - std::abs(sg - (p.n_rings - 1));
  return n;
}

cudaError_t launch_smooth_front(const FinParams& p, cudaStream_t s) {
  cudaError_t e;
  const unsigned planes = (unsigned)finalize_planes(p);
  const long long I = (long long)p.R * p.T;
  if ((e = dispatch_kt<RadialL>(p.KT[0], p, dim3(smooth_blocks((long long)p.V * p.T), planes), s)) != cudaSuccess)
    return e;
  return dispatch_kt<ViewL>(p.KT[1], p, dim3(smooth_blocks(I), planes), s);
}

// the driver's tensor-map encoder, looked up once (no link against libcuda)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// The TMA-staged axial pass applies when the FP32 working sinogram can be
// described as a 2D tensor of n^2 planes of J bins (16-byte aligned base,
// plane pitch J * 4 a multiple of 16 bytes), segments fit the shared-memory
// tile (n_rings <= kTmaMaxRings), the window radius is instantiated, x T <
// 2^32 for every bin x of a plane (exact LOR by multiply-high), and the
// environment does not switch it off (PSC_AXIAL_TMA=0).  The map describes
// 256-bin by 1-plane boxes.
static bool axial_tma_map(const FinParams& p, CUtensorMap* map, int tw) {
  const char* env = std::getenv("PSC_AXIAL_TMA");
  if (env && env[0] == '0') return false;
  const long long J = (long long)p.V * p.R * p.T;
  if (p.KT[2] < 0 || p.n_rings > kTmaMaxRings || J % 4 != 0 || J * p.T >= (1LL << 32) ||
      ((uintptr_t)p.scratch & 15) != 0)
    return false;
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)J, (cuuint64_t)p.n_rings * (cuuint64_t)p.n_rings};
  const cuuint64_t strides[1] = {(cuuint64_t)J * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)tw, 1};
  const cuuint32_t elem[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p.scratch, dims, strides, box, elem,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KT, bool kDivide, bool kNorm, bool kFault = false, int TW = kSmoothThreads>
static cudaError_t run_axial_tma(const FinParams& p, const CUtensorMap& map, dim3 grid, int rows, cudaStream_t s) {
  const size_t smem = (size_t)rows * TW * sizeof(float);
  auto k = smooth_axial_tma_kernel<KT, kDivide, kNorm, kFault, TW>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, TW, smem, s>>>(p, map);
  return cudaGetLastError();
}

template <int I = 0, class F>
static cudaError_t for_window_radius(int kt, F&& f) {
  constexpr int n = (int)(sizeof(kWindowRadii) / sizeof(kWindowRadii[0]));
  if constexpr (I == n) {
    return cudaErrorInvalidValue;
  } else {
    if (kt == kWindowRadii[I]) return f(std::integral_constant<int, kWindowRadii[I]>{});
    return for_window_radius<I + 1>(kt, f);
  }
}

cudaError_t launch_smooth_axial(const FinParams& p, int lo, int hi, cudaStream_t s) {
  if (hi <= lo) return cudaSuccess;
  FinParams q = p;
  q.seg0 = lo;
  CUtensorMap map, map_narrow;
  if (axial_tma_map(p, &map, kSmoothThreads) && axial_tma_map(p, &map_narrow, kSmoothThreads / 2)) {
    // every tile wait is bounded; PSC_FAULT_TMA_WAIT=1 (tests of the timeout
    // path) runs the kFault instantiation where there is one (window radius
    // 8, no normalisation, not the normalisation sinogram)
    const char* inj = std::getenv("PSC_FAULT_TMA_WAIT");
    const bool fault = inj && inj[0] == '1' && p.KT[2] == 8 && !p.divide_acc && !p.rnorm;
    // segments of at most kTmaShortRows planes in launches of their own,
    // whose smaller tiles let 6 CTAs share an SM's shared memory; the long
    // middle segments run tiles half as wide (128 bins, half the shared
    // memory per CTA) in CTAs of 128 threads
    const int n = p.n_rings, S = std::min(kTmaShortRows, n);
    const int c1 = std::max(lo, std::min(hi, S)), c2 = std::max(c1, std::min(hi, 2 * n - 1 - S));
    const int cuts[4] = {lo, c1, c2, hi};
    const long long J = (long long)p.V * p.R * p.T;
    for (int r = 0; r < 3; ++r) {
      const int a = cuts[r], b = cuts[r + 1];
      if (b <= a) continue;
      int rows = 0;  // the longest segment of [a, b)
      for (int sg = a; sg < b; ++sg) rows = std::max(rows, n - std::abs(sg - (n - 1)));
      q.seg0 = a;
      const bool narrow = rows > kTmaShortRows;
      constexpr int kNarrow = kSmoothThreads / 2;
      const dim3 grid((unsigned)((J + (narrow ? kNarrow : kSmoothThreads) - 1) / (narrow ? kNarrow : kSmoothThreads)),
                      (unsigned)(b - a));
      const cudaError_t e = for_window_radius(p.KT[2], [&](auto kt) -> cudaError_t {
        constexpr int KT = decltype(kt)::value;
        if constexpr (KT == 8)
          if (fault)
            return narrow ? run_axial_tma<KT, false, false, true, kNarrow>(q, map_narrow, grid, rows, s)
                          : run_axial_tma<KT, false, false, true>(q, map, grid, rows, s);
        if (narrow) {
          if (p.divide_acc) return run_axial_tma<KT, true, false, false, kNarrow>(q, map_narrow, grid, rows, s);
          if (p.rnorm) return run_axial_tma<KT, false, true, false, kNarrow>(q, map_narrow, grid, rows, s);
          return run_axial_tma<KT, false, false, false, kNarrow>(q, map_narrow, grid, rows, s);
        }
        if (p.divide_acc) return run_axial_tma<KT, true, false>(q, map, grid, rows, s);
        if (p.rnorm) return run_axial_tma<KT, false, true>(q, map, grid, rows, s);
        return run_axial_tma<KT, false, false>(q, map, grid, rows, s);
      });
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  return dispatch_kt<AxialL>(p.KT[2], q, dim3(smooth_blocks((long long)p.R * p.T), (unsigned)((hi - lo) * p.V)), s);
}

cudaError_t launch_finalize(const FinParams& p, int sms, cudaStream_t s) {
  if (!p.smooth) return launch_finalize_planes(p, 0, finalize_planes(p), sms, s);
  cudaError_t e;
  if ((e = launch_smooth_front(p, s)) != cudaSuccess) return e;
  const bool all = p.seg_hi <= p.seg_lo;
  return launch_smooth_axial(p, all ? 0 : p.seg_lo, all ? 2 * p.n_rings - 1 : p.seg_hi, s);
}

}  // namespace psc
