// postproc.cu -- post-processing of int64 fixed-point sinograms: mashing of
// views and TOF bins (Sec. 4 names it as a way to need fewer counts and less
// smoothing time) and the sum over the scanner's rotational symmetries
// (Sec. 2.2.4 averages the sensitivity sinograms over them).  Both are exact
// integer sums, so their results do not depend on summation order.
//
// Layout of a sinogram: [plane = ring_a * n_rings + ring_b][view][rad][tof],
// with the integer LOR formula of the binning: for crystals a < b, f = a + b
// (f -= n and s = -1 when f >= n, else s = +1), view = f >> 1, radial
// s (n/2 - (b - a)) + n/2 - 1 less the centred clip offset.
#include <algorithm>

#include "psc_internal.h"

namespace psc {

namespace {

// out[p][v / vf][r][t / tf] = sum of the vf x tf block; grid (ceil(R T2 /
// 256), V2, planes)
__global__ void mash_kernel(const long long* __restrict__ in, long long* __restrict__ out, int V, int R, int T,
                            int vf, int tf) {
  const int V2 = V / vf, T2 = T / tf;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R * T2) return;
  const int r = c / T2, t2 = c - r * T2;
  const long long p = blockIdx.z;
  const int v2 = blockIdx.y;
  const long long* row0 = in + ((p * V + (long long)v2 * vf) * R + r) * T + (long long)t2 * tf;
  const long long vstride = (long long)R * T;
  long long sum = 0;
  if (tf == 1 && vf <= 8) {  // all loads of the block in flight at once
    long long x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = j < vf ? __ldg(row0 + j * vstride) : 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) sum += x[j];
  } else {
    for (int j = 0; j < vf; ++j)
      for (int u = 0; u < tf; ++u) sum += __ldg(row0 + j * vstride + u);
  }
  out[((p * V2 + v2) * R + r) * T2 + t2] = sum;
}

// the crystal pair a < b of (view, unclipped radial index): the inverse of
// the binning's LOR formula (one of s = +1, -1 gives a valid pair)
__device__ __forceinline__ void lor_crystals(int n, int v, int r_full, int& a, int& b) {
  const int q = r_full - n / 2 + 1;
  a = b = -1;
#pragma unroll
  for (int si = 0; si < 2; ++si) {
    const int s = si ? -1 : 1;
    const int d = n / 2 - s * q;
    if (d < 1 || d > n - 1) continue;
    const int f = 2 * v + (d & 1) + (s < 0 ? n : 0);  // a + b
    const int a2 = f - d;
    if (a2 < 0 || (a2 & 1)) continue;
    const int lo = a2 >> 1, hi = (f + d) >> 1;
    if (lo < hi && hi < n && a < 0) {
      a = lo;
      b = hi;
    }
  }
}

// out[bin] = sum over the n / step rotations by k * step crystals of in at
// the rotated LOR: (a + c, b + c) mod n; when the order reverses, the ring
// indices swap and the TOF bin mirrors.  grid (ceil(R T / 256), V, planes)
__global__ void rotate_sum_kernel(const long long* __restrict__ in, long long* __restrict__ out, int n,
                                  int n_rings, int R, int T, int step) {
  const int V = n / 2;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R * T) return;
  const int r = c / T, t = c - r * T;
  const int v = blockIdx.y;
  const int p = blockIdx.z;
  const int ra = p / n_rings, rb = p - ra * n_rings;
  const int rad_off = (n - 1 - R) / 2;
  int a, b;
  lor_crystals(n, v, r + rad_off, a, b);
  long long sum = 0;
  int a2 = a, b2 = b;  // (a + k step, b + k step) mod n, kept below n by one subtraction
  for (int k = 0; k < n / step; ++k, a2 += step, b2 += step) {
    if (a2 >= n) a2 -= n;
    if (b2 >= n) b2 -= n;
    const bool flip = a2 > b2;
    const int lo = flip ? b2 : a2, hi = flip ? a2 : b2;
    int f = lo + hi, s = 1;
    if (f >= n) {
      f -= n;
      s = -1;
    }
    const int v2 = f >> 1;
    const int r2 = s * (n / 2 - (hi - lo)) + n / 2 - 1 - rad_off;
    const long long p2 = flip ? (long long)rb * n_rings + ra : p;
    const int t2 = flip ? T - 1 - t : t;
    sum += __ldg(in + ((p2 * V + v2) * R + r2) * T + t2);
  }
  out[(((long long)p * V + v) * R + r) * T + t] = sum;
}

// bin index of the LOR (a + c, b + c) mod n of plane (ra, rb) and TOF bin t:
// when the order reverses, the rings swap and the TOF bin mirrors
__device__ __forceinline__ long long rotated_bin(int n, int n_rings, int R, int T, int rad_off, int a2, int b2,
                                                 int ra, int rb, int t) {
  const bool flip = a2 > b2;
  const int lo = flip ? b2 : a2, hi = flip ? a2 : b2;
  int f = lo + hi, s = 1;
  if (f >= n) {
    f -= n;
    s = -1;
  }
  const int v2 = f >> 1;
  const int r2 = s * (n / 2 - (hi - lo)) + n / 2 - 1 - rad_off;
  const long long p2 = flip ? (long long)rb * n_rings + ra : (long long)ra * n_rings + rb;
  const int t2 = flip ? T - 1 - t : t;
  return ((p2 * (n / 2) + v2) * R + r2) * T + t2;
}

// The same sum, one orbit at a time, for n / step even.  A rotation by
// step crystals moves an LOR by step views, so every orbit has members in
// views [0, step): an LOR x and its half-turn partner (rotation by n / 2
// crystals).  The one of the two with the lower bin index sums the input
// over the n / step rotations of x and writes that sum to every member of
// the orbit (the sum is the same for all of them): one read and one write
// per bin.  grid (ceil(R T / 256), step, planes)
__global__ void rotate_orbit_kernel(const long long* __restrict__ in, long long* __restrict__ out, int n,
                                    int n_rings, int R, int T, int step) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R * T) return;
  const int r = c / T, t = c - r * T;
  const int v = blockIdx.y;
  const int p = blockIdx.z;
  const int ra = p / n_rings, rb = p - ra * n_rings;
  const int rad_off = (n - 1 - R) / 2;
  int a, b;
  lor_crystals(n, v, r + rad_off, a, b);
  const int h = n / 2;
  const long long self = (((long long)p * h + v) * R + r) * T + t;
  const long long partner =
      rotated_bin(n, n_rings, R, T, rad_off, a + h >= n ? a + h - n : a + h, b + h >= n ? b + h - n : b + h, ra, rb, t);
  if (partner < self) return;
  long long sum = 0;
  int a2 = a, b2 = b;
  for (int k = 0; k < n / step; ++k, a2 += step, b2 += step) {
    if (a2 >= n) a2 -= n;
    if (b2 >= n) b2 -= n;
    sum += __ldg(in + rotated_bin(n, n_rings, R, T, rad_off, a2, b2, ra, rb, t));
  }
  a2 = a;
  b2 = b;
  for (int k = 0; k < n / step; ++k, a2 += step, b2 += step) {
    if (a2 >= n) a2 -= n;
    if (b2 >= n) b2 -= n;
    out[rotated_bin(n, n_rings, R, T, rad_off, a2, b2, ra, rb, t)] = sum;
  }
}

// Span mashing: the segment of span-mashed output plane o, and its axial sum
// z = ra + rb.  Segment k (k = -K..K) holds the ring differences
// [k span - h, k span + h] (h = (span - 1) / 2) within the ring range, and
// the axial sums from its smallest |d| to 2 n - 2 minus it (every other one
// when it holds a single ring difference); output planes run over the
// segments in order, each by z ascending.
struct SpanPlane {
  int d_lo, d_hi, z;
};

__host__ __device__ inline int span_count(int n, int span, int k, int& d_lo, int& d_hi, int& m, int& step) {
  const int h = (span - 1) / 2;
  d_lo = max(k * span - h, -(n - 1));
  d_hi = min(k * span + h, n - 1);
  m = (d_lo <= 0 && 0 <= d_hi) ? 0 : min(abs(d_lo), abs(d_hi));
  step = d_hi > d_lo ? 1 : 2;
  return (2 * n - 2 - 2 * m) / step + 1;
}

__device__ inline SpanPlane span_plane(int n, int span, int o) {
  const int K = (n - 1 + (span - 1) / 2) / span;
  int d_lo = 0, d_hi = 0, m = 0, step = 1;
  for (int k = -K; k <= K; ++k) {
    const int c = span_count(n, span, k, d_lo, d_hi, m, step);
    if (o < c || k == K) break;
    o -= c;
  }
  return SpanPlane{d_lo, d_hi, m + o * step};
}

// grid (column blocks, output planes): each output bin sums the input planes
// (ra, rb) of its segment with ra + rb = z, read once each (exact int64)
__global__ void __launch_bounds__(256) span_kernel(const long long* __restrict__ in, long long* __restrict__ out,
                                                   int n, int span, long long J) {
  const SpanPlane sp = span_plane(n, span, (int)blockIdx.y);
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < J; j += (long long)gridDim.x * blockDim.x) {
    long long sum = 0;
    for (int d = sp.d_lo; d <= sp.d_hi; ++d) {
      if ((sp.z + d) & 1) continue;
      const int ra = (sp.z - d) / 2, rb = (sp.z + d) / 2;
      if (ra >= 0 && ra < n && rb >= 0 && rb < n) sum += __ldg(in + (long long)(ra * n + rb) * J + j);
    }
    out[(long long)blockIdx.y * J + j] = sum;
  }
}

}  // namespace

int span_planes(int n_rings, int span) {
  const int K = (n_rings - 1 + (span - 1) / 2) / span;
  int total = 0, d_lo, d_hi, m, step;
  for (int k = -K; k <= K; ++k) total += span_count(n_rings, span, k, d_lo, d_hi, m, step);
  return total;
}

cudaError_t launch_span(const long long* in, long long* out, int n_rings, int span, long long J, int sms,
                        cudaStream_t s) {
  const int planes = span_planes(n_rings, span);
  const long long per = std::max(1LL, std::min((J + 255) / 256, 8LL * sms / planes + 1));
  span_kernel<<<dim3((unsigned)per, (unsigned)planes), 256, 0, s>>>(in, out, n_rings, span, J);
  return cudaGetLastError();
}

cudaError_t launch_mash(const long long* in, long long* out, int planes, int V, int R, int T, int vf, int tf,
                        cudaStream_t s) {
  const int cols = R * (T / tf);
  mash_kernel<<<dim3((cols + 255) / 256, V / vf, planes), 256, 0, s>>>(in, out, V, R, T, vf, tf);
  return cudaGetLastError();
}

cudaError_t launch_rotate_sum(const long long* in, long long* out, int n_crystals, int n_rings, int R, int T,
                              int step, cudaStream_t s) {
  if ((n_crystals / step) % 2 == 0)
    rotate_orbit_kernel<<<dim3((R * T + 255) / 256, step, n_rings * n_rings), 256, 0, s>>>(in, out, n_crystals,
                                                                                          n_rings, R, T, step);
  else
    rotate_sum_kernel<<<dim3((R * T + 255) / 256, n_crystals / 2, n_rings * n_rings), 256, 0, s>>>(
        in, out, n_crystals, n_rings, R, T, step);
  return cudaGetLastError();
}

}  // namespace psc
