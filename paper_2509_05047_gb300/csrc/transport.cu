// transport.cu -- fused emission -> Woodcock transport -> detection -> LUT
// weight -> LOR/TOF binning kernel (Sec. 2.2.1-2.2.3 of the paper; the
// simulator itself is the project's own design).
//
// One thread owns one history at a time (grid-stride over the history
// range).  Material cross sections and the Woodcock majorant are staged in
// shared memory; voxels, alias table and LUT are read through the read-only
// path from L2.  A history either adds one fixed-point weight to the int64
// accumulator or nothing (Sec. 2.2.3: events are weighted or discarded,
// never duplicated).  Integer atomics make the sinogram independent of
// launch shape and history order.
#include "psc_internal.h"

namespace psc {

struct Photon {
  float3 pos, dir;
  float e, path;
  int n_c, n_r, n_steps;
  Hit hit;
};

struct Counters {
  unsigned int cls[8];
  unsigned int steps, compton, rayleigh, photo, binned, rng, tries, detected;
  unsigned long long weight;
};

__device__ __forceinline__ float interp_scalar(const float* t, int n_tab, int e0, float e) {
  const float fe = e - (float)e0;
  const int i = max(0, min((int)fe, n_tab - 2));
  const float f = fe - (float)i;
  const float a = t[i], b = t[i + 1];
  return a + f * (b - a);
}

__device__ __forceinline__ float4 interp_xs(const float4* t, int n_tab, int e0, float e) {
  const float fe = e - (float)e0;
  const int i = max(0, min((int)fe, n_tab - 2));
  const float f = fe - (float)i;
  const float4 a = t[i], b = t[i + 1];
  return make_float4(a.x + f * (b.x - a.x), a.y + f * (b.y - a.y), a.z + f * (b.z - a.z), 0.0f);
}

// Woodcock delta tracking of one photon, then detection.
__device__ __forceinline__ void track(const SimParams& P, const float4* s_xs, const float* s_maj,
                                      const float* s_kappa, Rng& rng, Photon& p, Counters& cnt) {
  const PhantomParams& ph = P.ph;
  for (;;) {
    if (p.n_steps >= kMaxSteps) {
      p.hit.status = kStepLimit;
      return;
    }
    const float mu_max = interp_scalar(s_maj, ph.n_tab, ph.e0, p.e);
    if (!(mu_max > 0.0f)) break;
    const float dist = -logf(rng.next()) / mu_max;
    const float qx = p.pos.x + dist * p.dir.x;
    const float qy = p.pos.y + dist * p.dir.y;
    const float qz = p.pos.z + dist * p.dir.z;
    const float fx = (qx - ph.ox) * ph.inv_dx;
    const float fy = (qy - ph.oy) * ph.inv_dy;
    const float fz = (qz - ph.oz) * ph.inv_dz;
    if (!(fx >= 0.0f && fx < (float)ph.nx && fy >= 0.0f && fy < (float)ph.ny && fz >= 0.0f &&
          fz < (float)ph.nz))
      break;  // outside the grid is vacuum: straight to the detector
    const int ix = min((int)fx, ph.nx - 1);
    const int iy = min((int)fy, ph.ny - 1);
    const int iz = min((int)fz, ph.nz - 1);
    p.pos = make_float3(qx, qy, qz);
    p.path += dist;
    ++p.n_steps;
    ++cnt.steps;
    const float2 vx = __ldg(ph.vox + ((long long)iz * ph.ny + iy) * ph.nx + ix);
    const float rho = vx.x;
    const int m = __float_as_int(vx.y);
    const float4 cum = interp_xs(s_xs + m * ph.n_tab, ph.n_tab, ph.e0, p.e);
    const float t = rng.next() * mu_max;
    if (t < rho * cum.x) {  // Compton
      float x, c;
      cnt.tries += sample_compton(rng, p.e, x, c);
      rotate(p.dir, c, rng.next());
      p.e = p.e / x;
      ++p.n_c;
      ++cnt.compton;
      if (p.e < P.sc.e_lo) {
        p.hit.status = kEnergyWindow;
        return;
      }
    } else if (t < rho * cum.y) {  // Rayleigh
      int tries;
      const float c = sample_rayleigh(rng, p.e, s_kappa[m], tries);
      cnt.tries += tries;
      rotate(p.dir, c, rng.next());
      ++p.n_r;
      ++cnt.rayleigh;
    } else if (t < rho * cum.z) {  // photo-absorption
      ++cnt.photo;
      p.hit.status = kAbsorbed;
      return;
    }  // else virtual collision
  }
  p.hit = detect(P.sc, p.pos, p.dir, p.e);
  p.path += p.hit.dist;
}

__device__ __forceinline__ long long bin_key(const ScannerParams& S, int ca, int cb, int ra, int rb,
                                             float delta) {
  const int N = S.n_crystals;
  int f = ca + cb, s = 1;
  if (f >= N) {
    f -= N;
    s = -1;
  }
  const int view = f >> 1;
  const int r = s * (N / 2 - (cb - ca)) + N / 2 - 1 - S.rad_off;
  if (r < 0 || r >= S.n_rad) return -1;
  const float g = floorf(delta * S.inv_tof_bin + S.tof_half);
  if (!(g >= 0.0f && g < (float)S.n_tof)) return -1;
  const int plane = ra * S.n_rings + rb;
  return (((long long)plane * S.n_views + view) * S.n_rad + r) * S.n_tof + (int)g;
}

template <int DT>
__device__ __forceinline__ void run_history(const SimParams& P, const float4* s_xs,
                                            const float* s_maj, const float* s_kappa,
                                            unsigned long long h, Counters& cnt, int& cls,
                                            long long& key, long long& q) {
  const PhantomParams& ph = P.ph;
  key = -1;
  q = 0;
  // emission (stream 0, blocks 0 and 1)
  const uint4 b0 = philox_block(P.seed, h, 0, 0);
  const uint4 b1 = philox_block(P.seed, h, 1, 0);
  const long long col = (long long)(((unsigned long long)b0.x * (unsigned long long)ph.n_vox) >> 32);
  const double pr = __ldg(ph.alias_prob + col);
  const int v = ((double)u01(b0.y) < pr) ? (int)col : __ldg(ph.alias_idx + col);
  const int ix = v % ph.nx, iy = (v / ph.nx) % ph.ny, iz = v / (ph.nx * ph.ny);
  const float3 e0 = make_float3(ph.ox + ((float)ix + u01(b0.z)) * ph.dx,
                                ph.oy + ((float)iy + u01(b0.w)) * ph.dy,
                                ph.oz + ((float)iz + u01(b1.x)) * ph.dz);
  const float ct = 2.0f * u01(b1.y) - 1.0f;
  float sp, cp;
  sincospif(2.0f * u01(b1.z), &sp, &cp);
  const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
  const float3 d = make_float3(st * cp, st * sp, ct);

  Photon A, B;
  A.pos = e0;
  A.dir = d;
  A.e = kEmitKeV;
  A.path = 0.0f;
  A.n_c = A.n_r = A.n_steps = 0;
  Rng rng;
  rng.init(P.seed, h, 1);
  track(P, s_xs, s_maj, s_kappa, rng, A, cnt);
  cnt.rng += 2 + rng.block;
  if (A.hit.status != kDetected) {
    cls = A.hit.status;
    return;
  }
  B.pos = e0;
  B.dir = make_float3(-d.x, -d.y, -d.z);
  B.e = kEmitKeV;
  B.path = 0.0f;
  B.n_c = B.n_r = B.n_steps = 0;
  rng.init(P.seed, h, 2);
  ++cnt.detected;  // photon A
  track(P, s_xs, s_maj, s_kappa, rng, B, cnt);
  cnt.rng += rng.block;
  if (B.hit.status != kDetected) {
    cls = B.hit.status;
    return;
  }
  ++cnt.detected;  // photon B
  if (A.hit.crystal == B.hit.crystal) {
    cls = kSameCrystal;
    return;
  }
  const bool a_first = A.hit.crystal < B.hit.crystal;
  const Photon& pa = a_first ? A : B;
  const Photon& pb = a_first ? B : A;
  float delta = 0.5f * (pa.path - pb.path);
  if (P.sc.tof_sigma > 0.0f) {  // Gaussian TOF blur (stream 0, block 2), Box-Muller
    const uint4 b2 = philox_block(P.seed, h, 2, 0);
    ++cnt.rng;
    const float g = sqrtf(-2.0f * logf(u01(b2.x))) * cospif(2.0f * u01(b2.y));
    delta += P.sc.tof_sigma * g;
  }
  key = bin_key(P.sc, pa.hit.crystal, pb.hit.crystal, pa.hit.ring, pb.hit.ring, delta);
  if (key < 0) {
    cls = kOutOfRange;
    return;
  }
  const bool scattered = (A.n_c + A.n_r + B.n_c + B.n_r) > 0;
  cls = scattered ? kScatter : kTrue;
  const bool take = scattered ? (P.bin_mask & 1) : (P.bin_mask & 2);
  if (!take && P.q_out == nullptr) return;
  const float w =
      lut_prob<DT>(P.lut, A.e, A.hit.alpha, A.hit.beta,
                   A.hit.crystal % P.sc.module_t, A.hit.ring % P.sc.module_a) *
      lut_prob<DT>(P.lut, B.e, B.hit.alpha, B.hit.beta, B.hit.crystal % P.sc.module_t,
                   B.hit.ring % P.sc.module_a);
  q = __float2ll_rn(w * 4294967296.0f);
  if (take) {
    atomicAdd(P.acc + key, (unsigned long long)q);
    ++cnt.binned;
    cnt.weight += (unsigned long long)q;
  }
}

template <int DT>
__global__ void __launch_bounds__(256) transport_kernel(const __grid_constant__ SimParams P) {
  extern __shared__ float4 smem[];
  const int n_xs = P.ph.n_mat * P.ph.n_tab;
  float4* s_xs = smem;
  float* s_maj = reinterpret_cast<float*>(smem + n_xs);
  float* s_kappa = s_maj + P.ph.n_tab;
  for (int i = threadIdx.x; i < n_xs; i += blockDim.x) {
    const int m = i / P.ph.n_tab, k = i - m * P.ph.n_tab;
    s_xs[i] = P.ph.xs[m * P.ph.n_e + P.ph.e0 + k];
  }
  for (int i = threadIdx.x; i < P.ph.n_tab; i += blockDim.x) s_maj[i] = P.ph.maj[P.ph.e0 + i];
  if (threadIdx.x < kMaxMaterials)
    s_kappa[threadIdx.x] = threadIdx.x < P.ph.n_mat ? P.ph.kappa[threadIdx.x] : 0.0f;
  __syncthreads();

  Counters cnt = {};
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.n;
       i += stride) {
    int cls;
    long long key, q;
    run_history<DT>(P, s_xs, s_maj, s_kappa, P.first + i, cnt, cls, key, q);
#pragma unroll
    for (int k = 0; k < 8; ++k) cnt.cls[k] += (cls == k) ? 1u : 0u;
    if (P.cls_out) P.cls_out[i] = (int8_t)cls;
    if (P.key_out) P.key_out[i] = key;
    if (P.q_out) P.q_out[i] = q;
  }

  if (P.stats == nullptr) return;
  // warp-reduce the counters, one atomic per warp and counter
  unsigned long long vals[kStatCount] = {};
#pragma unroll
  for (int k = 0; k < 8; ++k) vals[k] = cnt.cls[k];
  vals[kStatSteps] = cnt.steps;
  vals[kStatCompton] = cnt.compton;
  vals[kStatRayleigh] = cnt.rayleigh;
  vals[kStatPhoto] = cnt.photo;
  vals[kStatBinned] = cnt.binned;
  vals[kStatWeight] = cnt.weight;
  vals[kStatRng] = cnt.rng;
  vals[kStatTries] = cnt.tries;
  vals[kStatDetected] = cnt.detected;
#pragma unroll
  for (int k = 0; k < kStatCount; ++k) {
    unsigned long long x = vals[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(P.stats + k, x);
  }
}

size_t transport_smem_bytes(const SimParams& p) {
  return sizeof(float4) * (size_t)p.ph.n_mat * p.ph.n_tab + sizeof(float) * (p.ph.n_tab + kMaxMaterials);
}

template <int DT>
static cudaError_t launch_dt(const SimParams& p, int grid, int block, cudaStream_t s) {
  const size_t smem = transport_smem_bytes(p);
  cudaError_t e = cudaFuncSetAttribute(transport_kernel<DT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  transport_kernel<DT><<<grid, block, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_transport(const SimParams& p, int grid, int block, cudaStream_t s) {
  switch (p.lut.dtype) {
    case 0: return launch_dt<0>(p, grid, block, s);
    case 1: return launch_dt<1>(p, grid, block, s);
    case 2: return launch_dt<2>(p, grid, block, s);
    default: return launch_dt<-1>(p, grid, block, s);
  }
}

cudaError_t transport_occupancy(int lut_dtype, int block, size_t smem, int* blocks_per_sm) {
  switch (lut_dtype) {
    case 0: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, transport_kernel<0>, block, smem);
    case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, transport_kernel<1>, block, smem);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, transport_kernel<2>, block, smem);
    default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, transport_kernel<-1>, block, smem);
  }
}

}  // namespace psc
