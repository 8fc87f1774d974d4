// psc_device.cuh -- device-side parameter blocks and the per-photon
// arithmetic of the scatter Monte Carlo path (sm_103a).
//
// Shared by the transport and finalize translation units of libpsc only.
// Everything here is FP32 transport arithmetic (FP64 only for the alias
// probabilities and the sinogram post-processing), written for the GPU.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "psc.h"

#ifndef PSC_DEBUG
#define PSC_DEBUG 0
#endif

namespace psc {

// ---------------------------------------------------------------------------
// Bounds-checked debug build (PSC_DEBUG=1; libpsc_debug.so).  Every indexed
// access on the hot path passes its index through dbg_idx: an index outside
// [0, bound) is recorded (the first one in full, all of them counted) and
// replaced by 0, so the access stays inside its array, the kernel finishes,
// and the host call that launched it fails with PSC_EDEVICE naming the site.
// Release builds compile the checks out.
// ---------------------------------------------------------------------------
enum : unsigned {
  kSiteSelfTest = 0, kSiteAlias = 1, kSiteVoxel = 2, kSiteMaterial = 3, kSiteKappa = 4, kSiteLut = 5,
  kSiteAcc = 6, kSiteHistOut = 7, kSiteSlot = 8, kSiteFinBin = 9, kSiteFinLor = 10, kSiteFinColumn = 11
};

struct DebugRecord {
  unsigned long long count;    // violations seen
  unsigned long long index, bound;
  unsigned site, pad;
};

__device__ __forceinline__ long long dbg_idx(DebugRecord* rec, unsigned site, long long i, long long bound) {
#if PSC_DEBUG
  if ((unsigned long long)i >= (unsigned long long)bound) {
    if (rec && atomicAdd(&rec->count, 1ull) == 0ull) {
      rec->site = site;
      rec->index = (unsigned long long)i;
      rec->bound = (unsigned long long)bound;
    }
    return 0;
  }
#else
  (void)rec;
  (void)site;
  (void)bound;
#endif
  return i;
}

constexpr int kMaxMaterials = 8;
constexpr int kMaxSteps = 4096;     // Woodcock steps per photon (safety bound)
constexpr int kMaxTries = 64;       // rejection-sampling tries, last proposal kept
constexpr int kRingWords = 8;       // per-lane window of the current Philox sub-stream
constexpr float kPolarEps = 1e-6f;  // |d_z| > 1 - eps: rotate about the z axis
constexpr float kRestKeV = 511.0f;
constexpr float kEmitKeV = 511.0f;
constexpr int kMaxSmoothRadius = 64;

enum : int {
  kAbsorbed = 0, kLostAxial = 1, kEnergyWindow = 2, kStepLimit = 3,
  kSameCrystal = 4, kOutOfRange = 5, kTrue = 6, kScatter = 7, kDetected = 15
};

// statistics slots (psc_stats order)
enum : int {
  kStatClass0 = 0, kStatSteps = 8, kStatCompton = 9, kStatRayleigh = 10, kStatPhoto = 11,
  kStatBinned = 12, kStatWeight = 13, kStatRng = 14, kStatTries = 15, kStatDetected = 16,
  kStatAtomics = 17, kStatCount = 18
};

struct ScannerParams {
  float radius, r2, half_len, inv_pitch;
  float e_lo, e_hi;
  float e_res_k;               // energy resolution: sigma(E) = e_res_k sqrt(E) (keV); 0 = exact
  float e_kill;                // a Compton photon below this energy cannot be detected
  float crystals_per_radian;   // N / (2 pi)
  float inv_tof_bin, tof_half, tof_sigma;
  int n_crystals, n_rings, module_t, module_a, n_tof, n_rad, n_views, rad_off;
  // gaps between modules and blocks (gap_mode 0: none, 1: lost, 2: edge assignment)
  int gap_mode, n_mod, n_blk;
  float mod_phi, inv_mod_phi, gap_gamma, inv_crys_phi;  // module pitch, gap (rad), 1 / crystal width
  float blk_pitch, inv_blk_pitch, gap_a, inv_ring_w;    // block pitch, axial gap (mm), 1 / ring width
  float gap_t_mm, depth, doi, mu;                       // edge-assignment geometry (mm, 1/mm)
  int escape_words;  // words of the photon's stream that detection reads: energy blur 2, edge draws 2
};

struct PhantomParams {
  int nx, ny, nz;
  int n_mat, n_e;              // tables hold nodes E = 0 .. n_e - 1 keV
  int n_tab, e0;               // nodes staged per launch: E = e0 .. e0 + n_tab - 1 keV
  long long n_vox;
  uint32_t m_nx, m_nxy;        // floor(2^32 / nx), floor(2^32 / (nx ny)) (2^32 - 1 for 1)
  float ox, oy, oz, inv_dx, inv_dy, inv_dz, dx, dy, dz;
  const float2* vox;           // {density, material id bits}
  const uint2* alias;          // per alias column {acceptance threshold on x >> 9, alias voxel}
  const float4* xs;            // [n_mat][n_e] cumulative {C, C+R, C+R+P, 0} (mm^-1 per g/cm^3)
  const float* maj;            // [n_e] Woodcock majorant (mm^-1), rounded up
  const float* kappa;          // [n_mat]
};

struct LutParams {
  const void* data;            // [n_apos][n_tpos][n_e][n_a][n_b], dtype below
  int dtype;                   // -1 none, 0 f32, 1 f16, 2 bf16
  int n_e, n_a, n_b, n_tpos, n_apos;
  float e_min, e_scale, a_min, a_scale, b_min, b_scale;  // g = (x - min) * scale - 0.5
  // entries between successive transaxial / axial positions; 0 on a position axis of one
  // bin (a LUT without crystal information), so every photon reads position 0
  long long t_stride, a_stride;
  long long size;              // entries (bounds checks of the debug build)
};

// one simulation request: histories [first, first + n) of seed's streams
struct Job {
  ScannerParams sc;
  PhantomParams ph;
  LutParams lut;
  unsigned long long seed, first, n;
  unsigned long long chunk;    // histories per work item
  unsigned long long* acc;     // int64 fixed-point sinogram
  int8_t* cls_out;             // optional listmode outputs, indexed by history - first
  long long* key_out;
  long long* q_out;
  int bin_mask;
};

// optional listmode records of a job (kept out of Job, which the kernel
// stages in shared memory)
struct ListmodeOut {
  psc_listmode_event* out;
  unsigned long long* count;
  unsigned long long cap;
};

constexpr int kMaxJobs = 48;   // jobs per launch (kernel parameter space)

// one persistent launch over the chunks of several jobs; chunk c belongs to
// the first job j with c < chunk_end[j]
struct BatchParams {
  Job jobs[kMaxJobs];
  unsigned long long chunk_end[kMaxJobs];
  int n_jobs;
  unsigned long long* next_chunk;  // work counter, zero at launch
  unsigned long long* stats;       // kStatCount counters or nullptr
  uint32_t* cold;                  // per-CTA slot fields kept out of shared memory
  DebugRecord* dbg;                // bounds-check record of the debug build
  ListmodeOut lm[kMaxJobs];
};
static_assert(sizeof(BatchParams) <= 32764, "kernel parameter space");

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 -> 64-bit
// multiplications, key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// uniform in (0,1): odd multiples of 2^-24 (exact in FP32)
__device__ __forceinline__ float u01(uint32_t x) {
  return (float)((x >> 9) * 2u + 1u) * 0x1p-24f;
}

__device__ __forceinline__ uint4 philox_block(unsigned long long seed, unsigned long long hist,
                                              uint32_t block, uint32_t stream) {
  return philox4x32_10(make_uint4((uint32_t)hist, (uint32_t)(hist >> 32), block, stream),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// direction after scattering by polar cosine c and azimuth 2 pi u
__device__ __forceinline__ void rotate(float3& d, float c, float u) {
  const float sn = sqrtf(fmaxf(0.0f, 1.0f - c * c));
  float sp, cp;
  sincospif(2.0f * u, &sp, &cp);
  if (fabsf(d.z) > 1.0f - kPolarEps) {
    const float sg = d.z > 0.0f ? 1.0f : -1.0f;
    d = make_float3(sn * cp, sn * sp, sg * c);
    return;
  }
  const float rr = sqrtf(1.0f - d.z * d.z);
  const float nx = c * d.x + sn * (cp * d.x * d.z - sp * d.y) / rr;
  const float ny = c * d.y + sn * (cp * d.y * d.z + sp * d.x) / rr;
  const float nz = c * d.z - sn * cp * rr;
  d = make_float3(nx, ny, nz);
}

// ---------------------------------------------------------------------------
// 5D LUT: multilinear in (E, alpha, beta) on bin-centre nodes, clamped;
// exact in the two crystal positions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void lut_axis(float x, float lo, float scale, int n, int& i0, int& i1,
                                         float& f) {
  if (n == 1) { i0 = 0; i1 = 0; f = 0.0f; return; }
  float g = (x - lo) * scale - 0.5f;
  g = fminf(fmaxf(g, 0.0f), (float)(n - 1));
  int i = min((int)g, n - 2);
  i0 = i;
  i1 = i + 1;
  f = g - (float)i;
}

// entry i of the LUT block at p (the element type follows DT)
template <int DT>
__device__ __forceinline__ float lut_load(const void* p, int i) {
  if (DT == 0) return __ldg(reinterpret_cast<const float*>(p) + i);
  if (DT == 1) return __half2float(__ldg(reinterpret_cast<const __half*>(p) + i));
  return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(p) + i));
}

template <int DT>
__device__ __forceinline__ float lut_prob(const LutParams& L, float e, float a, float b, int tpos,
                                          int apos, DebugRecord* dbg = nullptr) {
  if (DT < 0) return 1.0f;
  int e0, e1, a0, a1, b0, b1;
  float fe, fa, fb;
  lut_axis(e, L.e_min, L.e_scale, L.n_e, e0, e1, fe);
  lut_axis(a, L.a_min, L.a_scale, L.n_a, a0, a1, fa);
  lut_axis(b, L.b_min, L.b_scale, L.n_b, b0, b1, fb);
  // the (tpos, apos) block, then 32-bit offsets inside it
  long long pos = (long long)apos * L.a_stride + (long long)tpos * L.t_stride;
#if PSC_DEBUG
  {  // the block's first and last taps, or block 0 at taps 0
    const long long last = pos + ((long long)(e1 * L.n_a + a1) * L.n_b + b1);
    if (dbg_idx(dbg, kSiteLut, last, L.size) != last || dbg_idx(dbg, kSiteLut, pos, L.size) != pos) {
      pos = 0;
      e0 = e1 = a0 = a1 = b0 = b1 = 0;
    }
  }
#endif
  const void* p = DT == 0 ? (const void*)(reinterpret_cast<const float*>(L.data) + pos)
                          : (const void*)(reinterpret_cast<const __half*>(L.data) + pos);
  const int r00 = (e0 * L.n_a + a0) * L.n_b, r01 = (e0 * L.n_a + a1) * L.n_b;
  const int r10 = (e1 * L.n_a + a0) * L.n_b, r11 = (e1 * L.n_a + a1) * L.n_b;
  const float v000 = lut_load<DT>(p, r00 + b0), v001 = lut_load<DT>(p, r00 + b1);
  const float v010 = lut_load<DT>(p, r01 + b0), v011 = lut_load<DT>(p, r01 + b1);
  const float v100 = lut_load<DT>(p, r10 + b0), v101 = lut_load<DT>(p, r10 + b1);
  const float v110 = lut_load<DT>(p, r11 + b0), v111 = lut_load<DT>(p, r11 + b1);
  const float gb = 1.0f - fb, ga = 1.0f - fa, ge = 1.0f - fe;
  const float w00 = gb * v000 + fb * v001, w01 = gb * v010 + fb * v011;
  const float w10 = gb * v100 + fb * v101, w11 = gb * v110 + fb * v111;
  const float w0 = ga * w00 + fa * w01, w1 = ga * w10 + fa * w11;
  return ge * w0 + fe * w1;
}

}  // namespace psc
