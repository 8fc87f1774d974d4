// transport.cu -- fused emission -> Woodcock transport -> detection -> LUT
// weight -> LOR/TOF binning kernel (Sec. 2.2.1-2.2.3 of the paper; the
// simulator itself is the project's own design).
//
// Each lane runs a small state machine over its histories:
//
//   EMIT -> STEP <-> {COMPTON, RAYLEIGH} -> ESCAPE -> (photon B) STEP ...
//        -> ESCAPE -> COINC -> EMIT (next history)
//
// and every loop iteration executes each section once, for all lanes in
// that state together.  Lanes of a warp therefore stay converged on the hot
// section (one Woodcock step per iteration), and the code holds a single
// copy of each section, so the instruction cache is not thrashed by inlined
// copies of the photon loop.  One rejection-sampling try runs per iteration.
//
// Random numbers: a history's sub-streams (0: emission + TOF blur, 1: photon
// A, 2: photon B) are read through an 8-word per-lane window in shared
// memory; the only Philox4x32-10 evaluation sits at the top of the loop and
// appends one block when the lane's next section needs more words than the
// window holds.  The words consumed, and their order, are those of the
// per-history definition, so results do not depend on the schedule.
//
// A history adds one fixed-point weight to the int64 accumulator or nothing
// (Sec. 2.2.3: weighted or discarded, never duplicated); lanes of a warp
// that hit the same bin combine their weights before one atomic.
#include "psc_internal.h"

namespace psc {

enum : int {
  kEmit = 0, kStep = 1, kCompton = 2, kRayleigh = 3, kEscape = 4, kCoinc = 5, kNumSections = 6,
  kFinish = 6, kDone = 7
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

// incidence angles (degrees) of direction d at the hit with radial unit
// vector (nx, ny): transaxial atan2(d.t, d.n), axial atan2(d_z, d.n)
__device__ __forceinline__ void angles(float nx, float ny, float3 d, float& alpha, float& beta) {
  const float dn = d.x * nx + d.y * ny;
  const float dt = -d.x * ny + d.y * nx;
  alpha = atan2f(dt, dn) * 57.29577951308232f;
  beta = atan2f(d.z, dn) * 57.29577951308232f;
}

struct Lane {
  unsigned long long h;    // current history id
  unsigned long long m;    // index of the lane's current history within its share
  int state, photon, tries;
  uint32_t stream, k, nb;  // sub-stream, next word, blocks generated
  float3 pos, dir;
  float e, path;
  int nint, nsteps;
  float3 e0, d0;           // emission point and photon A's initial direction
  // photon A at the detector
  int a_cr, a_rg, a_scat;
  float a_e, a_path, a_nx, a_ny;
  float3 a_dir;
  // photon B at the detector (set by ESCAPE, used by COINC)
  int b_cr, b_rg;
  float b_nx, b_ny;
};

template <int DT>
__global__ void __launch_bounds__(256, 3) transport_kernel(const __grid_constant__ BatchParams B) {
  extern __shared__ float4 smem[];
  const unsigned tid = threadIdx.x, bdim = blockDim.x;
  uint32_t* ring = reinterpret_cast<uint32_t*>(smem);  // [kRingWords][blockDim]
  float4* s_xs = reinterpret_cast<float4*>(ring + kRingWords * bdim);
  __shared__ Job s_job;                       // the job of the current chunk
  __shared__ int s_j;
  __shared__ unsigned long long s_lo;         // first history of the chunk
  __shared__ unsigned s_len, s_next;          // chunk length, next offset to hand out
  __shared__ unsigned long long s_cnt[kStatCount];
  for (int i = tid; i < kStatCount; i += bdim) s_cnt[i] = 0;
  const unsigned lane_id = tid & 31u;
  const bool stats = B.stats != nullptr;
  int cached = -1;

  for (;;) {
    // ---- fetch the next chunk of (job, history range) ----
    if (tid == 0) {
      const unsigned long long c = atomicAdd(B.next_chunk, 1ull);
      int j = -1;
      if (c < B.chunk_end[B.n_jobs - 1]) {
        j = 0;
        while (B.chunk_end[j] <= c) ++j;
        const unsigned long long c0 = j ? B.chunk_end[j - 1] : 0ull;
        const unsigned long long lo = B.jobs[j].first + (c - c0) * B.jobs[j].chunk;
        const unsigned long long hi = B.jobs[j].first + B.jobs[j].n;
        s_lo = lo;
        s_len = (unsigned)min(B.jobs[j].chunk, hi - lo);
        s_next = 0;
      }
      s_j = j;
    }
    __syncthreads();
    const int jcur = s_j;
    if (jcur < 0) break;
    if (jcur != cached) {  // stage the job and its phantom's tables
      const int* src = reinterpret_cast<const int*>(&B.jobs[jcur]);
      for (int i = tid; i < (int)(sizeof(Job) / sizeof(int)); i += bdim)
        reinterpret_cast<int*>(&s_job)[i] = src[i];
      const PhantomParams& pg = B.jobs[jcur].ph;
      const int n_xs = pg.n_mat * pg.n_tab;
      float* s_maj = reinterpret_cast<float*>(s_xs + n_xs);
      float* s_kappa = s_maj + pg.n_tab;
      for (int i = tid; i < n_xs; i += bdim) {
        const int mm = i / pg.n_tab, kk = i - mm * pg.n_tab;
        s_xs[i] = pg.xs[mm * pg.n_e + pg.e0 + kk];
      }
      for (int i = tid; i < pg.n_tab; i += bdim) s_maj[i] = pg.maj[pg.e0 + i];
      if (tid < (unsigned)kMaxMaterials) s_kappa[tid] = (int)tid < pg.n_mat ? pg.kappa[tid] : 0.0f;
      cached = jcur;
    }
    __syncthreads();

    const Job& J = s_job;
    const PhantomParams& ph = J.ph;
    const ScannerParams& S = J.sc;
    const float* s_maj = reinterpret_cast<const float*>(s_xs + ph.n_mat * ph.n_tab);
    const float* s_kappa = s_maj + ph.n_tab;
    const uint2 key = make_uint2((uint32_t)J.seed, (uint32_t)(J.seed >> 32));
    const bool blur = S.tof_sigma > 0.0f;

  auto word = [&](uint32_t w) -> uint32_t { return ring[(w & (kRingWords - 1)) * bdim + tid]; };
  auto uni = [&](uint32_t w) -> float { return u01(word(w)); };
  // warp-aggregated counter increment (lanes of the calling branch)
  auto count = [&](bool pred, int slot) {
    if (!stats) return;
    const unsigned act = __activemask();
    const unsigned b = __ballot_sync(act, pred);
    if (b && lane_id == (unsigned)(__ffs(act) - 1)) atomicAdd(&s_cnt[slot], (unsigned long long)__popc(b));
  };

  Lane L;
  {
    const unsigned off = atomicAdd(&s_next, 1u);
    L.h = s_lo + off;
    L.state = off < s_len ? kEmit : kDone;
  }
  L.stream = 0;
  L.k = 0;
  L.nb = 0;

  // a history ends: remember its class; the FINISH block records it
  int fin_cls = 0;
  long long fin_key = -1, fin_q = 0;
  auto finish = [&](int cls, long long key_out, long long q_out) {
    fin_cls = cls;
    fin_key = key_out;
    fin_q = q_out;
    L.state = kFinish;
  };

  // per-section cost weights of the warp scheduler (1024 / approximate
  // instructions of one execution of the section)
  constexpr int kW[kNumSections] = {1024 / 140, 1024 / 90, 1024 / 70, 1024 / 60, 1024 / 80, 1024 / 300};
  constexpr int kNeed[kNumSections] = {7, 2, 4, 3, 0, 2};

  while (__any_sync(0xffffffffu, L.state != kDone)) {
    // ---- FINISH: record the ended history, move to the lane's next one ----
    if (L.state == kFinish) {
      const unsigned long long i = L.h - J.first;
      if (J.cls_out) J.cls_out[i] = (int8_t)fin_cls;
      if (J.key_out) J.key_out[i] = fin_key;
      if (J.q_out) J.q_out[i] = fin_q;
      if (stats) atomicAdd(&s_cnt[kStatClass0 + fin_cls], 1ull);
      const unsigned off = atomicAdd(&s_next, 1u);
      if (off < s_len) {
        L.h = s_lo + off;
        L.state = kEmit;
        L.stream = 0;
        L.k = 0;
        L.nb = 0;
      } else {
        L.state = kDone;
      }
    }

    // ---- warp vote: run the section that serves the most lanes per cost ----
    int sec = -1, best = 0;
#pragma unroll
    for (int q = 0; q < kNumSections; ++q) {
      const unsigned m = __ballot_sync(0xffffffffu, L.state == q);
      const int score = __popc(m) * kW[q];
      if (score > best) {
        best = score;
        sec = q;
      }
    }
    if (sec < 0) continue;  // only finished lanes this iteration
    const bool mine = L.state == sec;

    // ---- refill the section's lanes: the single Philox evaluation ----
    int need = kNeed[0];
#pragma unroll
    for (int q = 1; q < kNumSections; ++q) need = sec == q ? kNeed[q] : need;
    if (sec == kCoinc && !blur) need = 0;
    while (mine && L.k + need > 4 * L.nb) {
      const uint4 b = philox4x32_10(make_uint4((uint32_t)L.h, (uint32_t)(L.h >> 32), L.nb, L.stream), key);
      const uint32_t w0 = 4 * L.nb;
      ring[((w0 + 0) & (kRingWords - 1)) * bdim + tid] = b.x;
      ring[((w0 + 1) & (kRingWords - 1)) * bdim + tid] = b.y;
      ring[((w0 + 2) & (kRingWords - 1)) * bdim + tid] = b.z;
      ring[((w0 + 3) & (kRingWords - 1)) * bdim + tid] = b.w;
      ++L.nb;
      count(true, kStatRng);
    }
    if (!mine) continue;

    // ---- emission (stream 0, words 0..6) ----
    if (sec == kEmit) {
      const uint32_t w0 = word(0), w1 = word(1);
      const long long col = (long long)(((unsigned long long)w0 * (unsigned long long)ph.n_vox) >> 32);
      const uint2 at = __ldg(ph.alias + col);
      const int v = ((w1 >> 9) < at.x) ? (int)col : (int)at.y;
      const int ix = v % ph.nx, iy = (v / ph.nx) % ph.ny, iz = v / (ph.nx * ph.ny);
      L.e0 = make_float3(ph.ox + ((float)ix + uni(2)) * ph.dx, ph.oy + ((float)iy + uni(3)) * ph.dy,
                         ph.oz + ((float)iz + uni(4)) * ph.dz);
      const float ct = 2.0f * uni(5) - 1.0f;
      float sp, cp;
      sincospif(2.0f * uni(6), &sp, &cp);
      const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
      L.d0 = make_float3(st * cp, st * sp, ct);
      L.pos = L.e0;
      L.dir = L.d0;
      L.e = kEmitKeV;
      L.path = 0.0f;
      L.nint = 0;
      L.nsteps = 0;
      L.photon = 0;
      L.stream = 1;
      L.k = 0;
      L.nb = 0;
      L.state = kStep;
    }

    // ---- one Woodcock step ----
    if (sec == kStep) {
      bool moved = false;
      if (L.nsteps >= kMaxSteps) {
        finish(kStepLimit, -1, 0);
      } else {
        const float mu_max = interp_scalar(s_maj, ph.n_tab, ph.e0, L.e);
        if (!(mu_max > 0.0f)) {
          L.state = kEscape;
        } else {
          const float dist = -__logf(uni(L.k)) / mu_max;
          ++L.k;
          const float qx = L.pos.x + dist * L.dir.x;
          const float qy = L.pos.y + dist * L.dir.y;
          const float qz = L.pos.z + dist * L.dir.z;
          const float fx = (qx - ph.ox) * ph.inv_dx;
          const float fy = (qy - ph.oy) * ph.inv_dy;
          const float fz = (qz - ph.oz) * ph.inv_dz;
          if (!(fx >= 0.0f && fx < (float)ph.nx && fy >= 0.0f && fy < (float)ph.ny && fz >= 0.0f &&
                fz < (float)ph.nz)) {
            L.state = kEscape;  // outside the grid is vacuum: straight to the detector
          } else {
            moved = true;
            const int ix = min((int)fx, ph.nx - 1);
            const int iy = min((int)fy, ph.ny - 1);
            const int iz = min((int)fz, ph.nz - 1);
            L.pos = make_float3(qx, qy, qz);
            L.path += dist;
            ++L.nsteps;
            const float2 vx = __ldg(ph.vox + ((long long)iz * ph.ny + iy) * ph.nx + ix);
            const int mat = __float_as_int(vx.y);
            const float4 cum = interp_xs(s_xs + mat * ph.n_tab, ph.n_tab, ph.e0, L.e);
            const float t = uni(L.k) * mu_max;
            ++L.k;
            if (t < vx.x * cum.x) {
              L.state = kCompton;
              L.tries = 0;
            } else if (t < vx.x * cum.y) {
              L.state = kRayleigh;
              L.tries = mat << 16;  // the material id travels with the pending event
            } else if (t < vx.x * cum.z) {
              count(true, kStatPhoto);
              finish(kAbsorbed, -1, 0);
            }
          }
        }
      }
      count(moved, kStatSteps);
    }

    // ---- one Klein-Nishina try (Kahn's method on x = E/E') ----
    if (sec == kCompton) {
      const float r1 = uni(L.k), r2 = uni(L.k + 1), r3 = uni(L.k + 2);
      L.k += 3;
      ++L.tries;
      const float a = L.e / kRestKeV;
      const float two_a = 2.0f * a;
      float x, c;
      bool accept;
      if (r1 < (1.0f + two_a) / (9.0f + two_a)) {
        x = 1.0f + two_a * r2;
        c = 1.0f - (x - 1.0f) / a;
        accept = r3 < 4.0f * (1.0f / x - 1.0f / (x * x));
      } else {
        x = (1.0f + two_a) / (1.0f + two_a * r2);
        c = 1.0f - (x - 1.0f) / a;
        accept = r3 < 0.5f * (c * c + 1.0f / x);
      }
      count(true, kStatTries);
      if (accept || L.tries >= kMaxTries) {
        rotate(L.dir, c, uni(L.k));
        ++L.k;
        L.e = L.e / x;
        ++L.nint;
        count(true, kStatCompton);
        if (L.e < S.e_lo) finish(kEnergyWindow, -1, 0);
        else L.state = kStep;
      }
    }

    // ---- one Rayleigh try (material id in the upper half of tries) ----
    if (sec == kRayleigh) {
      const float u1 = uni(L.k), u2 = uni(L.k + 1);
      L.k += 2;
      ++L.tries;
      const float er = L.e / kRestKeV;
      const float b = s_kappa[L.tries >> 16] * er * er;
      const float sv = u1 / (1.0f + b * (1.0f - u1));
      const float c = 1.0f - 2.0f * sv;
      count(true, kStatTries);
      if (u2 < 0.5f * (1.0f + c * c) || (L.tries & 0xffff) >= kMaxTries) {
        rotate(L.dir, c, uni(L.k));
        ++L.k;
        ++L.nint;
        count(true, kStatRayleigh);
        L.state = kStep;
      }
    }

    // ---- the photon reaches the detector cylinder ----
    if (sec == kEscape) {
      const float3 p = L.pos, d = L.dir;
      const float a = d.x * d.x + d.y * d.y;
      int cls = kDetected, cr = 0, rg = 0;
      float nx = 0.0f, ny = 0.0f;
      if (!(a > 0.0f)) {
        cls = kLostAxial;
      } else {
        const float b = p.x * d.x + p.y * d.y;
        const float c = p.x * p.x + p.y * p.y - S.r2;
        const float sq = sqrtf(fmaxf(b * b - a * c, 0.0f));
        const float t = (b >= 0.0f) ? (-c) / (b + sq) : (sq - b) / a;
        const float hx = p.x + t * d.x, hy = p.y + t * d.y, hz = p.z + t * d.z;
        L.path += t;
        if (!(hz >= -S.half_len && hz < S.half_len)) {
          cls = kLostAxial;
        } else {
          rg = max(0, min((int)floorf((hz + S.half_len) * S.inv_pitch), S.n_rings - 1));
          float phi = atan2f(hy, hx);
          if (phi < 0.0f) phi += 6.283185307179586f;
          cr = max(0, min((int)floorf(phi * S.crystals_per_radian), S.n_crystals - 1));
          nx = hx / S.radius;
          ny = hy / S.radius;
          if (L.e < S.e_lo || L.e > S.e_hi) cls = kEnergyWindow;
        }
      }
      count(cls == kDetected, kStatDetected);
      if (cls != kDetected) {
        finish(cls, -1, 0);
      } else if (L.photon == 0) {
        L.a_cr = cr;
        L.a_rg = rg;
        L.a_scat = L.nint;
        L.a_e = L.e;
        L.a_path = L.path;
        L.a_nx = nx;
        L.a_ny = ny;
        L.a_dir = L.dir;
        L.pos = L.e0;  // photon B leaves back to back
        L.dir = make_float3(-L.d0.x, -L.d0.y, -L.d0.z);
        L.e = kEmitKeV;
        L.path = 0.0f;
        L.nint = 0;
        L.nsteps = 0;
        L.photon = 1;
        L.stream = 2;
        L.k = 0;
        L.nb = 0;
        L.state = kStep;
      } else if (cr == L.a_cr) {
        finish(kSameCrystal, -1, 0);
      } else {
        L.b_cr = cr;
        L.b_rg = rg;
        L.b_nx = nx;
        L.b_ny = ny;
        L.state = kCoinc;
        if (blur) {  // the TOF blur reads stream 0, block 2
          L.stream = 0;
          L.k = 8;
          L.nb = 2;
        }
      }
    }

    // ---- coincidence: TOF, LOR bin, LUT weight, accumulate ----
    if (sec == kCoinc) {
      const bool a_first = L.a_cr < L.b_cr;
      float delta = 0.5f * (a_first ? L.a_path - L.path : L.path - L.a_path);
      if (blur) {
        const float g = sqrtf(-2.0f * logf(uni(8))) * cospif(2.0f * uni(9));
        delta += S.tof_sigma * g;
      }
      const long long key_ = a_first ? bin_key(S, L.a_cr, L.b_cr, L.a_rg, L.b_rg, delta)
                                     : bin_key(S, L.b_cr, L.a_cr, L.b_rg, L.a_rg, delta);
      const bool scattered = (L.a_scat + L.nint) > 0;
      const int cls = key_ < 0 ? kOutOfRange : scattered ? kScatter : kTrue;
      const bool take = cls == kScatter ? (J.bin_mask & 1) : cls == kTrue ? (J.bin_mask & 2) : false;
      long long q = 0;
      if (key_ >= 0 && (take || J.q_out)) {
        float aa, ab, ba, bb;
        angles(L.a_nx, L.a_ny, L.a_dir, aa, ab);
        angles(L.b_nx, L.b_ny, L.dir, ba, bb);
        const float w = lut_prob<DT>(J.lut, L.a_e, aa, ab, L.a_cr % S.module_t, L.a_rg % S.module_a) *
                        lut_prob<DT>(J.lut, L.e, ba, bb, L.b_cr % S.module_t, L.b_rg % S.module_a);
        q = __float2ll_rn(w * 4294967296.0f);
      }
      // lanes that hit the same bin add their weights first, one atomic per bin
      const unsigned act = __activemask();
      const unsigned takers = __ballot_sync(act, take);
      if (take) {
        const unsigned peers = __match_any_sync(takers, (unsigned long long)key_);
        const unsigned hi = __reduce_add_sync(peers, (unsigned)(q >> 16));
        const unsigned lo = __reduce_add_sync(peers, (unsigned)(q & 0xffff));
        if (lane_id == (unsigned)(__ffs(peers) - 1)) {
          atomicAdd(J.acc + key_, ((unsigned long long)hi << 16) + lo);
          if (stats) atomicAdd(&s_cnt[kStatAtomics], 1ull);
        }
        if (stats) {
          atomicAdd(&s_cnt[kStatBinned], 1ull);
          atomicAdd(&s_cnt[kStatWeight], (unsigned long long)q);
        }
      }
      finish(cls, key_, cls == kOutOfRange ? 0 : q);
    }
  }

    __syncthreads();  // every lane is done with the chunk before the next fetch
  }

  if (!stats) return;
  __syncthreads();
  for (int i = threadIdx.x; i < kStatCount; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(B.stats + i, s_cnt[i]);
}

size_t transport_smem_bytes(const PhantomParams& ph, int block) {
  return sizeof(uint32_t) * kRingWords * block + sizeof(float4) * (size_t)ph.n_mat * ph.n_tab +
         sizeof(float) * (ph.n_tab + kMaxMaterials);
}

template <int DT>
static cudaError_t launch_dt(const BatchParams& p, int grid, int block, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(transport_kernel<DT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  transport_kernel<DT><<<grid, block, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_transport(const BatchParams& p, int lut_dtype, int grid, int block, size_t smem,
                             cudaStream_t s) {
  switch (lut_dtype) {
    case 0: return launch_dt<0>(p, grid, block, smem, s);
    case 1: return launch_dt<1>(p, grid, block, smem, s);
    case 2: return launch_dt<2>(p, grid, block, smem, s);
    default: return launch_dt<-1>(p, grid, block, smem, s);
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
