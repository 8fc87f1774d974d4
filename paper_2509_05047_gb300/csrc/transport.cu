// transport.cu -- fused emission -> Woodcock transport -> detection -> LUT
// weight -> LOR/TOF binning kernel (Sec. 2.2.1-2.2.3 of the paper; the
// simulator itself is the project's own design).
//
// A history is a small state machine:
//
//   EMIT -> STEP <-> {COMPTON, RAYLEIGH} -> ESCAPE -> (photon B) STEP ...
//        -> ESCAPE -> COINC -> next history
//
// Each warp owns a pool of kSlotsPerWarp photon slots whose state lives in
// shared memory (structure of arrays; the fields only emission, detection
// and coincidence touch live in an L2-resident global buffer instead, which
// leaves room for 32 warps per SM).  Every loop iteration the warp picks the
// section that the most slots wait for (weighting sections by their cost
// was measured slower, since it runs sections on fewer lanes), packs up to
// 32 slots in that state onto its 32 lanes, and runs the section once.  With
// twice as many slots as lanes the chosen section usually fills the warp,
// where one history per lane left most lanes idle (the states of 32
// histories spread over six sections).  The code holds a single copy of each
// section, and one rejection-sampling try runs per iteration.  Pools stay
// per warp, so warps never wait on each other: pools shared by two warps
// (barrier-coupled) and larger pools (fewer resident warps) both measured
// slower on this issue-bound loop.
//
// Random numbers: a history's sub-streams (0: emission + TOF blur, 1: photon
// A, 2: photon B) are read through an 8-word window per slot; the only
// Philox4x32-10 evaluation sits before the sections and appends one block
// when the slot's next section needs more words than the window holds.  The
// words consumed, and their order, are those of the per-history definition,
// so results do not depend on the schedule, the slot or the lane.
//
// A history adds one fixed-point weight to the int64 accumulator or nothing
// (Sec. 2.2.3: weighted or discarded, never duplicated); lanes of a warp
// that hit the same bin combine their weights before one atomic.
#include "psc_internal.h"

namespace psc {

enum : int {
  kEmit = 0, kStep = 1, kCompton = 2, kRayleigh = 3, kEscape = 4, kCoinc = 5, kNumSections = 6,
  kDone = 7
};

constexpr int kSlotsPerWarp = 64;

// fields of a photon slot kept in shared memory (used by every section):
// field f of slot g at slots[f * n_slots + g]
enum : int {
  F_PX, F_PY, F_PZ, F_DX, F_DY, F_DZ, F_E, F_PATH,          // the photon in flight
  F_K, F_NB, F_HLO, F_HHI, F_META, F_CNT, F_TRIES,          // stream position, history, state
  F_RING,                                                    // kRingWords words of the sub-stream
  kFields = F_RING + kRingWords
};
// fields read and written only at emission, detection and coincidence, kept
// in an L2-resident global buffer: field f of slot g of CTA b at
// cold[(b * kColdFields + f) * n_slots + g]
enum : int {
  C_E0X, C_E0Y, C_E0Z, C_D0X, C_D0Y, C_D0Z,                 // emission point, photon A direction
  C_ACRG, C_AE, C_APATH, C_ANX, C_ANY, C_ADX, C_ADY, C_ADZ,  // photon A at the detector
  C_BCRG, C_BNX, C_BNY,                                      // photon B at the detector
  C_APOS, C_BPOS,                                            // LUT positions (scanners with gaps)
  C_VOX, C_AZ, C_BZ, C_ASC,                                  // listmode records only
  kColdFields
};
// F_META = state | photon << 3 | stream << 4;  F_CNT = steps | interactions << 16;
// C_ACRG = crystal | ring << 16 | scattered << 31;  C_BCRG = crystal | ring << 16;
// C_APOS, C_BPOS = tpos | apos << 16;  C_ASC = photon A's F_CNT >> 15;
// listmode runs flag a Rayleigh interaction in bit 15 of F_CNT (steps stay below 2^15)
// F_TRIES = tries (| material << 16 for a pending Rayleigh event)
__host__ __device__ constexpr uint32_t meta(int state, int photon, int stream) {
  return (uint32_t)state | (uint32_t)photon << 3 | (uint32_t)stream << 4;
}


// 1 << s, and 0 for s >= 32 (the PTX shift clamps its amount to the width)
__device__ __forceinline__ unsigned shl_or_zero(unsigned s) {
  unsigned d;
  asm("shl.b32 %0, %1, %2;" : "=r"(d) : "r"(1u), "r"(s));
  return d;
}

// per-half maximum of two pairs of unsigned 16-bit values
__device__ __forceinline__ unsigned umax16x2(unsigned a, unsigned b) {
  unsigned d;
  asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

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

// Gaps between modules and blocks (Sec. 2.2.1-2.2.2).  A photon in a gap
// goes to the crystal at the gap's low (p) or high (1 - p) edge, p the
// relative probability that it is absorbed in the block on the low side:
// its straight line, at slope s = tan(theta) and cos(theta) = c against the
// radial direction, enters the blocks (depth D, faces doi below the
// detection cylinder, gap centred at x = 0, the photon at x0) and is
// absorbed in the first block it crosses with 1 - e^{-mu l1}, in the other
// with e^{-mu l1} (1 - e^{-mu l2}).  Crossing neither, the nearer side.
__device__ __forceinline__ float edge_prob(const ScannerParams& S, float x0, float s, float c, float gap) {
  float l1 = 0.0f, l2 = 0.0f;  // path lengths in the low and high block
  if (s != 0.0f) {
    const float ya = S.doi + (-0.5f * gap - x0) / s, yb = S.doi + (0.5f * gap - x0) / s;
    if (s > 0.0f) {  // the low block is crossed near the face, the high one deeper
      l1 = fmaxf(0.0f, fminf(S.depth, ya)) / c;
      l2 = fmaxf(0.0f, S.depth - fmaxf(0.0f, yb)) / c;
    } else {
      l2 = fmaxf(0.0f, fminf(S.depth, yb)) / c;
      l1 = fmaxf(0.0f, S.depth - fmaxf(0.0f, ya)) / c;
    }
  }
  const float first = s > 0.0f ? l1 : l2, second = s > 0.0f ? l2 : l1;
  const float pf = -expm1f(-S.mu * first);
  const float ps = expf(-S.mu * first) * -expm1f(-S.mu * second);
  const float p1 = s > 0.0f ? pf : ps, p2 = s > 0.0f ? ps : pf;
  if (!(p1 + p2 > 0.0f)) return x0 < 0.0f ? 1.0f : (x0 > 0.0f ? 0.0f : 0.5f);
  return p1 / (p1 + p2);
}

// LUT position and crystal of a detected photon on a scanner with gaps.
// Module m spans azimuth [m mod_phi, (m + 1) mod_phi) as [half gap | module_t
// crystals | half gap], block b the axial range [b blk_pitch, (b + 1)
// blk_pitch) in the same way.  Returns crystal | ring << 16 | lost << 31 in
// the low word (lost: in a gap, gap_mode 1) and tpos | apos << 16 in the high
// word.  Gap_mode 2 assigns a photon in a transaxial gap with u0, then one in
// an inner axial gap with the next of (u0, u1); at the scanner's axial ends
// only one block borders the gap.
__device__ __noinline__ unsigned long long place(const ScannerParams& S, float phi, float hz, float dx, float dy,
                                                 float dz, float nx, float ny, float u0, float u1) {
  const int m = min((int)floorf(phi * S.inv_mod_phi), S.n_mod - 1);
  const float u = phi - (float)m * S.mod_phi;
  int tp, bt = 0, cr = 0;
  float xt = 0.0f;
  if (u < 0.5f * S.gap_gamma) {
    tp = 0;
    bt = m;
    xt = u * S.radius;
  } else if (u >= S.mod_phi - 0.5f * S.gap_gamma) {
    tp = S.module_t + 1;
    bt = m + 1;
    xt = (u - S.mod_phi) * S.radius;
  } else {
    const int j = max(0, min((int)floorf((u - 0.5f * S.gap_gamma) * S.inv_crys_phi), S.module_t - 1));
    tp = j + 1;
    cr = m * S.module_t + j;
  }
  const float z = hz + S.half_len;
  const int b = max(0, min((int)floorf(z * S.inv_blk_pitch), S.n_blk - 1));
  const float w = z - (float)b * S.blk_pitch;
  int al, ba = 0, rg = 0;
  float xa = 0.0f;
  if (w < 0.5f * S.gap_a) {
    al = 0;
    ba = b;
    xa = w;
  } else if (w >= S.blk_pitch - 0.5f * S.gap_a) {
    al = S.module_a + 1;
    ba = b + 1;
    xa = w - S.blk_pitch;
  } else {
    const int j = max(0, min((int)floorf((w - 0.5f * S.gap_a) * S.inv_ring_w), S.module_a - 1));
    al = j + 1;
    rg = b * S.module_a + j;
  }
  const unsigned long long pos = (unsigned long long)((uint32_t)tp | (uint32_t)(b * (S.module_a + 2) + al) << 16)
                                 << 32;
  const bool gt = tp == 0 || tp == S.module_t + 1, ga = al == 0 || al == S.module_a + 1;
  if (S.gap_mode == 1) return pos | (gt || ga ? 1ull << 31 : 0ull) | (uint32_t)cr | (uint32_t)rg << 16;
  const float dn = dx * nx + dy * ny, dt = -dx * ny + dy * nx;
  if (gt) {
    const float p1 = edge_prob(S, xt, dt / dn, dn * rsqrtf(dn * dn + dt * dt), S.gap_t_mm);
    const int c0 = bt * S.module_t;
    cr = u0 < p1 ? (c0 == 0 ? S.n_crystals - 1 : c0 - 1) : (c0 == S.n_crystals ? 0 : c0);
  }
  if (ga) {
    if (ba == 0) {
      rg = 0;
    } else if (ba == S.n_blk) {
      rg = S.n_rings - 1;
    } else {
      const float p1 = edge_prob(S, xa, dz / dn, dn * rsqrtf(dn * dn + dz * dz), S.gap_a);
      rg = (gt ? u1 : u0) < p1 ? ba * S.module_a - 1 : ba * S.module_a;
    }
  }
  return pos | (uint32_t)cr | (uint32_t)rg << 16;
}

// incidence angles (degrees) of direction d at the hit with radial unit
// vector (nx, ny): transaxial atan2(d.t, d.n), axial atan2(d_z, d.n)
__device__ __forceinline__ void angles(float nx, float ny, float3 d, float& alpha, float& beta) {
  const float dn = d.x * nx + d.y * ny;
  const float dt = -d.x * ny + d.y * nx;
  alpha = atan2f(dt, dn) * 57.29577951308232f;
  beta = atan2f(d.z, dn) * 57.29577951308232f;
}


// kDebug: statistics counters and per-history listmode outputs are compiled
// in only when a launch asks for them, so the production loop stays small.
// kOneJob (production launches of a single job with an f32 LUT, the common
// case): the job's index in the kernel parameter space is the constant 0.
// kFixed (production launches of 512-thread CTAs, the default): the slot
// count is a compile-time constant, so every slot field access is an
// immediate offset from the slot's address (measured 10 % faster).
template <int DT, bool kDebug, bool kOneJob = false, bool kFixed = false>
__global__ void __launch_bounds__(512, 2) transport_kernel(const __grid_constant__ BatchParams B) {
  extern __shared__ float4 smem[];
  const unsigned tid = threadIdx.x, bdim = blockDim.x;
  const int n_slots = kFixed ? 16 * kSlotsPerWarp : (int)(bdim >> 5) * kSlotsPerWarp;
  uint32_t* slots = reinterpret_cast<uint32_t*>(smem);  // [kFields][n_slots]
  float4* s_xs = reinterpret_cast<float4*>(slots + kFields * n_slots);
  __shared__ int s_j;
  __shared__ unsigned long long s_lo;         // first history of the chunk
  __shared__ unsigned s_len, s_next;          // chunk length, next offset to hand out
  __shared__ unsigned long long s_cnt[kStatCount];
  __shared__ int s_sel[16][32];               // per warp: slot of each lane this iteration
  for (int i = tid; i < kStatCount; i += bdim) s_cnt[i] = 0;
  const unsigned lane_id = tid & 31u;
  const int warp = (int)(tid >> 5);
  const int g0 = warp * kSlotsPerWarp + (int)lane_id, g1 = g0 + 32;  // the slots this lane refills
  const bool stats = kDebug && B.stats != nullptr;
  int cached = -1;

  auto U = [&](int f, int g) -> uint32_t& { return slots[f * n_slots + g]; };
  auto Fv = [&](int f, int g) -> float { return __uint_as_float(slots[f * n_slots + g]); };
  auto setF = [&](int f, int g, float v) { slots[f * n_slots + g] = __float_as_uint(v); };
  uint32_t* cold = B.cold + (size_t)blockIdx.x * kColdFields * n_slots;
  auto CU = [&](int f, int g) -> uint32_t& { return cold[f * n_slots + g]; };
  auto Cv = [&](int f, int g) -> float { return __uint_as_float(cold[f * n_slots + g]); };
  auto setC = [&](int f, int g, float v) { cold[f * n_slots + g] = __float_as_uint(v); };

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
    const ListmodeOut lm = kDebug ? B.lm[jcur] : ListmodeOut{nullptr, nullptr, 0};
    if (jcur != cached) {  // stage the job's phantom tables
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

    // the job's parameters, read from the kernel parameter space (a
    // compile-time index for single-job launches, the CTA-uniform chunk's job
    // otherwise): operands of the instructions, not registers held across the
    // loop (a shared-memory copy made the multi-job instantiations spill)
    const Job& J = [&]() -> const Job& {
      if constexpr (kOneJob) return B.jobs[0];
      else return B.jobs[jcur];
    }();
    const PhantomParams& ph = J.ph;
    const ScannerParams& S = J.sc;
    const float* s_maj = reinterpret_cast<const float*>(s_xs + ph.n_mat * ph.n_tab);
    const float* s_kappa = s_maj + ph.n_tab;
    const uint2 key = make_uint2((uint32_t)J.seed, (uint32_t)(J.seed >> 32));
    const bool blur = S.tof_sigma > 0.0f;

    // warp-aggregated counter increment (lanes of the calling branch)
    auto count = [&](bool pred, int slot) {
      if (!stats) return;
      const unsigned act = __activemask();
      const unsigned b = __ballot_sync(act, pred);
      if (b && lane_id == (unsigned)(__ffs(act) - 1)) atomicAdd(&s_cnt[slot], (unsigned long long)__popc(b));
    };
    // slot g takes the chunk's next history, or is done
    auto start = [&](int g) {
      const unsigned off = atomicAdd(&s_next, 1u);
      if (off < s_len) {
        const unsigned long long h = s_lo + off;
        U(F_HLO, g) = (uint32_t)h;
        U(F_HHI, g) = (uint32_t)(h >> 32);
        U(F_META, g) = meta(kEmit, 0, 0);
        U(F_K, g) = 0;
        U(F_NB, g) = 0;
      } else {
        U(F_META, g) = kDone;
      }
    };
    // a history ends in slot g: record its class (and bin, weight), start the next
    auto finish = [&](int g, int cls, long long key_out, long long q_out) {
      const unsigned long long h = (unsigned long long)U(F_HHI, g) << 32 | U(F_HLO, g);
      const unsigned long long i = (unsigned long long)dbg_idx(B.dbg, kSiteHistOut, (long long)(h - J.first),
                                                               (long long)J.n);
      if (kDebug) {
        if (J.cls_out) J.cls_out[i] = (int8_t)cls;
        if (J.key_out) J.key_out[i] = key_out;
        if (J.q_out) J.q_out[i] = q_out;
        if (stats) atomicAdd(&s_cnt[kStatClass0 + cls], 1ull);
      }
      start(g);
    };

    start(g0);
    start(g1);
    __syncwarp();

    // words a section reads, one nibble per section: 7, 2, 4, 3, 0, 2.  After a refill
    // the window holds words [4 nb - kRingWords, 4 nb) with 4 nb < k + need + 4, so it
    // still holds word k only for need <= kRingWords - 3; EMIT (7) starts at k = 0.
    // Detection reads at most 4 (energy blur 2, edge draws 2).
    constexpr uint32_t kNeedNibbles = 0x203427u;
    static_assert(((kNeedNibbles >> 4) & 15u) <= kRingWords - 3 && ((kNeedNibbles >> 8) & 15u) <= kRingWords - 3 &&
                      ((kNeedNibbles >> 12) & 15u) <= kRingWords - 3 && ((kNeedNibbles >> 20) & 15u) <= kRingWords - 3 &&
                      4 <= kRingWords - 3 && (kNeedNibbles & 15u) <= kRingWords,
                  "a section's words must fit the Philox window");

    for (;;) {
      const int st0 = (int)(U(F_META, g0) & 7u), st1 = (int)(U(F_META, g1) & 7u);

      // ---- warp vote: the section that the most slots wait for ----
      // slot counts per state, one byte each (at most 64 slots): states 0..3
      // in lo, 4..7 in hi (sections 4, 5 in its bytes 0, 1), summed over the
      // warp by two reductions.  A state's bit is 1 << 8 st, or 1 << (8 st - 32)
      // in hi, where shift amounts of 32 and more (unsigned wrap included) give 0.
      const unsigned lo = shl_or_zero(8u * st0) + shl_or_zero(8u * st1);
      const unsigned hi = shl_or_zero(8u * st0 - 32u) + shl_or_zero(8u * st1 - 32u);
      const unsigned clo = __reduce_add_sync(0xffffffffu, lo), chi = __reduce_add_sync(0xffffffffu, hi);
      if ((clo | (chi & 0xffffu)) == 0u) break;  // every slot is done
      // the most-populated section, the lowest on a tie: keys count << 3 | (7 - q)
      // in 16-bit halves, two paired maxima, then the larger half.  A section
      // with slots outranks every empty one (key >= 8), so sec is never empty.
      const unsigned k01 = __byte_perm(clo, 0u, 0x4140) * 8u + 0x00060007u;
      const unsigned k23 = __byte_perm(clo, 0u, 0x4342) * 8u + 0x00040005u;
      const unsigned k45 = __byte_perm(chi, 0u, 0x4140) * 8u + 0x00020003u;
      const unsigned km = umax16x2(umax16x2(k01, k23), k45);
      const int sec = 7 - (int)(max(km & 0xffffu, km >> 16) & 7u);
      const unsigned sm0 = __ballot_sync(0xffffffffu, st0 == sec);
      const unsigned sm1 = __ballot_sync(0xffffffffu, st1 == sec);
      // ---- pack up to 32 slots in that state onto the lanes ----
      const unsigned below = (1u << lane_id) - 1u;
      const int n0 = __popc(sm0);
      if (st0 == sec) s_sel[warp][__popc(sm0 & below)] = g0;
      if (st1 == sec) {
        const int r = n0 + __popc(sm1 & below);
        if (r < 32) s_sel[warp][r] = g1;
      }
      __syncwarp();
      const int g = (int)lane_id < min(32, n0 + __popc(sm1))
                        ? (int)dbg_idx(B.dbg, kSiteSlot, s_sel[warp][lane_id], n_slots) : -1;
      __syncwarp();

      if (g >= 0) {
        // ---- refill the slot's window: the single Philox evaluation ----
        uint32_t k = U(F_K, g), nb = U(F_NB, g);
        int need = (int)((kNeedNibbles >> (4 * sec)) & 15u);
        if (sec == kEscape) need = S.escape_words;  // energy blur, edge-crystal draws
        if (sec == kCoinc && !blur) need = 0;
        if (k + need > 4 * nb) {
          const uint32_t hlo = U(F_HLO, g), hhi = U(F_HHI, g), stream = U(F_META, g) >> 4;
          do {
            const uint4 b = philox4x32_10(make_uint4(hlo, hhi, nb, stream), key);
            const uint32_t w0 = 4 * nb;
            U(F_RING + ((w0 + 0) & (kRingWords - 1)), g) = b.x;
            U(F_RING + ((w0 + 1) & (kRingWords - 1)), g) = b.y;
            U(F_RING + ((w0 + 2) & (kRingWords - 1)), g) = b.z;
            U(F_RING + ((w0 + 3) & (kRingWords - 1)), g) = b.w;
            ++nb;
            count(true, kStatRng);
          } while (k + need > 4 * nb);
          U(F_NB, g) = nb;
        }
        auto word = [&](uint32_t w) -> uint32_t { return U(F_RING + (w & (kRingWords - 1)), g); };
        auto uni = [&](uint32_t w) -> float { return u01(word(w)); };

        // ---- emission (stream 0, words 0..6) ----
        if (sec == kEmit) {
          const uint32_t w0 = word(0), w1 = word(1);
          const unsigned col = __umulhi(w0, (unsigned)ph.n_vox);  // n_vox < 2^31
          const uint2 at = __ldg(ph.alias + dbg_idx(B.dbg, kSiteAlias, col, ph.n_vox));
          const int v = ((w1 >> 9) < at.x) ? (int)col : (int)at.y;
          // v = (iz ny + iy) nx + ix: quotients from a multiply-high with floor(2^32 / d),
          // at most one below the true quotient, then one correction
          const unsigned nxy = (unsigned)(ph.nx * ph.ny);
          unsigned iz = __umulhi((unsigned)v, ph.m_nxy), rem = (unsigned)v - iz * nxy;
          if (rem >= nxy) {
            ++iz;
            rem -= nxy;
          }
          unsigned iy = __umulhi(rem, ph.m_nx), ix = rem - iy * (unsigned)ph.nx;
          if (ix >= (unsigned)ph.nx) {
            ++iy;
            ix -= (unsigned)ph.nx;
          }
          const float ex = ph.ox + ((float)ix + uni(2)) * ph.dx, ey = ph.oy + ((float)iy + uni(3)) * ph.dy,
                      ez = ph.oz + ((float)iz + uni(4)) * ph.dz;
          const float ct = 2.0f * uni(5) - 1.0f;
          float sp, cp;
          sincospif(2.0f * uni(6), &sp, &cp);
          const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
          const float dx = st * cp, dy = st * sp, dz = ct;
          setC(C_E0X, g, ex);
          setC(C_E0Y, g, ey);
          setC(C_E0Z, g, ez);
          setC(C_D0X, g, dx);
          setC(C_D0Y, g, dy);
          setC(C_D0Z, g, dz);
          if (kDebug && lm.out) CU(C_VOX, g) = (uint32_t)v;
          setF(F_PX, g, ex);
          setF(F_PY, g, ey);
          setF(F_PZ, g, ez);
          setF(F_DX, g, dx);
          setF(F_DY, g, dy);
          setF(F_DZ, g, dz);
          setF(F_E, g, kEmitKeV);
          setF(F_PATH, g, 0.0f);
          U(F_CNT, g) = 0;
          U(F_K, g) = 0;
          U(F_NB, g) = 0;
          U(F_META, g) = meta(kStep, 0, 1);
        }

        // ---- one Woodcock step ----
        if (sec == kStep) {
          bool moved = false, ended = false;
          const uint32_t cnt = U(F_CNT, g);
          if ((int)(cnt & 0x7fffu) >= kMaxSteps) {
            finish(g, kStepLimit, -1, 0);
          } else {
            const float e = Fv(F_E, g);
            const float mu_max = interp_scalar(s_maj, ph.n_tab, ph.e0, e);
            const uint32_t m = U(F_META, g);
            if (!(mu_max > 0.0f)) {
              U(F_META, g) = (m & ~7u) | kEscape;
            } else {
              const float px = Fv(F_PX, g), py = Fv(F_PY, g), pz = Fv(F_PZ, g);
              const float dx = Fv(F_DX, g), dy = Fv(F_DY, g), dz = Fv(F_DZ, g);
              const float dist = -__logf(uni(k)) / mu_max;
              ++k;
              const float qx = px + dist * dx;
              const float qy = py + dist * dy;
              const float qz = pz + dist * dz;
              const float fx = (qx - ph.ox) * ph.inv_dx;
              const float fy = (qy - ph.oy) * ph.inv_dy;
              const float fz = (qz - ph.oz) * ph.inv_dz;
              if (!(fx >= 0.0f && fx < (float)ph.nx && fy >= 0.0f && fy < (float)ph.ny && fz >= 0.0f &&
                    fz < (float)ph.nz)) {
                U(F_META, g) = (m & ~7u) | kEscape;  // outside the grid is vacuum: straight to the detector
              } else {
                moved = true;
                const int ix = min((int)fx, ph.nx - 1);
                const int iy = min((int)fy, ph.ny - 1);
                const int iz = min((int)fz, ph.nz - 1);
                setF(F_PX, g, qx);
                setF(F_PY, g, qy);
                setF(F_PZ, g, qz);
                setF(F_PATH, g, Fv(F_PATH, g) + dist);
                U(F_CNT, g) = cnt + 1u;
                const float2 vx = __ldg(ph.vox + dbg_idx(B.dbg, kSiteVoxel, (unsigned)((iz * ph.ny + iy) * ph.nx + ix),
                                                         ph.n_vox));  // n_vox < 2^31
                const int mat = (int)dbg_idx(B.dbg, kSiteMaterial, __float_as_int(vx.y), ph.n_mat);
                const float4 cum = interp_xs(s_xs + mat * ph.n_tab, ph.n_tab, ph.e0, e);
                const float t = uni(k) * mu_max;
                ++k;
                if (t < vx.x * cum.x) {
                  U(F_META, g) = (m & ~7u) | kCompton;
                  U(F_TRIES, g) = 0;
                } else if (t < vx.x * cum.y) {
                  U(F_META, g) = (m & ~7u) | kRayleigh;
                  U(F_TRIES, g) = (uint32_t)mat << 16;  // the material id travels with the pending event
                } else if (t < vx.x * cum.z) {
                  count(true, kStatPhoto);
                  ended = true;
                }
              }
              if (ended) finish(g, kAbsorbed, -1, 0);
              else U(F_K, g) = k;
            }
          }
          count(moved, kStatSteps);
        }

        // ---- one Klein-Nishina try (Kahn's method on x = E/E') ----
        if (sec == kCompton) {
          const float r1 = uni(k), r2 = uni(k + 1), r3 = uni(k + 2);
          k += 3;
          const uint32_t tries = U(F_TRIES, g) + 1u;
          const float e = Fv(F_E, g);
          const float a = e / kRestKeV;
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
          if (accept || (int)tries >= kMaxTries) {
            float3 d = make_float3(Fv(F_DX, g), Fv(F_DY, g), Fv(F_DZ, g));
            rotate(d, c, uni(k));
            ++k;
            const float e1 = e / x;
            count(true, kStatCompton);
            if (e1 < S.e_kill) {
              finish(g, kEnergyWindow, -1, 0);
            } else {
              setF(F_DX, g, d.x);
              setF(F_DY, g, d.y);
              setF(F_DZ, g, d.z);
              setF(F_E, g, e1);
              U(F_CNT, g) += 1u << 16;
              U(F_K, g) = k;
              U(F_META, g) = (U(F_META, g) & ~7u) | kStep;
            }
          } else {
            U(F_TRIES, g) = tries;
            U(F_K, g) = k;
          }
        }

        // ---- one Rayleigh try (material id in the upper half of tries) ----
        if (sec == kRayleigh) {
          const float u1 = uni(k), u2 = uni(k + 1);
          k += 2;
          const uint32_t tries = U(F_TRIES, g) + 1u;
          const float e = Fv(F_E, g);
          const float er = e / kRestKeV;
          const float b = s_kappa[dbg_idx(B.dbg, kSiteKappa, tries >> 16, ph.n_mat)] * er * er;
          const float sv = u1 / (1.0f + b * (1.0f - u1));
          const float c = 1.0f - 2.0f * sv;
          count(true, kStatTries);
          if (u2 < 0.5f * (1.0f + c * c) || (int)(tries & 0xffffu) >= kMaxTries) {
            float3 d = make_float3(Fv(F_DX, g), Fv(F_DY, g), Fv(F_DZ, g));
            rotate(d, c, uni(k));
            ++k;
            count(true, kStatRayleigh);
            setF(F_DX, g, d.x);
            setF(F_DY, g, d.y);
            setF(F_DZ, g, d.z);
            U(F_CNT, g) = (U(F_CNT, g) + (1u << 16)) | (kDebug ? 0x8000u : 0u);
            U(F_META, g) = (U(F_META, g) & ~7u) | kStep;
          } else {
            U(F_TRIES, g) = tries;
          }
          U(F_K, g) = k;
        }

        // ---- the photon reaches the detector cylinder ----
        if (sec == kEscape) {
          const float px = Fv(F_PX, g), py = Fv(F_PY, g), pz = Fv(F_PZ, g);
          const float dx = Fv(F_DX, g), dy = Fv(F_DY, g), dz = Fv(F_DZ, g);
          const float e = Fv(F_E, g);
          float path = Fv(F_PATH, g);
          const float a = dx * dx + dy * dy;
          int cls = kDetected, cr = 0, rg = 0;
          uint32_t pos = 0;  // LUT position tpos | apos << 16 (scanners with gaps)
          float nx = 0.0f, ny = 0.0f, hz_det = 0.0f;
          if (!(a > 0.0f)) {
            cls = kLostAxial;
          } else {
            const float b = px * dx + py * dy;
            const float c = px * px + py * py - S.r2;
            const float sq = sqrtf(fmaxf(b * b - a * c, 0.0f));
            const float t = (b >= 0.0f) ? (-c) / (b + sq) : (sq - b) / a;
            const float hx = px + t * dx, hy = py + t * dy, hz = pz + t * dz;
            hz_det = hz;
            path += t;
            if (!(hz >= -S.half_len && hz < S.half_len)) {
              cls = kLostAxial;
            } else {
              rg = max(0, min((int)floorf((hz + S.half_len) * S.inv_pitch), S.n_rings - 1));
              float phi = atan2f(hy, hx);
              if (phi < 0.0f) phi += 6.283185307179586f;
              cr = max(0, min((int)floorf(phi * S.crystals_per_radian), S.n_crystals - 1));
              nx = hx / S.radius;
              ny = hy / S.radius;
              float ed = e;  // the energy the window tests: blurred by the resolution, if any
              if (S.e_res_k > 0.0f) {
                ed = e + S.e_res_k * sqrtf(e) * (sqrtf(-2.0f * __logf(uni(k))) * cospif(2.0f * uni(k + 1)));
                k += 2;
              }
              if (ed < S.e_lo || ed > S.e_hi) cls = kEnergyWindow;
              if (S.gap_mode && cls == kDetected) {
                // two words cover both edge draws (the axial one is the second only after a
                // transaxial one); the window holds them since escape_words counts them
                const float u0 = S.gap_mode == 2 ? uni(k) : 0.0f, u1 = S.gap_mode == 2 ? uni(k + 1) : 0.0f;
                const unsigned long long r = place(S, phi, hz, dx, dy, dz, nx, ny, u0, u1);
                if ((uint32_t)r >> 31) {
                  cls = kLostAxial;  // lost in a gap
                } else {
                  cr = (int)((uint32_t)r & 0xffffu);
                  rg = (int)(((uint32_t)r >> 16) & 0x7fffu);
                }
                pos = (uint32_t)(r >> 32);
              }
            }
          }
          count(cls == kDetected, kStatDetected);
          const uint32_t m = U(F_META, g);
          if (cls != kDetected) {
            finish(g, cls, -1, 0);
          } else if (((m >> 3) & 1u) == 0) {  // photon A: keep it, launch photon B back to back
            const uint32_t nint = U(F_CNT, g) >> 16;
            CU(C_ACRG, g) = (uint32_t)cr | (uint32_t)rg << 16 | (nint > 0 ? 1u << 31 : 0u);
            if (S.gap_mode) CU(C_APOS, g) = pos;
            if (kDebug && lm.out) {
              setC(C_AZ, g, hz_det);
              CU(C_ASC, g) = U(F_CNT, g) >> 15;
            }
            setC(C_AE, g, e);
            setC(C_APATH, g, path);
            setC(C_ANX, g, nx);
            setC(C_ANY, g, ny);
            setC(C_ADX, g, dx);
            setC(C_ADY, g, dy);
            setC(C_ADZ, g, dz);
            setF(F_PX, g, Cv(C_E0X, g));
            setF(F_PY, g, Cv(C_E0Y, g));
            setF(F_PZ, g, Cv(C_E0Z, g));
            setF(F_DX, g, -Cv(C_D0X, g));
            setF(F_DY, g, -Cv(C_D0Y, g));
            setF(F_DZ, g, -Cv(C_D0Z, g));
            setF(F_E, g, kEmitKeV);
            setF(F_PATH, g, 0.0f);
            U(F_CNT, g) = 0;
            U(F_K, g) = 0;
            U(F_NB, g) = 0;
            U(F_META, g) = meta(kStep, 1, 2);
          } else if (cr == (int)(CU(C_ACRG, g) & 0xffffu)) {
            finish(g, kSameCrystal, -1, 0);
          } else {
            CU(C_BCRG, g) = (uint32_t)cr | (uint32_t)rg << 16;
            if (S.gap_mode) CU(C_BPOS, g) = pos;
            if (kDebug && lm.out) setC(C_BZ, g, hz_det);
            setC(C_BNX, g, nx);
            setC(C_BNY, g, ny);
            setF(F_PATH, g, path);
            if (blur) {  // the TOF blur reads stream 0, block 2
              U(F_META, g) = meta(kCoinc, 1, 0);
              U(F_K, g) = 8;
              U(F_NB, g) = 2;
            } else {
              U(F_META, g) = meta(kCoinc, 1, 2);
            }
          }
        }

        // ---- coincidence: TOF, LOR bin, LUT weight, accumulate ----
        if (sec == kCoinc) {
          const uint32_t acrg = CU(C_ACRG, g), bcrg = CU(C_BCRG, g);
          const int a_cr = (int)(acrg & 0xffffu), a_rg = (int)((acrg >> 16) & 0x7fffu);
          const int b_cr = (int)(bcrg & 0xffffu), b_rg = (int)(bcrg >> 16);
          const float a_path = Cv(C_APATH, g), path = Fv(F_PATH, g);
          const bool a_first = a_cr < b_cr;
          float delta = 0.5f * (a_first ? a_path - path : path - a_path);
          if (blur) {
            const float gs = sqrtf(-2.0f * logf(uni(8))) * cospif(2.0f * uni(9));
            delta += S.tof_sigma * gs;
          }
          const long long key_ = a_first ? bin_key(S, a_cr, b_cr, a_rg, b_rg, delta)
                                         : bin_key(S, b_cr, a_cr, b_rg, a_rg, delta);
          const bool scattered = (acrg >> 31) != 0u || (U(F_CNT, g) >> 16) > 0u;
          const int cls = key_ < 0 ? kOutOfRange : scattered ? kScatter : kTrue;
          const bool take = cls == kScatter ? (J.bin_mask & 1) : cls == kTrue ? (J.bin_mask & 2) : false;
          long long q = 0;
          if (key_ >= 0 && (take || (kDebug && (J.q_out || lm.out)))) {
            float aa, ab, ba, bb;
            angles(Cv(C_ANX, g), Cv(C_ANY, g), make_float3(Cv(C_ADX, g), Cv(C_ADY, g), Cv(C_ADZ, g)), aa, ab);
            angles(Cv(C_BNX, g), Cv(C_BNY, g), make_float3(Fv(F_DX, g), Fv(F_DY, g), Fv(F_DZ, g)), ba, bb);
            int a_tp = a_cr % S.module_t, a_ap = a_rg % S.module_a, b_tp = b_cr % S.module_t,
                b_ap = b_rg % S.module_a;
            if (S.gap_mode) {
              const uint32_t pa = CU(C_APOS, g), pb = CU(C_BPOS, g);
              a_tp = (int)(pa & 0xffffu);
              a_ap = (int)(pa >> 16);
              b_tp = (int)(pb & 0xffffu);
              b_ap = (int)(pb >> 16);
            }
            const float w = lut_prob<DT>(J.lut, Cv(C_AE, g), aa, ab, a_tp, a_ap, B.dbg) *
                            lut_prob<DT>(J.lut, Fv(F_E, g), ba, bb, b_tp, b_ap, B.dbg);
            q = __float2ll_rn(w * 4294967296.0f);
          }
          if (kDebug && lm.out) {
            const unsigned long long slot = atomicAdd(lm.count, 1ull);
            if (slot < lm.cap) {
              psc_listmode_event* r = lm.out + slot;
              r->history = (unsigned long long)U(F_HHI, g) << 32 | U(F_HLO, g);
              r->q = key_ < 0 ? 0 : q;
              r->voxel = (int)CU(C_VOX, g);
              r->cls = cls;
              r->delta_mm = 0.5f * (a_path - path);
              r->energy_kev[0] = Cv(C_AE, g);
              r->energy_kev[1] = Fv(F_E, g);
              float pa = atan2f(Cv(C_ANY, g), Cv(C_ANX, g)), pb = atan2f(Cv(C_BNY, g), Cv(C_BNX, g));
              r->phi[0] = pa < 0.0f ? pa + 6.283185307179586f : pa;
              r->phi[1] = pb < 0.0f ? pb + 6.283185307179586f : pb;
              r->z_mm[0] = Cv(C_AZ, g);
              r->z_mm[1] = Cv(C_BZ, g);
              r->dir[0][0] = Cv(C_ADX, g);
              r->dir[0][1] = Cv(C_ADY, g);
              r->dir[0][2] = Cv(C_ADZ, g);
              r->dir[1][0] = Fv(F_DX, g);
              r->dir[1][1] = Fv(F_DY, g);
              r->dir[1][2] = Fv(F_DZ, g);
              r->crystal[0] = a_cr;
              r->crystal[1] = b_cr;
              r->ring[0] = a_rg;
              r->ring[1] = b_rg;
              const uint32_t sa = CU(C_ASC, g), sb = U(F_CNT, g) >> 15;
              r->n_scatter[0] = (uint16_t)min(sa >> 1, 65535u);
              r->n_scatter[1] = (uint16_t)min(sb >> 1, 65535u);
              r->rayleigh[0] = (uint8_t)(sa & 1u);
              r->rayleigh[1] = (uint8_t)(sb & 1u);
              for (int b = 0; b < 6; ++b) r->pad[b] = 0;
            }
          }
          // lanes that hit the same bin add their weights first, one atomic per bin
          const unsigned act = __activemask();
          const unsigned takers = __ballot_sync(act, take);
          if (take) {
            const unsigned peers = __match_any_sync(takers, (unsigned long long)key_);
            const unsigned hi = __reduce_add_sync(peers, (unsigned)(q >> 16));
            const unsigned lo = __reduce_add_sync(peers, (unsigned)(q & 0xffff));
            if (lane_id == (unsigned)(__ffs(peers) - 1)) {
              atomicAdd(J.acc + dbg_idx(B.dbg, kSiteAcc, key_,
                                        (long long)S.n_rings * S.n_rings * S.n_views * S.n_rad * S.n_tof),
                        ((unsigned long long)hi << 16) + lo);
              if (stats) atomicAdd(&s_cnt[kStatAtomics], 1ull);
            }
            if (stats) {
              atomicAdd(&s_cnt[kStatBinned], 1ull);
              atomicAdd(&s_cnt[kStatWeight], (unsigned long long)q);
            }
          }
          finish(g, cls, key_, cls == kOutOfRange ? 0 : q);
        }
      }
      __syncwarp();  // slot updates are visible to the lanes that vote on them next
    }

    __syncthreads();  // every slot is done with the chunk before the next fetch
  }

  if (!stats) return;
  __syncthreads();
  for (int i = threadIdx.x; i < kStatCount; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(B.stats + i, s_cnt[i]);
}

size_t transport_cold_words(int grid, int block) {
  return (size_t)grid * kColdFields * (size_t)(block / 32) * kSlotsPerWarp;
}

size_t transport_smem_bytes(const PhantomParams& ph, int block) {
  return sizeof(uint32_t) * kFields * (size_t)(block / 32) * kSlotsPerWarp +
         sizeof(float4) * (size_t)ph.n_mat * ph.n_tab + sizeof(float) * (ph.n_tab + kMaxMaterials);
}

template <int DT, bool kDebug, bool kOneJob = false, bool kFixed = false>
static cudaError_t launch_dt(const BatchParams& p, int grid, int block, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(transport_kernel<DT, kDebug, kOneJob, kFixed>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  transport_kernel<DT, kDebug, kOneJob, kFixed><<<grid, block, smem, s>>>(p);
  return cudaGetLastError();
}

template <int DT>
static cudaError_t launch_dt(const BatchParams& p, int grid, int block, size_t smem, cudaStream_t s) {
  bool debug = p.stats != nullptr;
  for (int j = 0; j < p.n_jobs; ++j)
    debug |= p.jobs[j].cls_out || p.jobs[j].key_out || p.jobs[j].q_out || p.lm[j].out;
  if (debug) return launch_dt<DT, true>(p, grid, block, smem, s);
  if (block != 512) return launch_dt<DT, false>(p, grid, block, smem, s);
  if constexpr (DT == 0) {
    if (p.n_jobs == 1) return launch_dt<0, false, true, true>(p, grid, block, smem, s);
  }
  return launch_dt<DT, false, false, true>(p, grid, block, smem, s);
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

// both instantiations of a LUT type share launch bounds and shared memory.
// The query counts dynamic shared memory above 48 KB only once the kernel
// may use it, so the attribute is set first (else the first launch of a
// kernel would size its grid for one CTA per SM).
template <int DT>
static cudaError_t occupancy_dt(int block, size_t smem, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(transport_kernel<DT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, transport_kernel<DT, false>, block, smem);
}

cudaError_t transport_occupancy(int lut_dtype, int block, size_t smem, int* blocks_per_sm) {
  switch (lut_dtype) {
    case 0: return occupancy_dt<0>(block, smem, blocks_per_sm);
    case 1: return occupancy_dt<1>(block, smem, blocks_per_sm);
    case 2: return occupancy_dt<2>(block, smem, blocks_per_sm);
    default: return occupancy_dt<-1>(block, smem, blocks_per_sm);
  }
}

}  // namespace psc
