/* psc.h -- C ABI of the GB300 PET scatter Monte Carlo library (libpsc.so).
 *
 * The library computes the scatter estimate of Noe et al., "Object
 * independent scatter sensitivities for PET, applied to scatter estimation
 * through fast Monte Carlo simulation" (arXiv 2509.05047), Sec. 2.2:
 * annihilation photon pairs are emitted from an activity image and
 * transported through a known attenuation image (Sec. 2.3, step 2 of the
 * joint estimation loop in Sec. 2.3.3), detected on a cylinder that keeps
 * every photon crossing it (Sec. 2.2.1), weighted by the product of the two
 * photons' 5D detection probabilities (Sec. 2.2.1-2.2.2), binned into an
 * LOR x TOF sinogram, optionally smoothed with a normalisation sinogram
 * (Sec. 2.3.2) and multiplied by the scatter-sensitivity sinogram
 * (Sec. 2.2.4).
 *
 * Conventions
 *   - Units: mm, keV, g/cm^3, cm^2/g, degrees.
 *   - Every call returns PSC_OK (0) or a negative PSC_E* code; the message of
 *     the calling thread's last failure is psc_last_error().  No exception or
 *     abort crosses the ABI.
 *   - "host" pointers are read during the call and may be freed after it;
 *     "device" pointers are caller-owned CUDA device memory on the context's
 *     device (for example a torch tensor's data_ptr()).
 *   - Calls that take a stream enqueue work on it asynchronously; a NULL
 *     stream is the legacy default stream.
 *   - Objects (scanner, materials, phantom, LUT, sinogram, accumulator) are
 *     copied to device memory owned by the context until psc_unload or
 *     psc_destroy; they are identified by positive int32 ids.
 *   - Array layouts: voxels [nz][ny][nx]; LUT [apos][tpos][E][alpha][beta];
 *     sinograms [plane][view][radial][tof] with plane = ring_a * n_rings +
 *     ring_b; per-LOR inputs [plane][view][radial] apply to every TOF bin.
 *   - Stream capture: psc_acc_zero, psc_acc_read / write, psc_simulate and
 *     psc_simulate_batch (without stats), psc_simulate_batch_tuned (on a
 *     request mix it has already tuned) and psc_finalize (psc_finalize_host
 *     with copy_stream == stream) can be captured into a CUDA graph on one
 *     stream, after the same calls have run once outside the capture (their
 *     working buffers are allocated then; a capture cannot allocate or wait,
 *     and such a call returns PSC_EINVAL).  Captured launches take their order
 *     from the graph: replays are not ordered against the context's other
 *     launches, or against psc_update_activity, except by the caller (for
 *     example, one stream).
 */
#ifndef PSC_H
#define PSC_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PSC_OK = 0,
  PSC_EINVAL = -1,    /* invalid argument */
  PSC_ENOMEM = -2,    /* device memory or admission budget exhausted */
  PSC_ENOTFOUND = -3, /* unknown object id or wrong object kind */
  PSC_ETIMEOUT = -4,  /* a bounded wait expired */
  PSC_EDEVICE = -5,   /* CUDA error */
  PSC_EOVERFLOW = -6  /* fixed-point headroom or size limit exceeded */
};

/* history classes (psc_stats.class_counts and listmode output) */
enum {
  PSC_CLASS_ABSORBED = 0,      /* a photon was photo-absorbed */
  PSC_CLASS_LOST_AXIAL = 1,    /* a photon missed the cylinder's axial extent */
  PSC_CLASS_ENERGY_WINDOW = 2, /* a photon's energy left [e_lo, e_hi] */
  PSC_CLASS_STEP_LIMIT = 3,    /* safety bound of 4096 tracking steps reached */
  PSC_CLASS_SAME_CRYSTAL = 4,  /* both photons in one transaxial crystal */
  PSC_CLASS_OUT_OF_RANGE = 5,  /* TOF or clipped radial bin outside the sinogram */
  PSC_CLASS_TRUE = 6,          /* both detected, neither interacted */
  PSC_CLASS_SCATTER = 7        /* both detected, >= 1 Compton or Rayleigh event */
};

enum { PSC_LUT_F32 = 0, PSC_LUT_F16 = 1, PSC_LUT_BF16 = 2 };
enum { PSC_BIN_SCATTER = 1, PSC_BIN_TRUES = 2 };

typedef struct psc_ctx psc_ctx;
typedef void* psc_stream; /* a cudaStream_t */

/* Cylindrical scanner at the depth of interaction (Sec. 2.1.1, 2.2.1). */
typedef struct {
  double radius;        /* cylinder radius (mm) */
  double ring_pitch;    /* axial ring pitch (mm); axial extent n_rings * ring_pitch, centred */
  int32_t n_crystals;   /* crystals per ring, even; crystal c spans azimuth [2 pi c/N, 2 pi (c+1)/N) */
  int32_t n_rings;
  int32_t module_t;     /* LUT transaxial position = crystal mod module_t */
  int32_t module_a;     /* LUT axial position = ring mod module_a */
  double e_lo, e_hi;    /* energy window (keV) */
  int32_t n_tof;        /* TOF bins of (l_a - l_b)/2, bin t covers [(t - n_tof/2) w, (t + 1 - n_tof/2) w) */
  int32_t n_rad;        /* radial bins kept: centred clip of the n_crystals - 1 bins (same parity) */
  double tof_bin_mm;    /* w (mm) */
  double tof_sigma_mm;  /* Gaussian TOF blur sigma of (l_a - l_b)/2 (mm), 0 = none */
  double e_res_fwhm;    /* energy resolution: FWHM as a fraction of 511 keV at 511 keV, scaling as
                           sqrt(E) (the no-LUT mode of Sec. 2.2.1 uses 0.112 with a 425-650 keV
                           window); 0 = exact energies.  The window tests the blurred energy; a
                           Compton-scattered photon is dropped below e_lo - 5 sigma(e_lo). */
  /* Gaps between detector modules and blocks (Sec. 2.2.1-2.2.2, Figs. "crystals" and "gap
   * assignment").  gap_mode 0: crystals fill the ring and the axial extent.  1 or 2: the
   * ring holds n_crystals / module_t modules and the axial extent n_rings / module_a blocks,
   * each [half gap | crystals | half gap]; LUT positions are module-local 0 .. module_t + 1
   * (0 and module_t + 1 are the virtual crystals of the half gaps) and block * (module_a + 2)
   * + 0 .. module_a + 1.  Mode 1 loses photons in a gap.  Mode 2 gives them the LUT value
   * of their virtual crystal, then one random word assigns them to one of the gap's two
   * edge crystals with the relative detection probability of the two blocks: from the path
   * lengths l1, l2 of the photon's line through the blocks, 1 - exp(-mu l) for the block it
   * meets first and exp(-mu l_first) (1 - exp(-mu l)) for the other. */
  int32_t gap_mode;
  double gap_t_mm;          /* transaxial gap width at the detection radius */
  double gap_a_mm;          /* axial gap width between blocks */
  double crystal_depth_mm;  /* crystal length along the radius */
  double doi_mm;            /* depth of the detection cylinder below the block face */
  double mu_block;          /* attenuation coefficient of the crystals (1/mm) */
} psc_scanner_desc;

/* Materials: mass attenuation tables on the grid E = 0, 1, ..., n_e-1 keV
 * (n_e >= 512), host arrays [n_mat][n_e]; 1 <= n_mat <= 8. */
typedef struct {
  int32_t n_mat;
  int32_t n_e;
  const double* compton;   /* host */
  const double* rayleigh;  /* host */
  const double* photo;     /* host */
  const double* kappa;     /* host [n_mat]: Rayleigh form factor (1 + b s)^-2, b = kappa (E/511)^2 */
} psc_materials_desc;

/* Voxel phantom: attenuation (material id + density) and activity. */
typedef struct {
  int32_t nx, ny, nz;
  double dx, dy, dz;           /* voxel size (mm) */
  double ox, oy, oz;           /* min corner of voxel (0,0,0) (mm); grid must lie inside the cylinder */
  const uint8_t* material;     /* host [nz][ny][nx], ids < n_mat of the materials object */
  const float* density;        /* host [nz][ny][nx] g/cm^3, >= 0 */
  const float* activity;       /* host [nz][ny][nx], >= 0, positive sum */
} psc_phantom_desc;

/* 5D single-photon detection-probability LUT (Sec. 2.2.2), multilinear in energy and the
 * two angles, exact in the crystal position.  The lower-dimensional LUTs of Sec. 2.2.2
 * (energy only; energy and angles; energy and crystals) are LUTs with one bin on each axis
 * they drop: constant along an angle axis, position 0 for every photon on a position axis. */
typedef struct {
  int32_t n_e, n_a, n_b;       /* energy, transaxial angle, axial angle bins */
  int32_t n_tpos, n_apos;      /* the scanner's LUT positions: module_t, module_a without gaps,
                                  module_t + 2, n_blocks (module_a + 2) with gaps; or 1 */
  double e_min, e_max;         /* keV; nodes at bin centres */
  double a_min, a_max;         /* deg */
  double b_min, b_max;         /* deg */
  int32_t dtype;               /* device storage: PSC_LUT_F32 / F16 / BF16 (rounded to nearest) */
  const float* data;           /* host [n_apos][n_tpos][n_e][n_a][n_b] in [0, 1] */
} psc_lut_desc;

/* Listmode record of one coincidence (Sec. 2.2.1: the simulator's list of non-random
 * coincidences), written by the debug path when psc_sim_args.lm_out is set: every
 * history whose two photons are detected inside the window in different crystals,
 * whatever its LOR/TOF bin.  Photon A travels along the emission direction, B against it.
 * 104 bytes, no implicit padding. */
typedef struct {
  uint64_t history;            /* history index */
  int64_t q;                   /* fixed-point weight rint(w 2^32) (0 when out of range) */
  int32_t voxel;               /* emission voxel, x fastest */
  int32_t cls;                 /* PSC class: 5 out of range, 6 true, 7 scatter */
  float delta_mm;              /* (path_A - path_B) / 2, before the TOF blur: the emission-time
                                  difference of the two detections times c / 2 */
  float energy_kev[2];         /* exact energies at detection */
  float phi[2];                /* azimuth of the hit on the detection cylinder, [0, 2 pi) */
  float z_mm[2];               /* axial coordinate of the hit */
  float dir[2][3];             /* unit directions at detection */
  int32_t crystal[2], ring[2]; /* assigned crystal and ring (after gap handling) */
  uint16_t n_scatter[2];       /* Compton + Rayleigh interactions (saturating at 65535) */
  uint8_t rayleigh[2];         /* 1 if any of them was a Rayleigh interaction */
  uint8_t pad[6];
} psc_listmode_event;

/* One simulation call (Sec. 2.2.1): histories [first_history,
 * first_history + n_histories) of the counter-based random stream keyed by
 * seed.  The result is independent of launch shape and of how the history
 * range is split across calls. */
typedef struct {
  uint64_t seed;
  uint64_t first_history;
  uint64_t n_histories;
  int32_t scanner, phantom, lut;   /* lut = 0: no LUT (every coincidence weighs 1) */
  int32_t acc;                     /* accumulator to add into */
  int32_t bin_mask;                /* PSC_BIN_SCATTER | PSC_BIN_TRUES; 0 = scatter */
  int32_t block, grid;             /* launch shape: block a multiple of 32 in [32, 512]; 0 = automatic */
  int8_t* cls_out;                 /* device [n_histories] history class, or NULL */
  int64_t* key_out;                /* device [n_histories] sinogram bin (-1 unless true/scatter), or NULL */
  int64_t* q_out;                  /* device [n_histories] fixed-point weight rint(w 2^32), or NULL */
  psc_listmode_event* lm_out;      /* device [lm_capacity] coincidence records, or NULL */
  uint64_t* lm_count;              /* device counter, required with lm_out: the call adds its number of
                                      coincidences; record k lands at lm_out[k] while k < lm_capacity
                                      (in no particular order; sort by history) */
  uint64_t lm_capacity;
} psc_sim_args;

typedef struct {
  uint64_t class_counts[8];
  uint64_t steps;                  /* Woodcock tracking steps (real + virtual) */
  uint64_t compton, rayleigh, photo;
  uint64_t binned;                 /* events added to the accumulator */
  uint64_t weight_sum;             /* sum of their fixed-point weights */
  uint64_t rng_blocks;             /* Philox4x32-10 blocks generated */
  uint64_t tries;                  /* Compton and Rayleigh rejection-sampling tries */
  uint64_t detected;               /* photons that reached the detector inside the window */
  uint64_t atomics;                /* global atomics issued (events of a warp in one bin share one) */
  int32_t grid, block;             /* launch shape of the call's (last) transport launch */
} psc_stats;

/* Sinogram post-processing (Sec. 2.2.4, 2.3.2). */
typedef struct {
  int32_t acc;
  int32_t sens;                    /* sensitivity sinogram id, 0 = none (1) */
  int32_t norm;                    /* smoothing-normalisation sinogram id, 0 = none */
  int32_t smooth;                  /* 0: no smoothing; 1: sigma applies */
  double sigma[3];                 /* Gaussian sigma in bins: radial, view, axial (within segment) */
  double scale;                    /* global factor (e.g. 1/histories, decay, Sec. 2.4.3) */
  int32_t sens_first;              /* 0 (paper order): smooth, then x sens; 1: x sens, then smooth */
  int32_t seg_lo, seg_hi;          /* finalize only the planes of ring-difference segments [seg_lo,
                                      seg_hi), segment rb - ra + n_rings - 1 (smoothing never crosses
                                      a segment, so each part is exact on its own; the output's other
                                      planes are unspecified, since out also serves as working
                                      memory); seg_lo == seg_hi: every plane */
} psc_finalize_args;

/* Context on one CUDA device.  mem_budget_bytes bounds the device memory of
 * resident objects (0 = no bound). */
int psc_create(psc_ctx** out, int32_t device, uint64_t mem_budget_bytes);
void psc_destroy(psc_ctx* ctx);
/* Message of the calling thread's last failed call ("" if none). */
const char* psc_last_error(void);

/* Scanner geometry (Sec. 2.1.1, 2.2.1). */
int psc_load_scanner(psc_ctx* ctx, const psc_scanner_desc* desc, int32_t* id);
/* Material cross-section tables (the simulator's physics input; Sec. 2.2.1). */
int psc_load_materials(psc_ctx* ctx, const psc_materials_desc* desc, int32_t* id);
/* Attenuation + activity images (Fig. "schematic sensitivities": the
 * simulator's two inputs); builds the emission alias table (FP64) and the
 * Woodcock majorant for this phantom. */
int psc_load_phantom(psc_ctx* ctx, const psc_phantom_desc* desc, int32_t materials, int32_t* id);
/* New activity image for a loaded phantom (joint activity/scatter
 * estimation, Sec. 2.3.3 step 2): rebuilds the alias table only.  Builds it
 * on the host, waits (host-side) for the transport launches issued so far
 * that read this phantom, then uploads it; other device work, on any
 * stream, keeps running.  Launches issued after the call returns use the
 * new image. */
int psc_update_activity(psc_ctx* ctx, int32_t phantom, const float* activity /* host */);
/* Copy a phantom's resident emission alias table to host arrays of n_vox
 * entries: column v is kept when (x >> 9) < threshold[v] for the Philox word
 * x of the acceptance draw (equivalently u < prob[v] of Vose's table), else
 * alias[v] is emitted. */
int psc_phantom_alias(psc_ctx* ctx, int32_t phantom, uint32_t* threshold /* host */,
                      int32_t* alias /* host */);
/* Detection-probability LUT (Sec. 2.2.2); data == NULL loads a LUT of ones. */
int psc_load_lut(psc_ctx* ctx, const psc_lut_desc* desc, int32_t* id);
/* Sensitivity (Sec. 2.2.4) or smoothing-normalisation (Sec. 2.3.2) sinogram
 * for a scanner: host f64, per_lor = 1 for [plane][view][rad], 0 for the
 * full [plane][view][rad][tof]. */
int psc_load_sinogram(psc_ctx* ctx, int32_t scanner, const double* host, int32_t per_lor,
                      int32_t* id);
/* int64 fixed-point accumulator sinogram (weight w adds rint(w * 2^32)). */
int psc_acc_create(psc_ctx* ctx, int32_t scanner, int32_t* id);
int psc_acc_zero(psc_ctx* ctx, int32_t acc, psc_stream stream);
/* An accumulator in caller-owned device memory (int64, the scanner's
 * sinogram size, 8-byte aligned, on the context's device): the context uses
 * it like one of psc_acc_create (simulate into it, finalize it) but neither
 * zeroes nor frees it, and it does not count against the memory budget.
 * For callers that exchange accumulators themselves, e.g. the sum over the
 * ranks that simulate parts of one request's histories, without a copy.
 * The memory must stay valid until psc_unload of the id. */
int psc_acc_wrap(psc_ctx* ctx, int32_t scanner, int64_t* device, int32_t* id);
/* Copy the raw accumulator out / in (checkpoint and resume): device int64
 * arrays of the scanner's sinogram size. */
int psc_acc_read(psc_ctx* ctx, int32_t acc, int64_t* out /* device */, psc_stream stream);
int psc_acc_write(psc_ctx* ctx, int32_t acc, const int64_t* in /* device */, psc_stream stream);
/* Simulate and accumulate (Sec. 2.2.1-2.2.3).  stats may be NULL; when
 * given, the call waits for the stream and fills it. */
int psc_simulate(psc_ctx* ctx, const psc_sim_args* args, psc_stats* stats, psc_stream stream);
/* Several requests in one persistent launch (continuous batching of uneven
 * requests): args[0..n) may use different scanners, phantoms, LUTs and
 * accumulators; their histories are split into work items that the GPU's
 * CTAs take in turn, so small and large requests share the device.  Each
 * request's accumulator receives exactly what psc_simulate would add alone.
 * The launch shape is args[0].block / args[0].grid; stats (if given) sum
 * over the batch. */
int psc_simulate_batch(psc_ctx* ctx, const psc_sim_args* args, int32_t n, psc_stats* stats,
                       psc_stream stream);
/* Launch schedule of a batched transport launch. */
typedef struct {
  int32_t block;            /* threads per CTA */
  int32_t grid;             /* CTAs (0: as many as fit on the device) */
  int32_t chunks_per_cta;   /* work items per CTA and request */
  int32_t max_chunk;        /* histories per work item at most */
  double rate;              /* histories/s this schedule reached in the probes */
  int32_t probed;           /* schedules timed by this call (0: the choice was cached) */
} psc_schedule;
/* psc_simulate_batch with a launch schedule picked by timed probes (no
 * counterpart in the paper): a few candidate schedules (CTA size, work items
 * per CTA, largest work item) each run the next slice of every request's
 * histories (1/48 of each budget), and the fastest runs the rest.  Every
 * history is simulated exactly once into its request's accumulator and
 * accumulators do not depend on the schedule, so the result equals
 * psc_simulate_batch's bit for bit.  The choice is cached per request mix
 * (the requests' scanner, phantom and LUT objects), so later calls on the
 * mix skip the probes.  The probes wait for the stream (host-side).  No
 * per-history outputs (cls_out, key_out, q_out, lm_out): PSC_EINVAL.
 * chosen (may be NULL) receives the schedule. */
int psc_simulate_batch_tuned(psc_ctx* ctx, const psc_sim_args* args, int32_t n, psc_schedule* chosen,
                             psc_stream stream);
/* Scatter estimate = acc * scale * 2^-32, [x norm -> smooth -> / norm],
 * x sens (Sec. 2.2.4, 2.3.2), written to out (device f64, sinogram size).
 * With smoothing, out also serves as the first pass's FP32 working buffer
 * until the last pass overwrites it.  Smoothing supports up to 255 rings
 * and (2 n_rings - 1) * n_crystals / 2 <= 65535, else PSC_EINVAL.  Where the
 * shape allows, the axial pass stages its tiles in shared memory by TMA
 * copies whose waits are bounded; a wait that runs out stops that pass (its
 * estimate is then incomplete) and the next finalize call on the context
 * returns PSC_EDEVICE.  PSC_AXIAL_TMA=0 in the environment switches the
 * staging off (same results). */
int psc_finalize(psc_ctx* ctx, const psc_finalize_args* args, double* out /* device */,
                 psc_stream stream);
/* The scatter estimate of psc_finalize delivered to host memory (the
 * end-to-end form for a caller that takes the estimate out of the device,
 * e.g. to hand it to a reconstruction on the host).  work: device f64 of
 * the scanner's sinogram size, holding the estimate (and the smoothing's
 * first FP32 pass) as psc_finalize's out does; out_host: host f64 of the
 * same size, best page-locked (psc_host_alloc gives the host link's rate).
 * The estimate is computed in parts (plane ranges without smoothing; the
 * axial pass in groups of whole ring-difference segments with it), and each
 * part is copied to out_host on copy_stream as soon as it is written, so
 * the transfer overlaps the rest of the finalize.  Kernels are enqueued on
 * stream; copy_stream (may be the same stream) waits for each part and
 * copies it: when copy_stream has reached the end of this call's work,
 * out_host holds the estimate.  work must not be overwritten before then
 * (order the next writer after an event on copy_stream).  Errors as
 * psc_finalize, and PSC_EINVAL for a NULL out_host. */
int psc_finalize_host(psc_ctx* ctx, const psc_finalize_args* args, double* work /* device */,
                      double* out_host /* host */, psc_stream stream, psc_stream copy_stream);
/* Smoothing-normalisation sinogram (Sec. 2.3.2: a heavily smoothed copy of
 * a sinogram divided by the sinogram itself, made once from the simulation
 * of a large cylinder): out[bin] = smooth(acc)[bin] / acc[bin], 0 where
 * acc[bin] == 0; sigma (host [3], bins: radial, view, axial) as in
 * psc_finalize_args.  out: device f64 of the scanner's sinogram size, used
 * as working memory until the last pass writes it.  The ratio is computed
 * in FP32 (the smoothed value's precision) and widened exactly.  Load it
 * with psc_load_sinogram (per bin) to use it as the normalisation. */
int psc_norm_sinogram(psc_ctx* ctx, int32_t acc, const double* sigma, double* out /* device */,
                      psc_stream stream);
/* Mashing (Sec. 4 lists it to need fewer counts and less smoothing): sums
 * view_factor adjacent views and tof_factor adjacent TOF bins of an
 * accumulator into out, device int64 [planes][views / view_factor][n_rad]
 * [n_tof / tof_factor]; the factors must divide the view and TOF counts.
 * Exact integer sums. */
int psc_acc_mash(psc_ctx* ctx, int32_t acc, int32_t view_factor, int32_t tof_factor,
                 int64_t* out /* device */, psc_stream stream);
/* Span (segment) mashing (Sec. 4 lists mashing among the ways to need fewer
 * counts and less smoothing; the paper gives no details, and the usual
 * Michelogram span is the reading): ring differences d = rb - ra are
 * grouped into segments of span (odd) consecutive values, segment k
 * (k = -K..K) holding [k span - (span-1)/2, k span + (span-1)/2] within the
 * ring range, and the planes of a segment with the same axial sum
 * z = ra + rb are added.  A segment's output planes run over z from its
 * smallest |d| to 2 n_rings - 2 minus it (every other z when it holds a
 * single ring difference); segments follow in order k = -K..K.  out: device
 * int64 [out_planes][n_crystals / 2][n_rad][n_tof], or NULL to query the
 * count; *out_planes (may be NULL) receives the number of output planes
 * (2025 -> 1379 for 45 rings at span 3; span 1 reorders the planes).  Exact
 * integer sums, each input plane read once.  PSC_EINVAL for an even span. */
int psc_acc_span(psc_ctx* ctx, int32_t acc, int32_t span, int64_t* out /* device */, int64_t* out_planes,
                 psc_stream stream);
/* Sum over the scanner's rotational symmetries (Sec. 2.2.4 averages the
 * sensitivity sinograms over 14 of them): out_acc = sum over the
 * n_crystals / step rotations by k * step crystals (step = crystals per
 * module) of acc at the rotated LOR; when a rotation reverses the crystal
 * order the rings swap and the TOF bin mirrors.  The orbit of an LOR visits
 * n_crystals / (2 step) views (14 for 448 crystals in modules of 16), each
 * twice.  Exact integer sums; the average is this sum with finalize scale
 * 1 / (n_crystals / step).  out_acc: another accumulator of the same
 * scanner; at most 255 rings. */
int psc_acc_rotate_sum(psc_ctx* ctx, int32_t acc, int32_t step, int32_t out_acc, psc_stream stream);
/* Allocation-free variant of psc_finalize for callers that cannot allocate
 * device memory (their device memory belongs to another allocator, is
 * capped, or must not be allocated once a real-time loop is running).  The
 * paper has no counterpart.  Inputs and the output are the caller's device
 * arrays: acc int64 and out f64 of n_rings^2 x (n_crystals/2) x n_rad x
 * n_tof bins (n_crystals even, n_rad in [1, n_crystals - 1] with
 * n_crystals - 1 - n_rad even, as for psc_load_scanner; else PSC_EINVAL);
 * sens / norm (NULL = none) per LOR when *_per_lor, else per bin; sigma
 * (host [3], NULL = no smoothing), scale and sens_first as in
 * psc_finalize_args.  The smoothing's working memory is one static device
 * array of 64 MiB per GPU: sinograms needing more than 4 bytes per bin plus
 * 8 per normalisation value (256-byte aligned) are rejected with
 * PSC_EOVERFLOW.  The calls make no cudaMalloc, cudaFree or allocating
 * library call.  The array lives in this library's image, and with CUDA's
 * default lazy module loading it is mapped on a device when the first
 * smoothing call on that device looks up its address
 * (cudaGetSymbolAddress): that first call takes 64 MiB of device memory
 * (plus the allocation granularity), later calls none, and the array stays
 * until the process exits.  So make the first call before another
 * allocator reserves the device's memory, or run with
 * CUDA_MODULE_LOADING=EAGER (the array is then mapped with the context);
 * it should also come before any stream capture.  The address is cached
 * per device for the life of the process: a device reset (cudaDeviceReset)
 * between calls is not supported.  All calls on a device share the array
 * and every call overwrites all of it that it reads, so nothing needs
 * clearing; calls that overlap on the GPU (other streams, other threads)
 * race on it and must be ordered by the caller. */
int psc_finalize_static(const int64_t* acc, int32_t n_rings, int32_t n_crystals, int32_t n_rad,
                        int32_t n_tof, const double* sens, int32_t sens_per_lor,
                        const double* norm, int32_t norm_per_lor, const double* sigma,
                        double scale, int32_t sens_first, double* out, psc_stream stream);
/* Free one object. */
int psc_unload(psc_ctx* ctx, int32_t id);
/* Voxel count of a loaded phantom (negative PSC_E* code on error). */
int64_t psc_phantom_voxels(psc_ctx* ctx, int32_t phantom);

/* ---- Request server (continuous batching) -------------------------------
 * One scatter estimate per request, as issued by each iteration of the joint
 * activity/scatter estimation (Sec. 2.3.3): simulate n_histories of a
 * resident phantom (optionally with a new activity image), then finalize
 * into the caller's device buffer.  A server thread admits requests when an
 * accumulator for their scanner fits the context's memory budget, runs every
 * active request's next slice of histories in one batched launch per epoch
 * (requests that arrive meanwhile join at the next epoch), and finalizes
 * finished requests on a second stream.  Each result is the same as when the
 * request runs alone. */
typedef struct {
  int32_t scanner, phantom, lut;   /* resident objects (lut 0: none) */
  uint64_t seed, first_history, n_histories;
  int32_t sens, norm, smooth;      /* as psc_finalize_args */
  double sigma[3];
  double scale;
  int32_t sens_first;
  double* out;                     /* device f64, the scanner's sinogram size; written on the
                                      server's streams, so no other work may be pending on it */
  const float* activity;           /* host [n_vox] new activity image; its alias table is built by
                                      psc_submit on the calling thread; NULL keeps the current one */
} psc_request;

typedef struct {
  int32_t max_active;              /* requests simulating at once */
  uint64_t epoch_histories;        /* histories per epoch, shared by the active requests */
  uint64_t min_slice;              /* smallest per-request slice of an epoch (0: 65536) */
} psc_server_config;

enum { PSC_REQ_WAITING = 0, PSC_REQ_ACTIVE = 1, PSC_REQ_FINALIZING = 2, PSC_REQ_DONE = 3,
       PSC_REQ_FAILED = 4 };

typedef struct {
  int32_t state;                   /* PSC_REQ_* */
  int32_t error;                   /* PSC_E* code of a failed request */
  double t_submit, t_start, t_done;  /* seconds since the server started */
} psc_request_status;

int psc_server_start(psc_ctx* ctx, const psc_server_config* cfg);
/* Finish every submitted request, then stop the server thread. */
int psc_server_stop(psc_ctx* ctx);
int psc_submit(psc_ctx* ctx, const psc_request* req, uint64_t* ticket);
int psc_poll(psc_ctx* ctx, uint64_t ticket, psc_request_status* status);
/* Block until the request is done (PSC_OK), failed (its error code) or
 * timeout_us microseconds have passed (PSC_ETIMEOUT). */
int psc_wait(psc_ctx* ctx, uint64_t ticket, int64_t timeout_us);
/* Bytes of device memory held by the context's objects. */
uint64_t psc_resident_bytes(const psc_ctx* ctx);

/* Page-locked host memory for reading results back (the finalized scatter estimate of
 * Sec. 2.3 is 8 bytes per sinogram bin, 43.8 GB at the paper's scale).  The buffer is
 * anonymous memory aligned to and advised for transparent huge pages, faulted in, and
 * registered with CUDA for every device (cudaHostRegister, portable).  Huge pages keep
 * the device's translations of the buffer few, so device-to-host copies into it run at
 * the host link's rate even while kernels run.  Its initial contents are unspecified
 * (faulted in with a nonzero byte per base page, so that the kernel does not take its
 * huge pages for unused zero pages and split them).  Independent of any context.
 *   bytes: size (> 0; rounded up to whole huge pages).  *ptr: the buffer, owned by the
 *   caller until psc_host_free.  Errors: PSC_EINVAL (NULL ptr, 0 bytes), PSC_ENOMEM
 *   (mapping failed), PSC_EDEVICE (registration failed; nothing is left allocated). */
int psc_host_alloc(uint64_t bytes, void** ptr);
/* Unregister and unmap a buffer of psc_host_alloc.  PSC_EINVAL for any other pointer
 * (nothing is freed). */
int psc_host_free(void* ptr);

#ifdef __cplusplus
}
#endif
#endif
