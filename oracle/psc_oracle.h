/* psc_oracle.h -- FP64 CPU oracle of the PET scatter Monte Carlo path.
 *
 * TEST INFRASTRUCTURE.  This is the plain, slow reference that the CUDA
 * library is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * What it computes (the scatter estimate of Sec. 2.2 / Fig. "schematic
 * sensitivities"): annihilation pairs are emitted from an activity image,
 * transported through an attenuation image, detected on a cylinder
 * (Sec. 2.2.1), weighted by the product of the two photons' 5D detection
 * probabilities (Sec. 2.2.1-2.2.2) and binned into an LOR x TOF sinogram.
 * The sinogram post-processing (sensitivity multiply Sec. 2.2.4, smoothing
 * Sec. 2.3.2) lives in oracle/sinogram.py.
 *
 * Units: mm, keV, g/cm^3, cm^2/g, degrees.
 */
#ifndef PSC_ORACLE_H
#define PSC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* history classes (first failing photon wins; photon 1 before photon 2) */
enum {
  ORC_ABSORBED = 0,      /* photo-absorbed in the phantom */
  ORC_LOST_AXIAL = 1,    /* missed the cylinder's axial extent */
  ORC_ENERGY_WINDOW = 2, /* energy left the window [e_lo, e_hi] */
  ORC_STEP_LIMIT = 3,    /* safety bound on tracking steps reached */
  ORC_SAME_CRYSTAL = 4,  /* both photons in one transaxial crystal */
  ORC_OUT_OF_RANGE = 5,  /* TOF bin (or clipped radial bin) outside the sinogram */
  ORC_TRUE = 6,          /* both detected, neither interacted */
  ORC_SCATTER = 7,       /* both detected, >= 1 Compton or Rayleigh event */
  ORC_N_CLASSES = 8,
  ORC_DETECTED = 15      /* photon status: reached the detector in the window */
};

typedef struct {
  double radius;       /* cylinder radius (mm) */
  double ring_pitch;   /* axial ring pitch (mm); axial extent L = n_rings * ring_pitch centred on z = 0 */
  int32_t n_crystals;  /* crystals per ring (even) */
  int32_t n_rings;
  int32_t module_t;    /* LUT transaxial position = crystal mod module_t */
  int32_t module_a;    /* LUT axial position = ring mod module_a */
  double e_lo, e_hi;   /* energy window (keV) */
  int32_t n_tof;
  int32_t n_rad;       /* radial bins kept (centred clip of the n_crystals-1 bins) */
  double tof_bin_mm;   /* TOF bin width of (l_a - l_b)/2 (mm) */
  double tof_sigma_mm; /* Gaussian blur sigma of (l_a - l_b)/2 (mm); 0 = none */
  double e_res;        /* energy resolution, FWHM as a fraction of 511 keV at 511 keV, scaling
                          as sqrt(E); 0 = exact energies.  The window then tests the blurred
                          energy, and a Compton photon is dropped below e_lo - 5 sigma(e_lo). */
  /* Gaps between detector modules (Sec. 2.2.1-2.2.2, Figs. "crystals" and "gap assignment").
   * gap_mode 0: crystals fill the ring and the axial extent (no gaps).  1 or 2: the ring
   * holds n_crystals / module_t modules and the axial extent n_rings / module_a blocks;
   * each module (block) is [half gap | module_t crystals (module_a rings) | half gap], and
   * LUT positions are the module-local index 0 .. module_t + 1 (0 and module_t + 1: the
   * virtual crystals of the half gaps) and block * (module_a + 2) + local index 0 ..
   * module_a + 1.  Mode 1 loses photons in a gap; mode 2 gives them the LUT probability of
   * their virtual crystal and then assigns them to one of the two edge crystals of the gap
   * with the relative detection probability of the two blocks (see orc_edge_prob). */
  int32_t gap_mode;
  double gap_t;          /* transaxial gap between modules (mm at the detection radius) */
  double gap_a;          /* axial gap between blocks (mm) */
  double crystal_depth;  /* crystal length along the radius (mm) */
  double doi;            /* depth of the detection cylinder below the block face (mm) */
  double mu_block;       /* attenuation coefficient of the crystals (1/mm) */
} orc_scanner;

typedef struct {
  int32_t n_mat;
  int32_t n_e;             /* table nodes at E = 0,1,...,n_e-1 keV */
  const double* compton;   /* [n_mat][n_e] mass attenuation (cm^2/g) */
  const double* rayleigh;  /* [n_mat][n_e] */
  const double* photo;     /* [n_mat][n_e] */
  const double* kappa;     /* [n_mat] Rayleigh form-factor parameter */
} orc_materials;

typedef struct {
  int32_t nx, ny, nz;
  double dx, dy, dz;       /* voxel size (mm) */
  double ox, oy, oz;       /* min corner of voxel (0,0,0) (mm) */
  const uint8_t* material; /* [nz][ny][nx] */
  const float* density;    /* [nz][ny][nx] g/cm^3 */
} orc_phantom;

typedef struct {
  int32_t n_e, n_a, n_b, n_tpos, n_apos;
  double e_min, e_max;     /* energy axis (keV): n_e bins, nodes at bin centres */
  double a_min, a_max;     /* transaxial incidence angle axis (deg) */
  double b_min, b_max;     /* axial incidence angle axis (deg) */
  const float* data;       /* [n_apos][n_tpos][n_e][n_a][n_b]; NULL => probability 1 */
  /* Lower-dimensional LUTs (Sec. 2.2.2: energy only; energy and angles; energy and
   * crystals) have one bin on each axis they drop: constant along an angle axis, and
   * position 0 for every photon on a position axis (n_tpos or n_apos = 1). */
} orc_lut;

/* Per-history listmode record (the simulator's listmode of Sec. 2.2.1 plus
 * the detector assignment of the unlisting step). */
typedef struct {
  int32_t cls, voxel, view, rad, plane, tof;
  int64_t key;             /* sinogram bin, -1 unless cls is TRUE or SCATTER */
  int64_t q;               /* rint(w * 2^32), 0 unless cls is TRUE or SCATTER */
  double w;                /* p_a * p_b */
  double delta;            /* (l_a - l_b)/2 (+ TOF blur) (mm) */
  double emit[3];          /* emission point */
  double dir[3];           /* initial direction of photon 1 (photon 2 = -dir) */
  int32_t status[2], crystal[2], ring[2], n_compton[2], n_rayleigh[2], n_steps[2];
  double energy[2], alpha[2], beta[2], path[2], prob[2];
  double hit[2][3];        /* detector cylinder hit point */
  double exit_pos[2][3];   /* last position inside the phantom grid */
  double exit_dir[2][3];   /* direction at detection */
  /* first Compton interaction of photon 1 (zeros if none) */
  double c_e_before, c_e_after, c_dir_before[3], c_dir_after[3];
  double e_det[2];         /* energy the window tested (blurred when e_res > 0) */
} orc_record;

/* Philox4x32-10 block function (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Vose alias table over n weights (FP64).  Returns 0, or -1 if the weights
 * are not finite and non-negative with a positive sum. */
int orc_alias_build(const float* weight, int64_t n, double* prob, int32_t* alias);

/* Woodcock majorant per energy node (mm^-1), n_e values. */
void orc_majorant(const orc_materials* mat, const orc_phantom* ph, double* maj);

/* Monte Carlo simulation of histories [first, first+n).  Any output pointer
 * may be NULL.  cls/key/q/w: per history.  acc: dense int64 sinogram of
 * n_planes*n_views*n_rad*n_tof bins, incremented by q of the histories whose
 * class is selected by bin_mask (bit 0 scatter, bit 1 trues).  counts: 8
 * class counters (added to).  n_threads <= 0: one thread.  Returns 0 or -1
 * on invalid input. */
int orc_simulate(const orc_scanner* sc, const orc_materials* mat, const orc_phantom* ph,
                 const double* alias_prob, const int32_t* alias_idx, const orc_lut* lut,
                 uint64_t seed, uint64_t first, uint64_t n, int32_t bin_mask, int32_t n_threads,
                 int8_t* cls, int64_t* key, int64_t* q, double* w, orc_record* rec,
                 int64_t* acc, uint64_t* counts);

/* Single-step entry points for the tests. */
void orc_sample_compton(double e, uint64_t seed, int64_t n, double* cos_theta, double* e_out);
void orc_sample_rayleigh(double e, double kappa, uint64_t seed, int64_t n, double* cos_theta);
double orc_lut_prob(const orc_lut* lut, double e, double alpha, double beta, int32_t tpos, int32_t apos);
/* Detection of a photon at pos (inside the cylinder) travelling along dir.
 * Returns ORC_DETECTED or a failure class; fills crystal, ring, hit[3],
 * alpha, beta (deg) and the straight distance to the hit. */
/* Module / block placement of a detector hit when the scanner has gaps: LUT positions,
 * crystal and ring (when not in a gap), the signed offset (mm) from the centre of the
 * transaxial (xt) and axial (xa) gap the hit is in, and the boundary index of that gap
 * (module bt - 1 | module bt; block ba - 1 | block ba, 0 and n_blocks at the scanner
 * ends).  Returns 1 for a transaxial gap, 2 for an axial gap, 3 for both, else 0. */
int orc_place(const orc_scanner* sc, const double hit[3], int32_t* tpos, int32_t* apos,
              int32_t* crystal, int32_t* ring, double* xt, double* xa, int32_t* bt, int32_t* ba);
/* Probability that a photon crossing the detection cylinder in a gap, at offset x0 (mm)
 * from the gap centre with incidence angle theta (deg, positive: the offset grows with
 * depth), is detected in block 1 (the negative-offset side) rather than block 2: the path
 * lengths l1, l2 of its line through the two blocks (depth 0 .. crystal_depth, the gap
 * |x| < gap / 2, the cylinder at depth doi) give the absolute probabilities of the block
 * met first, p = 1 - exp(-mu l), and of the other, exp(-mu l_first) (1 - exp(-mu l));
 * the result is p1 / (p1 + p2), or the nearer block when neither block is crossed. */
double orc_edge_prob(const orc_scanner* sc, double x0, double theta_deg, double gap);
int orc_detect(const orc_scanner* sc, const double pos[3], const double dir[3], double e,
               int32_t* crystal, int32_t* ring, double hit[3], double* alpha, double* beta,
               double* dist);
/* LOR/TOF bin of crystals ca < cb, rings ra, rb and TOF coordinate delta.
 * Returns ORC_SCATTER (= binnable) or ORC_OUT_OF_RANGE; fills the indices. */
int orc_bin(const orc_scanner* sc, int32_t ca, int32_t cb, int32_t ra, int32_t rb, double delta,
            int32_t* plane, int32_t* view, int32_t* rad, int32_t* tof, int64_t* key);

#ifdef __cplusplus
}
#endif
#endif
