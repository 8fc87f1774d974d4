/* psc_oracle.c -- FP64 CPU oracle of the PET scatter Monte Carlo path.
 *
 * TEST INFRASTRUCTURE: the independent reference for the CUDA library.  Only
 * tests, the smoke check and the benchmark's CPU-baseline leg use it.  It
 * shares no code with the CUDA library.  Plain C99, FP64 throughout, one
 * history at a time, written for reading rather than speed.
 *
 * The paper (Sec. 2.2.1) runs a GPU simulator that it does not describe; the
 * transport physics below is the project's own statement of standard
 * photon Monte Carlo:
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
 *     counter = (history id, block, stream); stream 0 = emission and TOF
 *     blur, stream 1 = photon 1, stream 2 = photon 2; uniform
 *     u = (2*(x >> 9) + 1) * 2^-24 in (0, 1);
 *   - emission: Vose alias table (Vose 1991) over voxel activity, uniform
 *     position in the voxel, isotropic direction, photons back to back at
 *     511 keV (no positron range, no acollinearity; no decay, Sec. 2.1);
 *   - transport: Woodcock delta tracking against an energy-dependent
 *     majorant; one uniform picks Compton / Rayleigh / photo-absorption /
 *     virtual; Compton angles by Kahn's rejection method (Kahn 1954) on the
 *     Klein-Nishina cross section, E' = E / (1 + (E/511)(1 - cos theta));
 *     Rayleigh angles from (1 + cos^2 theta) times a squared form factor
 *     (1 + b s)^-2, s = (1 - cos theta)/2, b = kappa (E/511)^2;
 *   - detection on a cylinder that keeps every photon crossing it
 *     (Sec. 2.2.1), crystal and ring from the hit point (Fig. "crystals"),
 *     incidence angles as in Fig. "angles" (range (-90, 90) degrees);
 *   - weight = product of the two photons' LUT detection probabilities,
 *     1 without a LUT (Sec. 2.2.1); the LUT is interpolated multilinearly in
 *     (energy, transaxial angle, axial angle) at bin-centre nodes and
 *     indexed exactly in the two crystal positions (Sec. 2.2.2);
 *   - TOF bin from the difference of the two photons' path lengths
 *     (Sec. 2.2.1), LOR bin from the crystal pair (span 1, no mashing).
 * Each event is weighted or discarded, never duplicated (Sec. 2.2.3).
 */
#include "psc_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define REST_KEV 511.0
#define EMIT_KEV 511.0
#define PI 3.14159265358979323846
#define MAX_STEPS 4096    /* tracking steps per photon (safety bound) */
#define MAX_TRIES 64      /* rejection-sampling tries (last proposal kept) */
#define POLAR_EPS 1e-6    /* |d_z| > 1 - POLAR_EPS: rotate about the z axis */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw 2011).  */
/* Ten rounds of two 32x32->64 multiplications; the key is bumped by the    */
/* Weyl constants between rounds.                                            */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_block(uint64_t seed, uint64_t hist, uint32_t block, uint32_t stream,
                         uint32_t out[4]) {
  uint32_t ctr[4] = {(uint32_t)hist, (uint32_t)(hist >> 32), block, stream};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* uniform in (0,1): odd multiples of 2^-24, exactly representable in FP32 */
static double u01(uint32_t x) { return (double)((x >> 9) * 2u + 1u) * 0x1p-24; }

/* a sequential stream of uniforms: draw k is word k%4 of block k/4 */
typedef struct {
  uint64_t seed, hist;
  uint32_t stream, block;
  uint32_t buf[4];
  int used;
} stream_t;

static void stream_init(stream_t* s, uint64_t seed, uint64_t hist, uint32_t stream) {
  s->seed = seed; s->hist = hist; s->stream = stream; s->block = 0; s->used = 4;
}

static double next_u(stream_t* s) {
  if (s->used == 4) {
    philox_block(s->seed, s->hist, s->block, s->stream, s->buf);
    s->block++;
    s->used = 0;
  }
  return u01(s->buf[s->used++]);
}

/* ------------------------------------------------------------------------ */
/* Vose's alias method (Vose 1991), deterministic work-list order.          */
/* ------------------------------------------------------------------------ */
int orc_alias_build(const float* weight, int64_t n, double* prob, int32_t* alias) {
  if (n <= 0) return -1;
  double sum = 0.0;
  for (int64_t i = 0; i < n; i++) {
    double a = (double)weight[i];
    if (!(a >= 0.0) || !isfinite(a)) return -1;
    sum += a;
  }
  if (!(sum > 0.0) || !isfinite(sum)) return -1;
  double* scaled = (double*)malloc(sizeof(double) * (size_t)n);
  int32_t* small = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* large = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t ns = 0, nl = 0;
  for (int64_t i = 0; i < n; i++) {
    scaled[i] = ((double)weight[i] * (double)n) / sum;
    if (scaled[i] < 1.0) small[ns++] = (int32_t)i; else large[nl++] = (int32_t)i;
  }
  while (ns > 0 && nl > 0) {
    int32_t s = small[--ns];
    int32_t l = large[--nl];
    prob[s] = scaled[s];
    alias[s] = l;
    scaled[l] = (scaled[l] + scaled[s]) - 1.0;
    if (scaled[l] < 1.0) small[ns++] = l; else large[nl++] = l;
  }
  while (nl > 0) { int32_t l = large[--nl]; prob[l] = 1.0; alias[l] = l; }
  while (ns > 0) { int32_t s = small[--ns]; prob[s] = 1.0; alias[s] = s; }
  free(scaled); free(small); free(large);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Cross-section tables: linear interpolation on the 1 keV grid.            */
/* ------------------------------------------------------------------------ */
static double interp(const double* t, int n, double e) {
  int i = (int)floor(e);
  if (i > n - 2) i = n - 2;
  if (i < 0) i = 0;
  double f = e - (double)i;
  return t[i] + f * (t[i + 1] - t[i]);
}

/* Majorant node k = max over the voxels of density * (mu/rho)_total(E_k), in
 * mm^-1.  Linear interpolation of these nodes bounds every voxel's
 * interpolated attenuation from above. */
void orc_majorant(const orc_materials* mat, const orc_phantom* ph, double* maj) {
  int nm = mat->n_mat, ne = mat->n_e;
  double* rho_max = (double*)calloc((size_t)nm, sizeof(double));
  int64_t nv = (int64_t)ph->nx * ph->ny * ph->nz;
  for (int64_t v = 0; v < nv; v++) {
    int m = ph->material[v];
    double r = (double)ph->density[v];
    if (m < nm && r > rho_max[m]) rho_max[m] = r;
  }
  for (int k = 0; k < ne; k++) {
    double best = 0.0;
    for (int m = 0; m < nm; m++) {
      double tot = mat->compton[m * ne + k] + mat->rayleigh[m * ne + k] + mat->photo[m * ne + k];
      double mu = rho_max[m] * tot / 10.0;
      if (mu > best) best = mu;
    }
    maj[k] = best;
  }
  free(rho_max);
}

/* ------------------------------------------------------------------------ */
/* Interaction sampling                                                     */
/* ------------------------------------------------------------------------ */

/* Kahn's rejection method for the Klein-Nishina distribution of
 * x = E/E' in [1, 1+2a], a = E/511: the density is proportional to
 * (x-1)/x^2 + (cos^2 + 1/x)/x^2; branch A (prob (1+2a)/(9+2a)) samples x
 * uniformly and accepts with 4(x-1)/x^2, branch B samples x ~ 1/x^2 and
 * accepts with (cos^2 + 1/x)/2. */
static void sample_compton(stream_t* s, double e, double* x_out, double* cos_out) {
  double a = e / REST_KEV;
  double x = 1.0, c = 1.0;
  for (int t = 0; t < MAX_TRIES; t++) {
    double r1 = next_u(s), r2 = next_u(s), r3 = next_u(s);
    int accept;
    if (r1 < (1.0 + 2.0 * a) / (9.0 + 2.0 * a)) {
      x = 1.0 + 2.0 * a * r2;
      c = 1.0 - (x - 1.0) / a;
      accept = r3 < 4.0 * (1.0 / x - 1.0 / (x * x));
    } else {
      x = (1.0 + 2.0 * a) / (1.0 + 2.0 * a * r2);
      c = 1.0 - (x - 1.0) / a;
      accept = r3 < 0.5 * (c * c + 1.0 / x);
    }
    if (accept) break;
  }
  *x_out = x;
  *cos_out = c;
}

/* Rayleigh: s = (1 - cos)/2 drawn from (1 + b s)^-2 on [0,1] by inversion,
 * s = u / (1 + b (1 - u)), then accepted with (1 + cos^2)/2 (Thomson). */
static double sample_rayleigh(stream_t* s, double e, double kappa) {
  double b = kappa * (e / REST_KEV) * (e / REST_KEV);
  double c = 1.0;
  for (int t = 0; t < MAX_TRIES; t++) {
    double u1 = next_u(s), u2 = next_u(s);
    double sv = u1 / (1.0 + b * (1.0 - u1));
    c = 1.0 - 2.0 * sv;
    if (u2 < 0.5 * (1.0 + c * c)) break;
  }
  return c;
}

/* new direction at polar cosine c and azimuth phi relative to d */
static void rotate(double d[3], double c, double phi) {
  double sn = sqrt(fmax(0.0, 1.0 - c * c));
  double cp = cos(phi), sp = sin(phi);
  if (fabs(d[2]) > 1.0 - POLAR_EPS) {
    double sg = d[2] > 0.0 ? 1.0 : -1.0;
    d[0] = sn * cp;
    d[1] = sn * sp;
    d[2] = sg * c;
    return;
  }
  double r = sqrt(1.0 - d[2] * d[2]);
  double nx = c * d[0] + sn * (cp * d[0] * d[2] - sp * d[1]) / r;
  double ny = c * d[1] + sn * (cp * d[1] * d[2] + sp * d[0]) / r;
  double nz = c * d[2] - sn * cp * r;
  d[0] = nx; d[1] = ny; d[2] = nz;
}

void orc_sample_compton(double e, uint64_t seed, int64_t n, double* cos_theta, double* e_out) {
  for (int64_t i = 0; i < n; i++) {
    stream_t s;
    stream_init(&s, seed, (uint64_t)i, 1);
    double x, c;
    sample_compton(&s, e, &x, &c);
    cos_theta[i] = c;
    e_out[i] = e / x;
  }
}

void orc_sample_rayleigh(double e, double kappa, uint64_t seed, int64_t n, double* cos_theta) {
  for (int64_t i = 0; i < n; i++) {
    stream_t s;
    stream_init(&s, seed, (uint64_t)i, 1);
    cos_theta[i] = sample_rayleigh(&s, e, kappa);
  }
}

/* ------------------------------------------------------------------------ */
/* Detection on the cylinder (Sec. 2.2.1, Figs. "crystals" and "angles")    */
/* ------------------------------------------------------------------------ */
int orc_detect(const orc_scanner* sc, const double p[3], const double d[3], double e,
               int32_t* crystal, int32_t* ring, double hit[3], double* alpha, double* beta,
               double* dist) {
  double R = sc->radius;
  double a = d[0] * d[0] + d[1] * d[1];
  if (!(a > 0.0)) return ORC_LOST_AXIAL;
  double b = p[0] * d[0] + p[1] * d[1];
  double c = p[0] * p[0] + p[1] * p[1] - R * R;
  double disc = b * b - a * c;
  double sq = sqrt(fmax(disc, 0.0));
  double t = (b >= 0.0) ? (-c) / (b + sq) : (sq - b) / a;
  hit[0] = p[0] + t * d[0];
  hit[1] = p[1] + t * d[1];
  hit[2] = p[2] + t * d[2];
  *dist = t;
  double half = 0.5 * sc->n_rings * sc->ring_pitch;
  if (!(hit[2] >= -half && hit[2] < half)) return ORC_LOST_AXIAL;
  int rg = (int)floor((hit[2] + half) / sc->ring_pitch);
  if (rg > sc->n_rings - 1) rg = sc->n_rings - 1;
  double phi = atan2(hit[1], hit[0]);
  if (phi < 0.0) phi += 2.0 * PI;
  int cr = (int)floor(phi * sc->n_crystals / (2.0 * PI));
  if (cr > sc->n_crystals - 1) cr = sc->n_crystals - 1;
  /* radial unit vector n and tangential unit vector t = z x n at the hit */
  double nx = hit[0] / R, ny = hit[1] / R;
  double dn = d[0] * nx + d[1] * ny;
  double dt = -d[0] * ny + d[1] * nx;
  *alpha = atan2(dt, dn) * (180.0 / PI);
  *beta = atan2(d[2], dn) * (180.0 / PI);
  *crystal = cr;
  *ring = rg;
  if (e < sc->e_lo || e > sc->e_hi) return ORC_ENERGY_WINDOW;
  return ORC_DETECTED;
}

/* ------------------------------------------------------------------------ */
/* Gaps between modules and blocks (Sec. 2.2.1-2.2.2)                        */
/* ------------------------------------------------------------------------ */
int orc_place(const orc_scanner* sc, const double hit[3], int32_t* tpos, int32_t* apos,
              int32_t* crystal, int32_t* ring, double* xt, double* xa, int32_t* bt, int32_t* ba) {
  int mt = sc->module_t, ma = sc->module_a;
  int n_mod = sc->n_crystals / mt, n_blk = sc->n_rings / ma;
  double R = sc->radius;
  /* transaxial: module m spans azimuth [m Phi, (m+1) Phi), half gaps of gamma / 2 at its ends */
  double Phi = 2.0 * PI / n_mod, gamma = sc->gap_t / R;
  double phi = atan2(hit[1], hit[0]);
  if (phi < 0.0) phi += 2.0 * PI;
  int m = (int)floor(phi / Phi);
  if (m > n_mod - 1) m = n_mod - 1;
  double u = phi - m * Phi;
  int flags = 0;
  *crystal = -1;
  *ring = -1;
  *xt = 0.0;
  *xa = 0.0;
  *bt = -1;
  *ba = -1;
  if (u < 0.5 * gamma) {
    *tpos = 0; *bt = m; *xt = u * R; flags |= 1;
  } else if (u >= Phi - 0.5 * gamma) {
    *tpos = mt + 1; *bt = m + 1; *xt = (u - Phi) * R; flags |= 1;
  } else {
    int j = (int)floor((u - 0.5 * gamma) / ((Phi - gamma) / mt));
    if (j > mt - 1) j = mt - 1;
    *tpos = j + 1;
    *crystal = m * mt + j;
  }
  /* axial: block b spans [b P, (b+1) P) from the scanner's lower end, half gaps at its ends */
  double L = sc->n_rings * sc->ring_pitch, P = L / n_blk, ga = sc->gap_a;
  double z = hit[2] + 0.5 * L;
  int b = (int)floor(z / P);
  if (b > n_blk - 1) b = n_blk - 1;
  if (b < 0) b = 0;
  double w = z - b * P;
  int al;
  if (w < 0.5 * ga) {
    al = 0; *ba = b; *xa = w; flags |= 2;
  } else if (w >= P - 0.5 * ga) {
    al = ma + 1; *ba = b + 1; *xa = w - P; flags |= 2;
  } else {
    int j = (int)floor((w - 0.5 * ga) / ((P - ga) / ma));
    if (j > ma - 1) j = ma - 1;
    al = j + 1;
    *ring = b * ma + j;
  }
  *apos = b * (ma + 2) + al;
  return flags;
}

double orc_edge_prob(const orc_scanner* sc, double x0, double theta_deg, double gap) {
  double D = sc->crystal_depth, y0 = sc->doi, mu = sc->mu_block;
  double th = theta_deg * PI / 180.0;
  double s = tan(th), c = cos(th);
  double l1 = 0.0, l2 = 0.0;
  if (s != 0.0) {
    /* the line x(y) = x0 + (y - y0) s meets x = -gap/2 at ya and x = +gap/2 at yb */
    double ya = y0 + (-0.5 * gap - x0) / s, yb = y0 + (0.5 * gap - x0) / s;
    if (s > 0.0) {  /* block 1 at small depth, block 2 at large depth */
      l1 = fmax(0.0, fmin(D, ya) - 0.0) / c;
      l2 = fmax(0.0, D - fmax(0.0, yb)) / c;
    } else {        /* block 2 at small depth, block 1 at large depth */
      l2 = fmax(0.0, fmin(D, yb) - 0.0) / c;
      l1 = fmax(0.0, D - fmax(0.0, ya)) / c;
    }
  }
  double first = s > 0.0 ? l1 : l2, second = s > 0.0 ? l2 : l1;
  double pf = 1.0 - exp(-mu * first);
  double ps = exp(-mu * first) * (1.0 - exp(-mu * second));
  double p1 = s > 0.0 ? pf : ps, p2 = s > 0.0 ? ps : pf;
  if (!(p1 + p2 > 0.0)) return x0 < 0.0 ? 1.0 : (x0 > 0.0 ? 0.0 : 0.5);
  return p1 / (p1 + p2);
}

/* ------------------------------------------------------------------------ */
/* 5D LUT (Sec. 2.2.2): multilinear in (E, alpha, beta) on bin-centre nodes,*/
/* clamped at the outer nodes; exact in (tpos, apos).                       */
/* ------------------------------------------------------------------------ */
static void axis_coord(double x, double lo, double hi, int n, int* i0, int* i1, double* f) {
  if (n == 1) { *i0 = 0; *i1 = 0; *f = 0.0; return; }
  double g = (x - lo) / ((hi - lo) / n) - 0.5;
  if (g < 0.0) g = 0.0;
  if (g > (double)(n - 1)) g = (double)(n - 1);
  int i = (int)floor(g);
  if (i > n - 2) i = n - 2;
  *i0 = i;
  *i1 = i + 1;
  *f = g - (double)i;
}

double orc_lut_prob(const orc_lut* L, double e, double alpha, double beta, int32_t tpos, int32_t apos) {
  if (L == NULL || L->data == NULL) return 1.0;
  if (L->n_tpos == 1) tpos = 0;  /* no crystal information on this axis */
  if (L->n_apos == 1) apos = 0;
  int ie[2], ia[2], ib[2];
  double fe, fa, fb;
  axis_coord(e, L->e_min, L->e_max, L->n_e, &ie[0], &ie[1], &fe);
  axis_coord(alpha, L->a_min, L->a_max, L->n_a, &ia[0], &ia[1], &fa);
  axis_coord(beta, L->b_min, L->b_max, L->n_b, &ib[0], &ib[1], &fb);
  double we[2] = {1.0 - fe, fe}, wa[2] = {1.0 - fa, fa}, wb[2] = {1.0 - fb, fb};
  int64_t base = ((int64_t)apos * L->n_tpos + tpos) * L->n_e;
  double v = 0.0;
  for (int j = 0; j < 2; j++)
    for (int k = 0; k < 2; k++)
      for (int l = 0; l < 2; l++) {
        int64_t idx = ((base + ie[j]) * L->n_a + ia[k]) * L->n_b + ib[l];
        v += we[j] * wa[k] * wb[l] * (double)L->data[idx];
      }
  return v;
}

/* ------------------------------------------------------------------------ */
/* LOR x TOF binning (Sec. 2.2.1): crystals ca < cb, span-1 planes.          */
/* ------------------------------------------------------------------------ */
int orc_bin(const orc_scanner* sc, int32_t ca, int32_t cb, int32_t ra, int32_t rb, double delta,
            int32_t* plane, int32_t* view, int32_t* rad, int32_t* tof, int64_t* key) {
  int N = sc->n_crystals;
  int f = ca + cb, s = 1;
  if (f >= N) { f -= N; s = -1; }
  int v = f >> 1;
  int r = s * (N / 2 - (cb - ca)) + N / 2 - 1;
  r -= (N - 1 - sc->n_rad) / 2;
  int t = (int)floor(delta / sc->tof_bin_mm + 0.5 * sc->n_tof);
  int p = ra * sc->n_rings + rb;
  *plane = p; *view = v; *rad = r; *tof = t;
  *key = -1;
  if (r < 0 || r >= sc->n_rad) return ORC_OUT_OF_RANGE;
  if (delta != delta || t < 0 || t >= sc->n_tof) return ORC_OUT_OF_RANGE;
  *key = (((int64_t)p * (N / 2) + v) * sc->n_rad + r) * sc->n_tof + t;
  return ORC_SCATTER;
}

/* ------------------------------------------------------------------------ */
/* One photon: Woodcock tracking, then detection.                           */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_scanner* sc;
  const orc_materials* mat;
  const orc_phantom* ph;
  const double* alias_prob;
  const int32_t* alias_idx;
  const orc_lut* lut;
  double* maj;
  uint64_t seed;
  int32_t bin_mask;
} sim_ctx;

typedef struct {
  int status;
  double pos[3], dir[3], e, path;
  int n_compton, n_rayleigh, n_steps;
  int crystal, ring;
  double hit[3], alpha, beta, prob, e_det;
  int have_c;
  double c_e_before, c_e_after, c_dir_before[3], c_dir_after[3];
} photon_t;

/* Energy resolution (the no-LUT mode of Sec. 2.2.1 uses 11.2 %): the
 * detected energy is E + sigma(E) g, g standard normal (Box-Muller on two
 * words of the photon's stream), sigma(E) = e_res sqrt(511 E) / 2.3548, so
 * the FWHM is e_res * 511 keV at 511 keV and scales as sqrt(E).  A photon
 * that Compton-scatters below e_lo - 5 sigma(e_lo) is dropped (without
 * resolution: below e_lo, which is exact since E never increases). */
static double e_sigma(const orc_scanner* sc, double e) {
  return sc->e_res * sqrt(511.0 * e) / 2.3548200450309493;
}

static double e_kill(const orc_scanner* sc) {
  if (!(sc->e_res > 0.0)) return sc->e_lo;
  return fmax(0.0, sc->e_lo - 5.0 * e_sigma(sc, sc->e_lo));
}

static void track_photon(const sim_ctx* X, stream_t* s, photon_t* p) {
  const orc_phantom* ph = X->ph;
  const orc_materials* mt = X->mat;
  int ne = mt->n_e;
  for (;;) {
    if (p->n_steps >= MAX_STEPS) { p->status = ORC_STEP_LIMIT; return; }
    double mu_max = interp(X->maj, ne, p->e);
    if (!(mu_max > 0.0)) break;                  /* nothing attenuates: leave the grid */
    double dist = -log(next_u(s)) / mu_max;
    double q[3];
    for (int k = 0; k < 3; k++) q[k] = p->pos[k] + dist * p->dir[k];
    double fx = (q[0] - ph->ox) / ph->dx, fy = (q[1] - ph->oy) / ph->dy, fz = (q[2] - ph->oz) / ph->dz;
    if (!(fx >= 0.0 && fx < ph->nx && fy >= 0.0 && fy < ph->ny && fz >= 0.0 && fz < ph->nz))
      break;                                     /* outside the grid is vacuum */
    int ix = (int)floor(fx), iy = (int)floor(fy), iz = (int)floor(fz);
    if (ix > ph->nx - 1) ix = ph->nx - 1;
    if (iy > ph->ny - 1) iy = ph->ny - 1;
    if (iz > ph->nz - 1) iz = ph->nz - 1;
    for (int k = 0; k < 3; k++) p->pos[k] = q[k];
    p->path += dist;
    p->n_steps++;
    int64_t v = ((int64_t)iz * ph->ny + iy) * ph->nx + ix;
    int m = ph->material[v];
    double rho = (double)ph->density[v];
    double mc = rho * interp(mt->compton + (int64_t)m * ne, ne, p->e) / 10.0;
    double mr = rho * interp(mt->rayleigh + (int64_t)m * ne, ne, p->e) / 10.0;
    double mp = rho * interp(mt->photo + (int64_t)m * ne, ne, p->e) / 10.0;
    double t = next_u(s) * mu_max;
    if (t < mc) {                                /* Compton */
      double x, c;
      double e0 = p->e, d0[3] = {p->dir[0], p->dir[1], p->dir[2]};
      sample_compton(s, p->e, &x, &c);
      double phi = 2.0 * PI * next_u(s);
      rotate(p->dir, c, phi);
      p->e = p->e / x;
      p->n_compton++;
      if (!p->have_c) {
        p->have_c = 1;
        p->c_e_before = e0;
        p->c_e_after = p->e;
        memcpy(p->c_dir_before, d0, sizeof d0);
        memcpy(p->c_dir_after, p->dir, sizeof d0);
      }
      if (p->e < e_kill(X->sc)) { p->status = ORC_ENERGY_WINDOW; return; }
    } else if (t < mc + mr) {                    /* Rayleigh */
      double c = sample_rayleigh(s, p->e, mt->kappa[m]);
      double phi = 2.0 * PI * next_u(s);
      rotate(p->dir, c, phi);
      p->n_rayleigh++;
    } else if (t < mc + mr + mp) {               /* photo-absorption */
      p->status = ORC_ABSORBED;
      return;
    }                                            /* else: virtual collision */
  }
  double dist;
  int st = orc_detect(X->sc, p->pos, p->dir, p->e, &p->crystal, &p->ring, p->hit, &p->alpha,
                      &p->beta, &dist);
  p->path += dist;
  p->e_det = p->e;
  if (X->sc->e_res > 0.0 && st != ORC_LOST_AXIAL) {
    double u1 = next_u(s), u2 = next_u(s);
    p->e_det = p->e + e_sigma(X->sc, p->e) * sqrt(-2.0 * log(u1)) * cos(2.0 * PI * u2);
    st = (p->e_det < X->sc->e_lo || p->e_det > X->sc->e_hi) ? ORC_ENERGY_WINDOW : ORC_DETECTED;
  }
  p->status = st;
  if (st != ORC_DETECTED) return;
  const orc_scanner* sc = X->sc;
  if (sc->gap_mode == 0) {
    p->prob = orc_lut_prob(X->lut, p->e, p->alpha, p->beta, p->crystal % sc->module_t,
                           p->ring % sc->module_a);
    return;
  }
  int32_t tpos, apos, cr, rg, bt, ba;
  double xt, xa;
  int flags = orc_place(sc, p->hit, &tpos, &apos, &cr, &rg, &xt, &xa, &bt, &ba);
  if (flags && sc->gap_mode == 1) { p->status = ORC_LOST_AXIAL; return; }  /* lost in a gap */
  p->prob = orc_lut_prob(X->lut, p->e, p->alpha, p->beta, tpos, apos);
  /* a photon in a gap goes to one of the gap's two edge crystals: accept-reject on one
   * word of its stream against the relative detection probability of the two blocks */
  int N = sc->n_crystals, cpm = sc->module_t, rpb = sc->module_a, n_blk = sc->n_rings / rpb;
  if (flags & 1) {
    double u = next_u(s);
    double p1 = orc_edge_prob(sc, xt, p->alpha, sc->gap_t);
    cr = u < p1 ? (bt * cpm - 1 + N) % N : (bt * cpm) % N;
  }
  if (flags & 2) {
    if (ba == 0) rg = 0;                      /* scanner end: one block only */
    else if (ba == n_blk) rg = sc->n_rings - 1;
    else {
      double u = next_u(s);
      double p1 = orc_edge_prob(sc, xa, p->beta, sc->gap_a);
      rg = u < p1 ? ba * rpb - 1 : ba * rpb;
    }
  }
  p->crystal = cr;
  p->ring = rg;
}

/* ------------------------------------------------------------------------ */
/* One history: emission, two photons, coincidence.                         */
/* ------------------------------------------------------------------------ */
static void run_history(const sim_ctx* X, uint64_t h, orc_record* r) {
  const orc_phantom* ph = X->ph;
  const orc_scanner* sc = X->sc;
  memset(r, 0, sizeof *r);
  uint32_t b0[4], b1[4];
  philox_block(X->seed, h, 0, 0, b0);
  philox_block(X->seed, h, 1, 0, b1);
  int64_t nv = (int64_t)ph->nx * ph->ny * ph->nz;
  int64_t col = (int64_t)(((uint64_t)b0[0] * (uint64_t)nv) >> 32);
  int64_t v = (u01(b0[1]) < X->alias_prob[col]) ? col : (int64_t)X->alias_idx[col];
  int64_t ix = v % ph->nx, iy = (v / ph->nx) % ph->ny, iz = v / ((int64_t)ph->nx * ph->ny);
  double e0[3] = {ph->ox + ((double)ix + u01(b0[2])) * ph->dx,
                  ph->oy + ((double)iy + u01(b0[3])) * ph->dy,
                  ph->oz + ((double)iz + u01(b1[0])) * ph->dz};
  double ct = 2.0 * u01(b1[1]) - 1.0;
  double phi = 2.0 * PI * u01(b1[2]);
  double st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double d[3] = {st * cos(phi), st * sin(phi), ct};
  r->voxel = (int32_t)v;
  memcpy(r->emit, e0, sizeof e0);
  memcpy(r->dir, d, sizeof d);

  photon_t P[2];
  for (int k = 0; k < 2; k++) {
    memset(&P[k], 0, sizeof P[k]);
    double sg = k == 0 ? 1.0 : -1.0;
    for (int j = 0; j < 3; j++) { P[k].pos[j] = e0[j]; P[k].dir[j] = sg * d[j]; }
    P[k].e = EMIT_KEV;
    stream_t s;
    stream_init(&s, X->seed, h, (uint32_t)(k + 1));
    track_photon(X, &s, &P[k]);
    r->status[k] = P[k].status;
    r->crystal[k] = P[k].crystal;
    r->ring[k] = P[k].ring;
    r->n_compton[k] = P[k].n_compton;
    r->n_rayleigh[k] = P[k].n_rayleigh;
    r->n_steps[k] = P[k].n_steps;
    r->energy[k] = P[k].e;
    r->e_det[k] = P[k].e_det;
    r->alpha[k] = P[k].alpha;
    r->beta[k] = P[k].beta;
    r->path[k] = P[k].path;
    r->prob[k] = P[k].prob;
    memcpy(r->hit[k], P[k].hit, sizeof P[k].hit);
    memcpy(r->exit_pos[k], P[k].pos, sizeof P[k].pos);
    memcpy(r->exit_dir[k], P[k].dir, sizeof P[k].dir);
  }
  if (P[0].have_c) {
    r->c_e_before = P[0].c_e_before;
    r->c_e_after = P[0].c_e_after;
    memcpy(r->c_dir_before, P[0].c_dir_before, sizeof r->c_dir_before);
    memcpy(r->c_dir_after, P[0].c_dir_after, sizeof r->c_dir_after);
  }
  r->key = -1;
  r->q = 0;
  if (P[0].status != ORC_DETECTED) { r->cls = P[0].status; return; }
  if (P[1].status != ORC_DETECTED) { r->cls = P[1].status; return; }
  if (P[0].crystal == P[1].crystal) { r->cls = ORC_SAME_CRYSTAL; return; }
  const photon_t* A = P[0].crystal < P[1].crystal ? &P[0] : &P[1];
  const photon_t* B = P[0].crystal < P[1].crystal ? &P[1] : &P[0];
  double delta = 0.5 * (A->path - B->path);
  if (sc->tof_sigma_mm > 0.0) {                  /* Gaussian TOF blur, Box-Muller */
    uint32_t b2[4];
    philox_block(X->seed, h, 2, 0, b2);
    double g = sqrt(-2.0 * log(u01(b2[0]))) * cos(2.0 * PI * u01(b2[1]));
    delta += sc->tof_sigma_mm * g;
  }
  r->delta = delta;
  int64_t key;
  int cb = orc_bin(sc, A->crystal, B->crystal, A->ring, B->ring, delta, &r->plane, &r->view,
                   &r->rad, &r->tof, &key);
  if (cb != ORC_SCATTER) { r->cls = ORC_OUT_OF_RANGE; return; }
  int scattered = (P[0].n_compton + P[0].n_rayleigh + P[1].n_compton + P[1].n_rayleigh) > 0;
  r->cls = scattered ? ORC_SCATTER : ORC_TRUE;
  r->key = key;
  r->w = P[0].prob * P[1].prob;
  r->q = (int64_t)llrint(r->w * 4294967296.0);
}

/* ------------------------------------------------------------------------ */
/* Driver: threads over contiguous history ranges; the sinogram is summed   */
/* afterwards in history order.                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  const sim_ctx* X;
  uint64_t first, n, off;
  int8_t* cls;
  int64_t* key;
  int64_t* q;
  double* w;
  orc_record* rec;
  uint64_t counts[ORC_N_CLASSES];
} job_t;

static void* run_job(void* arg) {
  job_t* J = (job_t*)arg;
  orc_record r;
  for (uint64_t i = 0; i < J->n; i++) {
    uint64_t idx = J->off + i;
    run_history(J->X, J->first + i, &r);
    J->counts[r.cls]++;
    if (J->cls) J->cls[idx] = (int8_t)r.cls;
    if (J->key) J->key[idx] = r.key;
    if (J->q) J->q[idx] = r.q;
    if (J->w) J->w[idx] = r.w;
    if (J->rec) J->rec[idx] = r;
  }
  return NULL;
}

static int check_inputs(const orc_scanner* sc, const orc_materials* mat, const orc_phantom* ph) {
  if (!sc || !mat || !ph) return -1;
  if (sc->n_crystals < 2 || (sc->n_crystals & 1) || sc->n_rings < 1 || sc->n_tof < 1) return -1;
  if (sc->n_rad < 1 || sc->n_rad > sc->n_crystals - 1 || ((sc->n_crystals - 1 - sc->n_rad) & 1)) return -1;
  if (!(sc->radius > 0.0) || !(sc->ring_pitch > 0.0) || !(sc->tof_bin_mm > 0.0)) return -1;
  if (sc->module_t < 1 || sc->module_a < 1) return -1;
  if (mat->n_mat < 1 || mat->n_e < 2) return -1;
  if (ph->nx < 1 || ph->ny < 1 || ph->nz < 1) return -1;
  int64_t nv = (int64_t)ph->nx * ph->ny * ph->nz;
  for (int64_t v = 0; v < nv; v++) if (ph->material[v] >= mat->n_mat) return -1;
  /* every grid corner strictly inside the cylinder */
  double R2 = sc->radius * sc->radius;
  for (int i = 0; i < 4; i++) {
    double x = ph->ox + ((i & 1) ? ph->nx * ph->dx : 0.0);
    double y = ph->oy + ((i & 2) ? ph->ny * ph->dy : 0.0);
    if (!(x * x + y * y < R2)) return -1;
  }
  return 0;
}

int orc_simulate(const orc_scanner* sc, const orc_materials* mat, const orc_phantom* ph,
                 const double* alias_prob, const int32_t* alias_idx, const orc_lut* lut,
                 uint64_t seed, uint64_t first, uint64_t n, int32_t bin_mask, int32_t n_threads,
                 int8_t* cls, int64_t* key, int64_t* q, double* w, orc_record* rec,
                 int64_t* acc, uint64_t* counts) {
  if (check_inputs(sc, mat, ph) != 0 || !alias_prob || !alias_idx) return -1;
  if (sc->gap_mode != 0 && (sc->n_crystals % sc->module_t || sc->n_rings % sc->module_a)) return -1;
  if (lut && lut->data) {
    int nt = sc->gap_mode ? sc->module_t + 2 : sc->module_t;
    int na = sc->gap_mode ? (sc->n_rings / sc->module_a) * (sc->module_a + 2) : sc->module_a;
    if ((lut->n_tpos != nt && lut->n_tpos != 1) || (lut->n_apos != na && lut->n_apos != 1)) return -1;
  }
  if (n == 0) return 0;
  sim_ctx X = {sc, mat, ph, alias_prob, alias_idx, lut, NULL, seed, bin_mask};
  X.maj = (double*)malloc(sizeof(double) * (size_t)mat->n_e);
  orc_majorant(mat, ph, X.maj);
  int own_key = 0, own_q = 0, own_cls = 0;
  if (acc && !key) { key = (int64_t*)malloc(sizeof(int64_t) * n); own_key = 1; }
  if (acc && !q) { q = (int64_t*)malloc(sizeof(int64_t) * n); own_q = 1; }
  if (acc && !cls) { cls = (int8_t*)malloc(n); own_cls = 1; }
  int nt = n_threads > 0 ? n_threads : 1;
  if ((uint64_t)nt > n) nt = (int)n;
  job_t* jobs = (job_t*)calloc((size_t)nt, sizeof(job_t));
  pthread_t* th = (pthread_t*)calloc((size_t)nt, sizeof(pthread_t));
  uint64_t chunk = n / (uint64_t)nt, rem = n % (uint64_t)nt, off = 0;
  for (int t = 0; t < nt; t++) {
    uint64_t m = chunk + ((uint64_t)t < rem ? 1 : 0);
    jobs[t] = (job_t){&X, first + off, m, off, cls, key, q, w, rec, {0}};
    off += m;
  }
  if (nt == 1) {
    run_job(&jobs[0]);
  } else {
    for (int t = 0; t < nt; t++) pthread_create(&th[t], NULL, run_job, &jobs[t]);
    for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
  }
  if (counts)
    for (int t = 0; t < nt; t++)
      for (int c = 0; c < ORC_N_CLASSES; c++) counts[c] += jobs[t].counts[c];
  if (acc) {
    for (uint64_t i = 0; i < n; i++) {
      int c = cls[i];
      int take = (c == ORC_SCATTER && (bin_mask & 1)) || (c == ORC_TRUE && (bin_mask & 2));
      if (take) acc[key[i]] += q[i];
    }
  }
  if (own_key) free(key);
  if (own_q) free(q);
  if (own_cls) free(cls);
  free(jobs);
  free(th);
  free(X.maj);
  return 0;
}
