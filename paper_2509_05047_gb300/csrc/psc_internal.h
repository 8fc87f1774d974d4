// psc_internal.h -- declarations shared by the translation units of libpsc
// (kernel launchers and their parameter blocks).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "psc_device.cuh"

struct psc_ctx;

namespace psc {

// set the calling thread's psc_last_error message; returns code
int set_error(int code, const char* msg);

struct FinParams {
  const long long* acc;
  double* out;
  float* scratch;              // FP32 working sinogram, n_bins floats (smoothing only)
  const double* sens;
  const double* norm;
  const double* rnorm;         // 1/norm (FP64), 0 where norm == 0: the smoothed epilogue's factor
  const float* sens32;         // FP32 copies (round to nearest) of sens and norm for the radial
  const float* norm32;         // pass, or nullptr: it then rounds the FP64 values itself
  int sens_per_lor, norm_per_lor;
  double c;                    // scale * 2^-32
  long long n_bins;
  int n_rings, V, R, T;
  int smooth, sens_first;
  int plane0;                  // first plane (index into the launch's planes) of a plain launch
  int seg0;                    // first ring-difference segment of an axial-pass launch
  int seg_lo, seg_hi;          // finalize only the planes of segments [seg_lo, seg_hi); equal: all
  DebugRecord* dbg;            // bounds-check record of the debug build (nullptr: none)
  int divide_acc;              // output smoothed / (acc * c), 0 where acc == 0 (normalisation sinogram)
  unsigned magic_T;            // ceil(2^32 / T) for exact i / T, 0 when T == 1
  int* status;                 // set nonzero when a tile wait of the axial pass timed out (or nullptr)
  int K[3];                    // truncation radius per axis (radial, view, axial)
  int KT[3];                   // instantiated window radius >= K, or -1: per-tap loop
  float g[3][2 * kMaxSmoothRadius + 1];  // weights centred on KT (on K when KT = -1), zero-padded
};

// sets the calling thread's psc_last_error() message, returns code
int psc_set_error(int code, const char* fmt, ...);

// the emission alias table of an activity image, built on the host
int alias_table(const float* activity, long long n_vox, std::vector<uint2>& tab);
// installs a prepared alias table: waits for the launches reading the
// phantom's current one, then uploads
int put_alias(psc_ctx* ctx, int32_t phantom, const uint2* tab, long long n_vox);

size_t transport_smem_bytes(const PhantomParams& ph, int block);
// 32-bit words of the global slot buffer a launch of grid x block needs
size_t transport_cold_words(int grid, int block);
cudaError_t launch_transport(const BatchParams& p, int lut_dtype, int grid, int block, size_t smem,
                             cudaStream_t s);
cudaError_t transport_occupancy(int lut_dtype, int block, size_t smem, int* blocks_per_sm);

// smoothing weights and window radii from sigma (bins, per axis): PSC_OK,
// or an error code with the message set
int finalize_plan(FinParams& p, const double sigma[3]);
cudaError_t launch_finalize(const FinParams& p, int sms, cudaStream_t s);
// the parts of launch_finalize: the unsmoothed product over planes [lo, hi);
// the radial and view passes over every plane; the axial pass (with the
// epilogue) over ring-difference segments [lo, hi) (segment d + n_rings - 1)
cudaError_t launch_finalize_planes(const FinParams& p, int lo, int hi, int sms, cudaStream_t s);
// planes a finalize covers: all, or those of its segment range
int finalize_planes(const FinParams& p);
cudaError_t launch_smooth_front(const FinParams& p, cudaStream_t s);
cudaError_t launch_smooth_axial(const FinParams& p, int lo, int hi, cudaStream_t s);
// sinogram post-processing of int64 accumulators (postproc.cu)
cudaError_t launch_mash(const long long* in, long long* out, int planes, int V, int R, int T, int vf, int tf,
                        cudaStream_t s);
// span mashing: output planes of n_rings rings at span (odd), and the launch
int span_planes(int n_rings, int span);
cudaError_t launch_span(const long long* in, long long* out, int n_rings, int span, long long J, int sms,
                        cudaStream_t s);
cudaError_t launch_rotate_sum(const long long* in, long long* out, int n_crystals, int n_rings, int R, int T,
                              int step, cudaStream_t s);
// 1/a (0 where a == 0) into r (FP64) and/or r32 (FP32), either may be nullptr
cudaError_t launch_reciprocal(const double* a, double* r, float* r32, long long n, int sms, cudaStream_t s);
// FP32 copy of a sinogram, round to nearest even
cudaError_t launch_narrow(const double* a, float* b, long long n, int sms, cudaStream_t s);

}  // namespace psc
