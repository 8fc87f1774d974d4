/* psc_peaks.h -- measurement kernels for the roofline of the scatter Monte Carlo
 * transport (Sec. 2.2.1-2.2.3 describe the simulation; these calls are not part of it).
 *
 * The transport's memory work is random: voxel, alias-table and LUT gathers that hit L2,
 * and int64 atomic adds scattered over a sinogram of up to 5.5e9 bins.  These two calls
 * measure what the device sustains for each, so the transport's own rates (from its
 * device counters) can be stated as fractions of them.  Both launch one kernel on
 * `stream` and return at once; time them with events on that stream.
 *
 * Return codes as in psc.h: 0, PSC_EINVAL (-1) for bad arguments, PSC_EDEVICE (-5) when
 * the launch fails.  Neither call takes a context or holds state. */
#ifndef PSC_PEAKS_H
#define PSC_PEAKS_H

#include <stdint.h>

#include "psc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* grid x block threads each add 1 to per_thread uniformly random slots of buf[n_slots]
 * (device int64, caller-owned; its contents change).  block: a multiple of 32 in
 * [32, 1024]; grid, per_thread >= 1. */
int psc_peak_random_atomics(int64_t* buf, uint64_t n_slots, int32_t grid, int32_t block, int32_t per_thread,
                            uint64_t seed, psc_stream stream);

/* grid x block threads each load per_thread (a multiple of 8) uniformly random 4-byte
 * entries of table[n] (device, caller-owned, values >= 0) and sum them; sink (device,
 * one float) is written only if a sum is negative, which keeps the loads live. */
int psc_peak_random_gather(const float* table, uint32_t n, int32_t grid, int32_t block, int32_t per_thread,
                           uint64_t seed, float* sink, psc_stream stream);

#ifdef __cplusplus
}
#endif
#endif
