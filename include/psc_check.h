/* psc_check.h -- device self-checks of the transport's random numbers (Sec. 2.2.1's
 * simulator draws every random number from a counter-based Philox4x32-10 stream; the
 * paper does not say which generator, the transport here uses Philox4x32-10 of Salmon et
 * al., SC'11).  Test infrastructure: both calls are synchronous, allocate and free their
 * own device buffers, and take host arrays.
 *
 * Return codes as in psc.h: 0, PSC_EINVAL (-1) for bad arguments, PSC_EDEVICE (-5). */
#ifndef PSC_CHECK_H
#define PSC_CHECK_H

#include <stdint.h>

#include "psc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The transport kernel's Philox4x32-10 on n inputs.  in: host [n][6] words
 * (counter c0..c3, key k0, k1); out: host [n][4] words.  1 <= n <= 2^24. */
int psc_check_philox(const uint32_t* in, int64_t n, uint32_t* out);

/* cuRAND's Philox4_32_10 device generator, initialised with (seed, subsequence, offset 0),
 * drawn with curand4 n_blocks times.  out: host [n_blocks][4] words.  1 <= n_blocks <= 2^20. */
int psc_check_curand_philox(uint64_t seed, uint64_t subsequence, int32_t n_blocks, uint32_t* out);

#ifdef __cplusplus
}
#endif
#endif
