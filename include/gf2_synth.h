/*
 * gf2_synth.h -- device-side seeded input generator (separate from the method).
 *
 * Fills a packed GF(2) matrix (layout of gf2.h) with the counter-based recipe
 * of the host module paper_1006_1744_gb300/synth.py, bit for bit:
 *   p == 0.5 and echelon_frac == 0: word(i, w) = mix(seed ^ mix((i << 32) | w));
 *   otherwise: bit(i, j) = (mix(seed ^ TAG_P ^ mix((i << 32) | j)) >> 11) < floor(p * 2^53),
 *              and row i is zero before column floor(echelon_frac * i * n / m).
 * mix() is the SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).
 * Padding bits and padding words (w >= ceil(n/64)) are written as zero.
 *
 *   A      -- DEVICE pointer, m rows of `stride` words, owned by the caller;
 *   stream -- cudaStream_t (NULL = legacy default stream); asynchronous.
 * Returns 0 on success, 1 for invalid arguments, 4 for a CUDA launch error.
 * This generator carries no part of the elimination arithmetic.
 */
#ifndef GF2_SYNTH_H
#define GF2_SYNTH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int gf2_synth_fill(uint64_t *A, int64_t m, int64_t n, int64_t stride, uint64_t seed, double p,
                   double echelon_frac, void *stream);

#ifdef __cplusplus
}
#endif
#endif
