/*
 * mdist_probe.h -- measurement probes, built into a separate library
 * (libmdist_probe.so) that only the tests and the benchmark load: instruction- and
 * MMA-throughput probes for roofline arithmetic, and an exactness check of the
 * tensor-core (tcgen05) multiply the Gram-matrix enumerator relies on.  Conventions
 * (return codes, host pointers) as in mdist.h.
 */
#ifndef MDIST_PROBE_H
#define MDIST_PROBE_H

#include "mdist.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Instruction-throughput probe on the current device, for roofline arithmetic:
 * which = 0: 32-bit POPC, 1: 3-input XOR (LOP3), 2: enumerator inner step (XOR + POPC
 * over 4 words, sum, running min), 3 / 4: the lower-bound step of filter groups of 2 /
 * 4 words (threshold never reached), operands in registers; one 1024-thread CTA
 * per SM, `iters` loop trips.  which = 5 / 6 / 7: tcgen05 kind::f8f6f4 MMAs (E4M3,
 * f16 accumulator, 128 x 256 x 32) issued back to back by one thread per SM on
 * shared-memory operands in the no-swizzle / 128-byte swizzle / 32-byte swizzle
 * layout, 4 MMAs per loop trip.  *ops_per_clock_per_sm = operations (codeword steps;
 * multiply-adds for the MMA probes) retired per SM per clock (clock64), *seconds =
 * launch time.  Allocates 64 B + 8 B per SM of device memory for its duration. */
int mdist_microbench(int which, int iters, double *ops_per_clock_per_sm, double *seconds);

/* Tensor-core check: D = A * B^T for A 128 x K and B N x K of E4M3 bytes (row-major,
 * host), K and N multiples of 32 up to 256, computed by tcgen05 kind::f8f6f4 with f32
 * accumulation in TMEM on one CTA; D 128 x N f32 (host).  Allocates its device buffers
 * for the call.  MDIST_ETIMEOUT if the MMA's completion wait ran out. */
int mdist_tc_probe(const uint8_t *A, const uint8_t *B, int N, int K, float *D);

#ifdef __cplusplus
}
#endif

#endif /* MDIST_PROBE_H */
