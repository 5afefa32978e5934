/*
 * blb_peaks.h -- integer-pipe throughput of the B300 for the ALU rooflines of
 * the benchmark (libblb_peaks.so, built beside libblb.so).  A measurement
 * helper with no counterpart in the paper and no part in the hot path.
 *
 * blb_peaks_int_rates runs two register-only kernels on every SM of the current
 * device, on `stream` (a cudaStream_t, NULL = default stream), and waits for
 * them: independent chains of (a) the NTT's lazy Cooley-Tukey butterfly on
 * 64-bit words (a Shoup product by a constant twiddle mod q, X + WY,
 * X - WY + 2q, the conditional 2q subtraction) and (b) a 64 x 64 -> 128-bit
 * multiply-accumulate (the base conversions' unit).  q is an odd modulus below
 * 2^62 (the butterfly's prime).  Outputs (host, nullable): operations per
 * second, and per SM cycle (the SM clock measured during the run from
 * %globaltimer and clock64).  It allocates its two small buffers with
 * cudaMalloc and frees them.  Returns 0, -1 for a bad q, -5 when allocation
 * fails, -6 when a CUDA call fails.
 */
#ifndef BLB_PEAKS_H
#define BLB_PEAKS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int blb_peaks_int_rates(uint64_t q, void* stream, double* bfly_per_s, double* mad128_per_s,
                        double* bfly_per_sm_cycle, double* mad128_per_sm_cycle);

/* The same measurement for the reduction of a 128-bit value mod q (a Barrett
 * reduction with floor(2^128 / q): three 64-bit partial products, two
 * conditional subtractions), in independent register chains whose next input
 * adds the previous result.  q odd, 3 <= q < 2^62.  Outputs (host, nullable):
 * reductions per second and per SM cycle.  Returns as blb_peaks_int_rates. */
int blb_peaks_reduce_rate(uint64_t q, void* stream, double* per_s, double* per_sm_cycle);

#ifdef __cplusplus
}
#endif
#endif
