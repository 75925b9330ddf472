/*
 * cbaa_bench.h -- measurement helpers exported by libcbaa.so.
 *
 * These calls are not part of the detector.  They measure the hardware
 * roofs that the detector's kernels are measured against.
 */
#ifndef CBAA_BENCH_H
#define CBAA_BENCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* L2 atomic-OR roof, async: issue n_ops single-bit reductions (atomicOr with
 * the result unused) at pseudo-random word addresses of dev_buf, the same
 * access pattern as the cube update of Alg. 1 without its address
 * arithmetic.  dev_buf: `words` uint32 words, words a power of two, 16-byte
 * aligned, owned by the caller; its contents afterwards are meaningless.
 * Returns CBAA_OK or a negative status (see cbaa.h). */
int cbaa_bench_red_or(uint32_t *dev_buf, size_t words, size_t n_ops, uint32_t seed, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CBAA_BENCH_H */
