/*
 * synth.h -- seeded synthetic pixel generators shared by the tests, the
 * benchmark and the oracle's inputs.  They hold no histogram arithmetic: they
 * only turn a counter into a byte.
 *
 * Pixel i of a generated stream is defined as follows.
 *   z_i = SplitMix64 output number i for the given seed: the state
 *         seed + (i + 1) * 0x9E3779B97F4A7C15 passed through the SplitMix64
 *         finaliser (Steele, Lea and Flood, "Fast splittable pseudorandom
 *         number generators", OOPSLA 2014; Vigna's reference constants).
 *   r_i = the high 32 bits of z_i.
 *   x_i = the smallest v in 0..255 with r_i < thr[v], where thr is a
 *         non-decreasing table of cumulative thresholds with thr[255] = 2^32.
 * A value v therefore appears with probability (thr[v] - thr[v-1]) / 2^32.
 * i is the pixel's global index within its stream, so a stream cut into
 * chunks or images is the same bytes whatever the cut.
 */
#ifndef HIST_SYNTH_H
#define HIST_SYNTH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Host generator.  out[j] = x_{counter0 + j} for j < n. */
void synth_fill_host(uint8_t* out, size_t n, const uint64_t thr[256], uint64_t seed,
                     uint64_t counter0);

/* Host generator over several threads (same bytes). */
void synth_fill_host_mt(uint8_t* out, size_t n, const uint64_t thr[256], uint64_t seed,
                        uint64_t counter0, int threads);

/* Device generator (same bytes), asynchronous on `stream` (a cudaStream_t).
 * Returns 0 or a CUDA error code. */
int synth_fill_device(uint8_t* d_out, size_t n, const uint64_t thr[256], uint64_t seed,
                      uint64_t counter0, void* stream);

/* synth_fill_device whose kernel lets the next kernel on `stream` start
 * early (griddepcontrol.launch_dependents at its start), as some library
 * kernels do: a kernel launched next with programmatic stream serialisation
 * may run while these bytes are written.  Same bytes. */
int synth_fill_device_early(uint8_t* d_out, size_t n, const uint64_t thr[256], uint64_t seed,
                            uint64_t counter0, void* stream);

/* Device ramp: d_out[j] = (counter0 + j) mod 256. */
int synth_ramp_device(uint8_t* d_out, size_t n, uint64_t counter0, void* stream);

#ifdef __cplusplus
}
#endif
#endif
