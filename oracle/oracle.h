/*
 * oracle.h -- plain CPU oracle for exact 256-bin histograms of 8-bit pixel
 * streams, the adaptive binning pattern and the degeneracy switch of
 * "Fast Histograms using Adaptive CUDA Streams" (Koppaka et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously correct
 * statement of what the GPU library computes.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or helper with the CUDA library; the struct layouts
 * below are restated here on purpose so that the two sides can be compared
 * byte for byte without either including the other.
 *
 * Integer arithmetic only.  Every result is exact.
 *
 * Parity status per function (what pins it is listed in the tests):
 *   oracle_hist_u64 / oracle_hist_u32   pinned (brute force, closed forms,
 *                                       invariants, a second counting method)
 *   oracle_degeneracy / oracle_switch   pinned (hand-computed cases, mixture
 *                                       expectation, Sec. III.C definition)
 *   oracle_default_pattern              pinned to the facts Sec. III.A states
 *                                       (960 sub-bins, 8 at bin 127, 1 at the
 *                                       first bins); the region layout itself
 *                                       is a reading of the missing Figure 1
 *   oracle_binning_pattern              pinned by invariants, special cases and
 *                                       hand-worked examples; the paper states
 *                                       no formula, so the rule is a reading
 *   oracle_batch_regime                 pinned by closed forms (constant, ramp,
 *                                       cycles at the 64-bin boundary, normal
 *                                       laws), the degeneracy boundary and a
 *                                       case that fixes the sample positions;
 *                                       no counterpart in the paper (the
 *                                       batched call's autotuner)
 */
#ifndef HIST_ORACLE_H
#define HIST_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_BINS 256
#define ORACLE_KMAX 32          /* at most one sub-bin per warp lane (Sec. III.A) */
#define ORACLE_BUDGET_MIN 256   /* one sub-bin per bin */
#define ORACLE_BUDGET_MAX 8192  /* 256 bins x 32 lanes */

#define ORACLE_FLAG_PLAIN 0u
#define ORACLE_FLAG_ADAPTIVE 1u

/* Binning pattern: sub-bin j (0 <= j < 2^log2k[b]) of bin b is table slot
 * off[b] + j; a pixel of value b seen by warp lane l goes to sub-bin
 * l mod 2^log2k[b] (Sec. III.A: sub-bins allotted to the lanes of a warp
 * cyclically).  776 bytes. */
typedef struct oracle_pattern {
  uint16_t off[ORACLE_BINS];
  uint8_t log2k[ORACLE_BINS];
  uint32_t budget; /* table length the pattern was built for */
  uint32_t used;   /* sum over b of 2^log2k[b]; used <= budget */
} oracle_pattern;

/* h[b] = #{ i < n : x[i] == b }  (the definition of a 256-bin histogram of
 * 8-bit pixels, Sec. III.A).  h is overwritten. */
void oracle_hist_u64(const uint8_t* x, size_t n, uint64_t h[ORACLE_BINS]);

/* Same, narrowed to u32.  Returns 0, or -1 (h untouched) if n >= 2^32. */
int oracle_hist_u32(const uint8_t* x, size_t n, uint32_t h[ORACLE_BINS]);

/* Degeneracy of a histogram (Sec. III.C): the largest bin count and the total.
 * maxbin = the lowest index among the bins holding the maximum (0 if all are
 * zero).  deg = max / total as a fraction, total = 0 gives deg = 0. */
void oracle_degeneracy(const uint64_t h[ORACLE_BINS], uint32_t* maxbin, uint64_t* max,
                       uint64_t* total);

/* Kernel switch (Sec. III.C): ADAPTIVE iff some bin reaches the critical
 * degeneracy theta, i.e. max * 1000 >= theta_milli * total with total > 0;
 * PLAIN otherwise. */
uint32_t oracle_switch(const uint64_t h[ORACLE_BINS], uint32_t theta_milli);

/* Default pattern for a stream's first chunk: the reading of Figure 1 as eight
 * regions of 32 bins with 1,2,4,8,8,4,2,1 sub-bins (960 in all), scaled by the
 * largest power of two s with 960*s <= budget (capped at 32 sub-bins), or one
 * sub-bin per bin if budget < 960.  Returns 0, or -1 if budget is out of range. */
int oracle_default_pattern(uint32_t budget, oracle_pattern* p);

/* Binning pattern from the previous histogram (Sec. III.B: indices recomputed
 * from past histograms; the paper gives no formula, this is the stated reading):
 *   T = sum h; T == 0 gives the default pattern.
 *   want[b] = 1 + floor((budget - 256) * h[b] / T)
 *   k0[b]   = min(32, largest power of two <= want[b])
 *   f       = the largest power of two <= 32 with sum_b max(f, k0[b]) <= budget
 *             (f = 1 always fits)
 *   k[b]    = max(f, k0[b])
 *   offsets: bins taken in order of decreasing k, ties by increasing bin
 *   index, each placed right after the previous one, so off[b] is a multiple
 *   of k[b].
 * Returns 0, or -1 if budget is out of range. */
int oracle_binning_pattern(const uint32_t h[ORACLE_BINS], uint32_t budget, oracle_pattern* p);

/* Distribution regime of one image of a batched call, from a sample (the
 * batch autotuner keeps one setting per regime; the paper has no such
 * classifier -- only its first test is the paper's, the degeneracy of
 * Sec. III.C):
 *   the sample is every pixel when n <= ORACLE_REGIME_SAMPLE (4096), else
 *   256 runs of 16 consecutive pixels, run t starting at floor(t * n / 256)
 *   (the runs do not overlap and end inside the image since n > 4096);
 *   m = min(n, 4096) is its size and h its 256-bin histogram.
 *   ORACLE_REGIME_DEGENERATE  max_b h[b] * 1000 >= theta_milli * m
 *   ORACLE_REGIME_PEAKED      otherwise, 64 * sum_b h[b]^2 >= m^2: the chance
 *                             that two sampled pixels are equal is at least
 *                             1/64 (at most 64 "effective" bins)
 *   ORACLE_REGIME_WIDE        otherwise, and for an empty image. */
#define ORACLE_REGIME_SAMPLE 4096u
#define ORACLE_REGIME_DEGENERATE 0u
#define ORACLE_REGIME_PEAKED 1u
#define ORACLE_REGIME_WIDE 2u
uint32_t oracle_batch_regime(const uint8_t* x, size_t n, uint32_t theta_milli);

/* Offsets for given sub-bin counts (the layout step of the two functions
 * above).  log2k[b] in 0..5.  Returns the number of slots used. */
uint32_t oracle_pattern_layout(const uint8_t log2k[ORACLE_BINS], uint16_t off[ORACLE_BINS]);

#ifdef __cplusplus
}
#endif
#endif
