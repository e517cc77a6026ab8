/*
 * hist_oracle.c -- the CPU oracle (test infrastructure only; see oracle.h).
 *
 * Plain loops, no blocking, no threads, no vector tricks: each function is
 * the definition it cites, written out so that it can be checked by eye.
 */
#include "oracle.h"

#include <string.h>

/* Sec. III.A: a 256-bin histogram of pixels valued 0..255. */
void oracle_hist_u64(const uint8_t* x, size_t n, uint64_t h[ORACLE_BINS]) {
  for (int b = 0; b < ORACLE_BINS; ++b) h[b] = 0;
  for (size_t i = 0; i < n; ++i) h[x[i]] += 1;
}

int oracle_hist_u32(const uint8_t* x, size_t n, uint32_t h[ORACLE_BINS]) {
  if ((uint64_t)n >= ((uint64_t)1 << 32)) return -1;
  uint64_t w[ORACLE_BINS];
  oracle_hist_u64(x, n, w);
  for (int b = 0; b < ORACLE_BINS; ++b) h[b] = (uint32_t)w[b];
  return 0;
}

/* Sec. III.C: degeneracy is the share of the stream held by its largest bin. */
void oracle_degeneracy(const uint64_t h[ORACLE_BINS], uint32_t* maxbin, uint64_t* max,
                       uint64_t* total) {
  uint32_t arg = 0;
  uint64_t m = 0, t = 0;
  for (uint32_t b = 0; b < ORACLE_BINS; ++b) {
    t += h[b];
    if (h[b] > m) { /* strict: the first bin reaching the maximum keeps it */
      m = h[b];
      arg = b;
    }
  }
  *maxbin = arg;
  *max = m;
  *total = t;
}

/* Sec. III.C: the stream uses the adaptive kernel when any bin of the last
 * histogram reaches the critical degeneracy theta, the plain one otherwise. */
uint32_t oracle_switch(const uint64_t h[ORACLE_BINS], uint32_t theta_milli) {
  uint32_t arg;
  uint64_t m, t;
  oracle_degeneracy(h, &arg, &m, &t);
  if (t == 0) return ORACLE_FLAG_PLAIN;
  /* max / total >= theta_milli / 1000, cross-multiplied; both products fit in
   * 128 bits, compare them exactly. */
  unsigned __int128 lhs = (unsigned __int128)m * 1000u;
  unsigned __int128 rhs = (unsigned __int128)t * theta_milli;
  return lhs >= rhs ? ORACLE_FLAG_ADAPTIVE : ORACLE_FLAG_PLAIN;
}

static uint32_t log2_floor_u64(uint64_t v) { /* v >= 1 */
  uint32_t r = 0;
  while (v > 1) {
    v >>= 1;
    r += 1;
  }
  return r;
}

uint32_t oracle_pattern_layout(const uint8_t log2k[ORACLE_BINS], uint16_t off[ORACLE_BINS]) {
  /* Largest sub-bin groups first, then the next size down, each group of one
   * size in increasing bin order.  Because every earlier group is a larger
   * power of two, each offset is a multiple of its own group size. */
  uint32_t next = 0;
  for (int lk = 5; lk >= 0; --lk) {
    for (int b = 0; b < ORACLE_BINS; ++b) {
      if (log2k[b] == lk) {
        off[b] = (uint16_t)next;
        next += 1u << lk;
      }
    }
  }
  return next;
}

/* Reading of Figure 1 (missing from the text): 960 = 32 * (1+2+4+8+8+4+2+1)
 * sub-bins, 8 at bin 127 (the maximum, Sec. III.A discussion of Table 2) and
 * 1 at the first bins. */
int oracle_default_pattern(uint32_t budget, oracle_pattern* p) {
  static const uint32_t region_k[8] = {1, 2, 4, 8, 8, 4, 2, 1};
  if (budget < ORACLE_BUDGET_MIN || budget > ORACLE_BUDGET_MAX) return -1;
  uint32_t scale = 0; /* largest power of two with 960 * scale <= budget */
  if (budget >= 960) scale = 1u << log2_floor_u64(budget / 960);
  memset(p, 0, sizeof(*p));
  for (int b = 0; b < ORACLE_BINS; ++b) {
    uint32_t k = 1;
    if (scale > 0) {
      k = region_k[b / 32] * scale;
      if (k > ORACLE_KMAX) k = ORACLE_KMAX;
    }
    p->log2k[b] = (uint8_t)log2_floor_u64(k);
  }
  p->budget = budget;
  p->used = oracle_pattern_layout(p->log2k, p->off);
  return 0;
}

/* Sec. III.B: the sub-histogram indices are recomputed from the previous
 * histogram so that frequent bins get more sub-bins. */
int oracle_binning_pattern(const uint32_t h[ORACLE_BINS], uint32_t budget, oracle_pattern* p) {
  if (budget < ORACLE_BUDGET_MIN || budget > ORACLE_BUDGET_MAX) return -1;
  uint64_t total = 0;
  for (int b = 0; b < ORACLE_BINS; ++b) total += h[b];
  if (total == 0) return oracle_default_pattern(budget, p);
  memset(p, 0, sizeof(*p));

  /* 1. proportional share: one sub-bin per bin plus the spare slots split in
   *    proportion to the counts, rounded down to a power of two, at most 32 */
  uint64_t spare = budget - ORACLE_BINS;
  uint32_t k[ORACLE_BINS];
  for (int b = 0; b < ORACLE_BINS; ++b) {
    /* spare < 2^13 and h[b] < 2^32, so the product fits in 64 bits */
    uint64_t want = 1 + (spare * (uint64_t)h[b]) / total;
    uint32_t kk = 1u << log2_floor_u64(want);
    k[b] = kk > ORACLE_KMAX ? ORACLE_KMAX : kk;
  }

  /* 2. floor: every bin is raised to at least f sub-bins, f the largest
   *    power of two up to 32 for which the raised table still fits */
  uint32_t floor_k = 1;
  for (uint32_t f = 2; f <= ORACLE_KMAX; f *= 2) {
    uint64_t sum = 0;
    for (int b = 0; b < ORACLE_BINS; ++b) sum += k[b] > f ? k[b] : f;
    if (sum <= budget) floor_k = f;
  }
  for (int b = 0; b < ORACLE_BINS; ++b) {
    uint32_t kk = k[b] > floor_k ? k[b] : floor_k;
    p->log2k[b] = (uint8_t)log2_floor_u64(kk);
  }

  /* 3. offsets */
  p->budget = budget;
  p->used = oracle_pattern_layout(p->log2k, p->off);
  return 0;
}

/* The batched call's regime of an image (oracle.h states the rule). */
uint32_t oracle_batch_regime(const uint8_t* x, size_t n, uint32_t theta_milli) {
  if (n == 0) return ORACLE_REGIME_WIDE;
  uint64_t m = n < ORACLE_REGIME_SAMPLE ? (uint64_t)n : ORACLE_REGIME_SAMPLE;
  uint64_t h[ORACLE_BINS];
  for (int b = 0; b < ORACLE_BINS; ++b) h[b] = 0;
  if (n <= ORACLE_REGIME_SAMPLE) {
    for (uint64_t i = 0; i < n; ++i) h[x[i]] += 1;
  } else {
    for (uint64_t t = 0; t < 256; ++t) {
      uint64_t start = (t * (uint64_t)n) / 256;
      for (uint64_t u = 0; u < 16; ++u) h[x[start + u]] += 1;
    }
  }
  uint64_t mx = 0, sq = 0;
  for (int b = 0; b < ORACLE_BINS; ++b) {
    if (h[b] > mx) mx = h[b];
    sq += h[b] * h[b];
  }
  if (mx * 1000u >= (uint64_t)theta_milli * m) return ORACLE_REGIME_DEGENERATE;
  if (64u * sq >= m * m) return ORACLE_REGIME_PEAKED;
  return ORACLE_REGIME_WIDE;
}
