/* synth_host.c -- host side of the generator defined in synth.h. */
#include "synth.h"

#include <pthread.h>

static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint8_t pick(const uint64_t thr[256], uint64_t r) {
  /* smallest v with r < thr[v]; thr[255] = 2^32 > r always */
  uint32_t lo = 0, hi = 255;
  while (lo < hi) {
    uint32_t mid = (lo + hi) / 2;
    if (r < thr[mid]) hi = mid;
    else lo = mid + 1;
  }
  return (uint8_t)lo;
}

void synth_fill_host(uint8_t* out, size_t n, const uint64_t thr[256], uint64_t seed,
                     uint64_t counter0) {
  for (size_t j = 0; j < n; ++j) out[j] = pick(thr, splitmix64_at(seed, counter0 + j) >> 32);
}

typedef struct {
  uint8_t* out;
  size_t n;
  const uint64_t* thr;
  uint64_t seed, counter0;
} job_t;

static void* run_job(void* arg) {
  job_t* j = (job_t*)arg;
  synth_fill_host(j->out, j->n, j->thr, j->seed, j->counter0);
  return 0;
}

void synth_fill_host_mt(uint8_t* out, size_t n, const uint64_t thr[256], uint64_t seed,
                        uint64_t counter0, int threads) {
  enum { MAXT = 256 };
  if (threads < 1) threads = 1;
  if (threads > MAXT) threads = MAXT;
  pthread_t tid[MAXT];
  job_t jobs[MAXT];
  size_t per = (n + threads - 1) / threads;
  int started = 0;
  for (int t = 0; t < threads; ++t) {
    size_t a = (size_t)t * per;
    if (a >= n) break;
    size_t b = a + per < n ? a + per : n;
    jobs[t] = (job_t){out + a, b - a, thr, seed, counter0 + a};
    if (pthread_create(&tid[t], 0, run_job, &jobs[t]) != 0) {
      run_job(&jobs[t]);
      tid[t] = 0;
      jobs[t].out = 0;
    }
    started = t + 1;
  }
  for (int t = 0; t < started; ++t)
    if (jobs[t].out) pthread_join(tid[t], 0);
}
