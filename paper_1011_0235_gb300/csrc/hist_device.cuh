// hist_device.cuh -- device building blocks shared by the one-shot, stream,
// batch and server kernels.
//
// Shared-memory histogram layouts (Sec. III.A):
//   PLAIN  one 256-slot sub-histogram per warp (the NVIDIA per-warp kernel):
//          pixel v of warp w -> slot w*256 + v.
//   SHIFT  a binning pattern in which every bin has the same number K = 2^lk
//          of sub-bins at off[b] = b*K: pixel v of lane l -> slot
//          (v << lk) + (l & (K-1)); no per-pixel table lookup.  K = 32 is the
//          lane-private table: each lane owns one bank, so a warp's 32
//          increments never meet in a bank whatever the pixel values.
//   LUT    any other pattern: slot = off[v] + (l & (k_v - 1)) read from a
//          per-(value, lane) slot table built once per CTA from the pattern.
// All increments are shared-memory atomics; the per-bin sums of the slots are
// the exact histogram whatever the pattern.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hist.h"

namespace histdev {

constexpr int kThreads = 1024;                  // threads per CTA
constexpr int kWarps = kThreads / 32;
constexpr int kTableWords = HIST_BUDGET_MAX;    // 8192 u32 slots (32 KiB)
constexpr int kLutWords = HIST_BINS * 32;       // one u32 slot index per (value, lane)
constexpr size_t kSmemBytes = (size_t)(kTableWords + kLutWords) * 4;  // 64 KiB dynamic
constexpr int kReplicas = 16;                   // global partial-histogram replicas

enum Path : int { PATH_PLAIN = 0, PATH_SHIFT = 1, PATH_LUT = 2 };

// Static shared state of a CTA (besides the dynamic table + LUT).
struct CtaShared {
  hist_pattern pat;          // pattern this CTA counts with
  uint32_t hist[HIST_BINS];  // a histogram being reduced (epilogues)
  uint32_t res[HIST_BINS];   // this CTA's partial result
  unsigned long long red[kWarps];
  uint32_t cls[8][8];        // per-warp class counts for the pattern layout
  int path;
  int lk;
  uint32_t flag;
  uint32_t kernel;
};

__device__ __forceinline__ uint4 ldg_stream(const uint4* p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  // bulk prefetch of [p, p+bytes) into L2; p 16-byte aligned, bytes a multiple of 16
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void shared_add(uint32_t* p, uint32_t v) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// ------------------------------------------------------------- counting --

template <int PATH, int LK>
__device__ __forceinline__ void count_word(uint32_t w, uint32_t* base, const uint32_t* lutb,
                                           uint32_t* table) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t v = (w >> (8 * k)) & 0xffu;
    if (PATH == PATH_LUT) shared_add(table + lutb[v << 5], 1u);
    else shared_add(base + (v << LK), 1u);
  }
}

template <int PATH, int LK>
__device__ __forceinline__ void count_vec(const uint4& q, uint32_t* base, const uint32_t* lutb,
                                          uint32_t* table) {
  count_word<PATH, LK>(q.x, base, lutb, table);
  count_word<PATH, LK>(q.y, base, lutb, table);
  count_word<PATH, LK>(q.z, base, lutb, table);
  count_word<PATH, LK>(q.w, base, lutb, table);
}

// Count the 16-byte vectors [begin, end) of p, this CTA's slice: thread t takes
// vectors begin + t, begin + t + kThreads, ... (coalesced), two loads in flight.
template <int PATH, int LK>
static __device__ void count_slice(const uint4* __restrict__ p, size_t begin, size_t end, uint32_t* table,
                            const uint32_t* lut) {
  const int lane = threadIdx.x & 31;
  uint32_t* base;
  if (PATH == PATH_PLAIN) base = table + (threadIdx.x >> 5) * HIST_BINS;
  else base = table + (lane & ((1 << LK) - 1));
  const uint32_t* lutb = lut + lane;
  size_t i = begin + threadIdx.x;
  for (; i + kThreads < end; i += 2 * kThreads) {
    const uint4 a = ldg_stream(p + i);
    const uint4 b = ldg_stream(p + i + kThreads);
    count_vec<PATH, LK>(a, base, lutb, table);
    count_vec<PATH, LK>(b, base, lutb, table);
  }
  if (i < end) count_vec<PATH, LK>(ldg_stream(p + i), base, lutb, table);
}

__device__ __forceinline__ void count_dispatch(int path, int lk, const uint4* p, size_t begin,
                                               size_t end, uint32_t* table, const uint32_t* lut) {
  if (begin >= end) return;
  if (path == PATH_PLAIN) count_slice<PATH_PLAIN, 0>(p, begin, end, table, lut);
  else if (path == PATH_LUT) count_slice<PATH_LUT, 0>(p, begin, end, table, lut);
  else {
    switch (lk) {
      case 5: count_slice<PATH_SHIFT, 5>(p, begin, end, table, lut); break;
      case 4: count_slice<PATH_SHIFT, 4>(p, begin, end, table, lut); break;
      case 3: count_slice<PATH_SHIFT, 3>(p, begin, end, table, lut); break;
      case 2: count_slice<PATH_SHIFT, 2>(p, begin, end, table, lut); break;
      case 1: count_slice<PATH_SHIFT, 1>(p, begin, end, table, lut); break;
      default: count_slice<PATH_SHIFT, 0>(p, begin, end, table, lut); break;
    }
  }
}

__device__ __forceinline__ void zero_table(uint32_t* table) {
  uint4* t4 = reinterpret_cast<uint4*>(table);
  for (int i = threadIdx.x; i < kTableWords / 4; i += kThreads) t4[i] = make_uint4(0, 0, 0, 0);
}

// Reduce the table to per-bin sums in cs.res (all threads call; ends synced).
// `part` is 1024 words of free shared memory.
static __device__ void flush_table(int path, int lk, const uint32_t* table, const hist_pattern& pat,
                            uint32_t* part, CtaShared& cs) {
  __syncthreads();
  const int b = threadIdx.x & 255, q = threadIdx.x >> 8;
  uint32_t s = 0;
  if (path == PATH_PLAIN) {
    for (int w = q; w < kWarps; w += 4) s += table[w * HIST_BINS + b];
  } else if (path == PATH_SHIFT) {
    const int K = 1 << lk;
    const uint32_t* row = table + (b << lk);
    if (K >= 4) {
      for (int i = 0; i < K / 4; ++i) s += row[(4 * i + q + b) & (K - 1)];
    } else if (q < K) {
      s += row[q];
    }
  } else {
    const int k = 1 << (pat.log2k[b] & 7);
    const uint32_t o = pat.off[b];
    for (int j = q; j < k && j < HIST_KMAX; j += 4) s += table[(o + j) & (kTableWords - 1)];
  }
  part[q * HIST_BINS + b] = s;
  __syncthreads();
  if (threadIdx.x < HIST_BINS)
    cs.res[threadIdx.x] = part[threadIdx.x] + part[256 + threadIdx.x] + part[512 + threadIdx.x] +
                          part[768 + threadIdx.x];
  __syncthreads();
}

// ----------------------------------------------------- block reductions --

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// Sum of v over threads 0..255 (others must pass 0); every thread gets it.
static __device__ unsigned long long sum256(unsigned long long v, CtaShared& cs) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0 && threadIdx.x < HIST_BINS) cs.red[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long t = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) t += cs.red[i];
  __syncthreads();
  return t;
}
static __device__ unsigned long long max256(unsigned long long v, CtaShared& cs) {
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0 && threadIdx.x < HIST_BINS) cs.red[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long t = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) t = cs.red[i] > t ? cs.red[i] : t;
  __syncthreads();
  return t;
}

// ------------------------------------------------------------ degeneracy --

// max * 1000 >= theta * total, exactly (128-bit products).
__device__ __forceinline__ bool reaches_theta(unsigned long long mx, unsigned long long total,
                                              uint32_t theta_milli) {
  if (total == 0) return false;
  const unsigned long long lhi = __umul64hi(mx, 1000ull), llo = mx * 1000ull;
  const unsigned long long rhi = __umul64hi(total, (unsigned long long)theta_milli),
                           rlo = total * (unsigned long long)theta_milli;
  return lhi > rhi || (lhi == rhi && llo >= rlo);
}

// Degeneracy (Sec. III.C) of a 256-bin histogram; value(b) is called by threads
// 0..255.  All threads call; all get the result.
template <class F>
__device__ hist_degeneracy_result degeneracy_block(F value, uint32_t theta_milli, CtaShared& cs) {
  const bool act = threadIdx.x < HIST_BINS;
  const unsigned long long h = act ? value(threadIdx.x) : 0ull;
  const unsigned long long total = sum256(h, cs);
  const unsigned long long mx = max256(h, cs);
  // lowest bin holding the maximum
  const unsigned long long key = (act && h == mx) ? (unsigned long long)(255 - threadIdx.x) : 0ull;
  const unsigned long long k = max256(act && h == mx ? key + 1 : 0ull, cs);
  hist_degeneracy_result r;
  r.max = mx;
  r.total = total;
  r.maxbin = (mx == 0) ? 0u : (uint32_t)(255 - (k - 1));
  r.flag = reaches_theta(mx, total, theta_milli) ? HIST_FLAG_ADAPTIVE : HIST_FLAG_PLAIN;
  return r;
}

// -------------------------------------------------------- binning pattern --

__device__ __forceinline__ uint32_t ilog2_u64(unsigned long long v) { return 63u - __clzll(v); }

// Offsets for the sub-bin counts lk (thread b < 256 holds lk of bin b): bins in
// order of decreasing k, ties by increasing bin index.  All threads call.
static __device__ void pattern_layout(uint32_t lk, uint32_t budget, hist_pattern& P, CtaShared& cs) {
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const bool act = t < HIST_BINS;
  uint32_t my_rank = 0;
#pragma unroll
  for (uint32_t c = 0; c < 6; ++c) {
    const unsigned m = __ballot_sync(0xffffffffu, act && lk == c);
    if (act && lk == c) my_rank = __popc(m & ((1u << lane) - 1u));
    if (act && lane == 0) cs.cls[w][c] = __popc(m);
  }
  __syncthreads();
  if (act) {
    uint32_t before = 0;
    for (int w2 = 0; w2 < w; ++w2) before += cs.cls[w2][lk];
    uint32_t base = 0;
    for (uint32_t c = 5; c > lk; --c) {
      uint32_t cnt = 0;
      for (int w2 = 0; w2 < 8; ++w2) cnt += cs.cls[w2][c];
      base += cnt << c;
    }
    P.off[t] = (uint16_t)(base + ((my_rank + before) << lk));
    P.log2k[t] = (uint8_t)lk;
    if (t == 0) {
      uint32_t used = 0;
      for (uint32_t c = 0; c < 6; ++c) {
        uint32_t cnt = 0;
        for (int w2 = 0; w2 < 8; ++w2) cnt += cs.cls[w2][c];
        used += cnt << c;
      }
      P.used = used;
      P.budget = budget;
    }
  }
  __syncthreads();
}

// Default pattern (reading of Figure 1), log2 of the sub-bins of bin b.
__device__ __forceinline__ uint32_t default_lk(uint32_t b, uint32_t budget) {
  if (budget < 960) return 0;
  const uint32_t ls = ilog2_u64(budget / 960);
  const uint32_t r = b >> 5;  // region
  const uint32_t rlk = (r < 4) ? r : 7 - r;  // 0,1,2,3,3,2,1,0
  const uint32_t lk = rlk + ls;
  return lk > 5 ? 5 : lk;
}

static __device__ void default_pattern_block(uint32_t budget, hist_pattern& P, CtaShared& cs) {
  const uint32_t lk = threadIdx.x < HIST_BINS ? default_lk(threadIdx.x, budget) : 0;
  pattern_layout(lk, budget, P, cs);
}

// Binning pattern from a histogram (Sec. III.B; rule stated in hist.h).
// value(b) is called by threads 0..255.  All threads call.
template <class F>
static __device__ void binning_pattern_block(F value, uint32_t budget, hist_pattern& P, CtaShared& cs) {
  const bool act = threadIdx.x < HIST_BINS;
  const unsigned long long h = act ? (unsigned long long)value(threadIdx.x) : 0ull;
  const unsigned long long total = sum256(h, cs);
  if (total == 0) {
    default_pattern_block(budget, P, cs);
    return;
  }
  const unsigned long long spare = budget - HIST_BINS;
  const unsigned long long want = 1ull + (spare * h) / total;
  uint32_t lk0 = ilog2_u64(want);
  lk0 = lk0 > 5 ? 5 : lk0;
  uint32_t lf = 0;
  for (uint32_t f = 1; f <= 5; ++f) {
    const uint32_t kk = act ? (1u << (lk0 > f ? lk0 : f)) : 0u;
    const unsigned long long s = sum256(kk, cs);
    if (s <= budget) lf = f;
  }
  const uint32_t lk = lk0 > lf ? lk0 : lf;
  pattern_layout(lk, budget, P, cs);
}

// ------------------------------------------------- pattern classification --

// Decide how a CTA realises pattern P (all threads call; P in shared memory):
// PATH_SHIFT when every bin has the same k = 2^lk and off[b] = b*k, else
// PATH_LUT, whose per-(value, lane) slot table is written to lut.
static __device__ void classify_pattern(const hist_pattern& P, uint32_t* lut, CtaShared& cs) {
  const bool act = threadIdx.x < HIST_BINS;
  const uint32_t lk0 = P.log2k[0];
  const int ok = !act || (P.log2k[threadIdx.x] == lk0 && lk0 <= 5 &&
                          (uint32_t)P.off[threadIdx.x] == ((uint32_t)threadIdx.x << lk0));
  const int uniform = __syncthreads_and(ok);
  if (uniform) {
    if (threadIdx.x == 0) {
      cs.path = PATH_SHIFT;
      cs.lk = (int)lk0;
    }
  } else {
    for (int e = threadIdx.x; e < kLutWords; e += kThreads) {
      const int v = e >> 5, l = e & 31;
      const uint32_t lk = P.log2k[v] > 5 ? 5u : P.log2k[v];
      lut[e] = ((uint32_t)P.off[v] + ((uint32_t)l & ((1u << lk) - 1u))) & (kTableWords - 1);
    }
    if (threadIdx.x == 0) {
      cs.path = PATH_LUT;
      cs.lk = 0;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------ partitions --

// Split n bytes at address a into an unaligned head, 16-byte vectors and a tail.
struct Split {
  size_t head;  // bytes before the first 16-byte boundary (<= 15)
  size_t nvec;  // 16-byte vectors
  size_t tail;  // bytes after the vectors (<= 15)
};
__host__ __device__ __forceinline__ Split split_bytes(const uint8_t* a, size_t n) {
  Split s;
  size_t h = (16 - ((uintptr_t)a & 15)) & 15;
  s.head = h < n ? h : n;
  s.nvec = (n - s.head) / 16;
  s.tail = n - s.head - s.nvec * 16;
  return s;
}

// Count head and tail bytes of a split into cs.res (one warp of the CTA).
__device__ __forceinline__ void count_edges(const uint8_t* a, const Split& sp, CtaShared& cs) {
  const int t = threadIdx.x;
  if (t < (int)sp.head) atomicAdd(&cs.res[a[t]], 1u);
  else if (t >= 16 && t < 16 + (int)sp.tail) atomicAdd(&cs.res[a[sp.head + sp.nvec * 16 + (t - 16)]], 1u);
}

}  // namespace histdev
