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

enum Path : int { PATH_PLAIN = 0, PATH_SHIFT = 1, PATH_LUT = 2 };

// Static shared state of a CTA (besides the dynamic table + LUT).
struct CtaShared {
  hist_pattern pat;          // pattern this CTA counts with
  uint32_t hist[HIST_BINS];  // a histogram being reduced (epilogues)
  uint32_t res[HIST_BINS];   // this CTA's partial result
  unsigned long long red[kWarps];
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

__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// One increment of the shared-memory word at byte address `a`.
__device__ __forceinline__ void shared_inc(uint32_t a) {
  asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(a) : "memory");
}
__device__ __forceinline__ uint32_t shared_ld(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}

// ------------------------------------------------------------- counting --
// Addresses are 32-bit byte offsets in the shared window: `base` is this
// thread's first slot (PLAIN: its warp's table; SHIFT: lane & (K-1)), `lutb`
// its lane's column of the slot table, `table` the table itself.

template <int PATH, int LK>
__device__ __forceinline__ void count_word(uint32_t w, uint32_t base, uint32_t lutb, uint32_t table) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t v = (w >> (8 * k)) & 0xffu;
    if (PATH == PATH_LUT) shared_inc(table + (shared_ld(lutb + (v << 7)) << 2));
    else shared_inc(base + (v << (LK + 2)));
  }
}

// The order in which a lane takes the 16 bytes of its vector (every layout
// but the shift layouts with 16 or 32 sub-bins per bin): lane l counts byte
// s ^ (l mod 16) at step s.  The increments of one
// step are one warp-wide shared-memory operation; when neighbouring pixels
// differ by a constant (a ramp: lane l holds values 16 l .. 16 l + 15), the
// natural order puts the warp's 16 distinct values in two banks (8-way
// conflicts), while this order spreads them over 16 banks.  Equal values
// still meet at one address, which costs nothing.  Two byte-permutes per
// 4 bytes: the first takes word i or i ^ 1 with its bytes in xor order, the
// second word i or i ^ 2 of the result.  Measured on 1 GiB (one-shot per-warp
// kernel): a ramp 1.19 -> 6.2 TB/s; uniform, constant and N(128, 8) data
// within 1.5 % of the natural order.  The same with the rule's 960-slot
// pattern of a ramp (two sub-bins per bin): 1.19 -> 6.26 TB/s.
struct LaneOrder {
  uint32_t a, b;  // byte-permute selectors
};
__device__ __forceinline__ LaneOrder lane_order() {
  const uint32_t c = threadIdx.x & 15u, x = c & 3u, hi = (c >> 2) & 1u;
  LaneOrder o;
  o.a = 0;
#pragma unroll
  for (uint32_t j = 0; j < 4; ++j) o.a |= (((j ^ x) + 4u * hi) << (4 * j));
  o.b = (c >> 3) ? 0x7654u : 0x3210u;
  return o;
}
__device__ __forceinline__ uint4 lane_permute(const uint4& q, const LaneOrder& o) {
  const uint32_t t0 = __byte_perm(q.x, q.y, o.a), t1 = __byte_perm(q.y, q.x, o.a);
  const uint32_t t2 = __byte_perm(q.z, q.w, o.a), t3 = __byte_perm(q.w, q.z, o.a);
  return make_uint4(__byte_perm(t0, t2, o.b), __byte_perm(t1, t3, o.b), __byte_perm(t2, t0, o.b),
                    __byte_perm(t3, t1, o.b));
}

template <int PATH, int LK>
__device__ __forceinline__ void count_vec(const uint4& q0, uint32_t base, uint32_t lutb, uint32_t table,
                                          const LaneOrder& o) {
  // the shift layouts with 16 or 32 sub-bins per bin give each lane its own
  // bank whatever the order (lane l uses bank l mod 2^LK of a bin's row)
  const uint4 q = (PATH == PATH_SHIFT && LK >= 4) ? q0 : lane_permute(q0, o);
  count_word<PATH, LK>(q.x, base, lutb, table);
  count_word<PATH, LK>(q.y, base, lutb, table);
  count_word<PATH, LK>(q.z, base, lutb, table);
  count_word<PATH, LK>(q.w, base, lutb, table);
}

// Shared-window addresses of this thread's slots for a layout.
template <int PATH, int LK>
__device__ __forceinline__ void thread_bases(const uint32_t* table, const uint32_t* lut, uint32_t& base,
                                             uint32_t& lutb, uint32_t& tab) {
  const uint32_t lane = threadIdx.x & 31;
  tab = smem_addr(table);
  if (PATH == PATH_PLAIN) base = tab + (threadIdx.x >> 5) * HIST_BINS * 4;
  else base = tab + ((lane & ((1u << LK) - 1u)) << 2);
  lutb = smem_addr(lut) + (lane << 2);
}

// Count the 16-byte vectors [begin, end) of p with threads 0..nthr-1 of the
// CTA: thread tid takes vectors begin + tid, begin + tid + nthr, ...
// (coalesced) in groups of UNROLL.  The loop is software-pipelined: a
// thread issues the loads of its next group before it counts the current
// one, so its loads stay in flight while it counts (about 9 % more
// throughput than loading and counting in turn).
template <int PATH, int LK, int UNROLL>
static __device__ void count_range(const uint4* __restrict__ p, size_t begin, size_t end, uint32_t* table,
                                   const uint32_t* lut, int tid, int nthr) {
  uint32_t base, lutb, tab;
  thread_bases<PATH, LK>(table, lut, base, lutb, tab);
  const LaneOrder o = lane_order();
  size_t i = begin + tid;
  if (i + (size_t)(UNROLL - 1) * nthr < end) {
    uint4 v[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) v[u] = ldg_stream(p + i + (size_t)u * nthr);
    i += (size_t)UNROLL * nthr;
    for (; i + (size_t)(UNROLL - 1) * nthr < end; i += (size_t)UNROLL * nthr) {
      uint4 w[UNROLL];
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) w[u] = ldg_stream(p + i + (size_t)u * nthr);
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) count_vec<PATH, LK>(v[u], base, lutb, tab, o);
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) v[u] = w[u];
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) count_vec<PATH, LK>(v[u], base, lutb, tab, o);
  }
  for (; i < end; i += nthr) count_vec<PATH, LK>(ldg_stream(p + i), base, lutb, tab, o);
}

// The whole CTA, two loads in flight.
template <int PATH, int LK>
static __device__ void count_slice(const uint4* __restrict__ p, size_t begin, size_t end, uint32_t* table,
                                   const uint32_t* lut) {
  count_range<PATH, LK, 2>(p, begin, end, table, lut, threadIdx.x, kThreads);
}

// Layout dispatch for count_range.
template <int UNROLL>
__device__ __forceinline__ void count_range_dispatch(int path, int lk, const uint4* p, size_t begin, size_t end,
                                                     uint32_t* table, const uint32_t* lut, int tid, int nthr) {
  if (begin >= end) return;
  if (path == PATH_PLAIN) count_range<PATH_PLAIN, 0, UNROLL>(p, begin, end, table, lut, tid, nthr);
  else if (path == PATH_LUT) count_range<PATH_LUT, 0, UNROLL>(p, begin, end, table, lut, tid, nthr);
  else {
    switch (lk) {
      case 5: count_range<PATH_SHIFT, 5, UNROLL>(p, begin, end, table, lut, tid, nthr); break;
      case 4: count_range<PATH_SHIFT, 4, UNROLL>(p, begin, end, table, lut, tid, nthr); break;
      case 3: count_range<PATH_SHIFT, 3, UNROLL>(p, begin, end, table, lut, tid, nthr); break;
      case 2: count_range<PATH_SHIFT, 2, UNROLL>(p, begin, end, table, lut, tid, nthr); break;
      case 1: count_range<PATH_SHIFT, 1, UNROLL>(p, begin, end, table, lut, tid, nthr); break;
      default: count_range<PATH_SHIFT, 0, UNROLL>(p, begin, end, table, lut, tid, nthr); break;
    }
  }
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

// count_dispatch as a call of its own, for kernels that run at 32 registers
// with other phases that need more: those spill around the call, and the
// counting loop keeps its registers.
static __device__ __noinline__ void count_call(int path, int lk, const uint4* p, size_t begin, size_t end,
                                               uint32_t* table, const uint32_t* lut) {
  count_dispatch(path, lk, p, begin, end, table, lut);
}

// The whole CTA with four loads in flight per thread, for kernels that run
// one CTA of 1024 threads per SM (64 registers): the SM then keeps as many
// bytes in flight as two CTAs with two loads each.
static __device__ __noinline__ void count_call4(int path, int lk, const uint4* p, size_t begin, size_t end,
                                                uint32_t* table, const uint32_t* lut) {
  count_range_dispatch<4>(path, lk, p, begin, end, table, lut, threadIdx.x, kThreads);
}

__device__ __forceinline__ void zero_table(uint32_t* table) {
  uint4* t4 = reinterpret_cast<uint4*>(table);
  for (int i = threadIdx.x; i < kTableWords / 4; i += kThreads) t4[i] = make_uint4(0, 0, 0, 0);
}

// Reduce the table to per-bin sums in cs.res (all threads call; ends with a barrier).
// `part` is 1024 words of free shared memory.  With `clear`, a layout whose
// reduction reads every table word (the lane-private table) also zeroes the
// table as it reads it; returns whether it did.
static __device__ bool flush_table(int path, int lk, uint32_t* table, const hist_pattern& pat, uint32_t* part,
                                   CtaShared& cs, bool clear = false) {
  __syncthreads();
  if (path == PATH_SHIFT && lk == 5) {
    // bin b is the 32 words of row b, one per lane: warp w reduces rows w,
    // w + 32, ... with one read per lane and a warp-wide add
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int b = w; b < HIST_BINS; b += kWarps) {
      const uint32_t v = table[(b << 5) + lane];
      if (clear) table[(b << 5) + lane] = 0;
      const uint32_t sum = __reduce_add_sync(0xffffffffu, v);
      if (lane == 0) cs.res[b] = sum;
    }
    __syncthreads();
    return clear;
  }
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
  return false;
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

// -------------------------------------------------------- binning pattern --

__device__ __forceinline__ uint32_t ilog2_u64(unsigned long long v) { return 63u - __clzll(v); }

// Default pattern (reading of Figure 1), log2 of the sub-bins of bin b.
__device__ __forceinline__ uint32_t default_lk(uint32_t b, uint32_t budget) {
  if (budget < 960) return 0;
  const uint32_t ls = ilog2_u64(budget / 960);
  const uint32_t r = b >> 5;  // region
  const uint32_t rlk = (r < 4) ? r : 7 - r;  // 0,1,2,3,3,2,1,0
  const uint32_t lk = rlk + ls;
  return lk > 5 ? 5 : lk;
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

// Split n bytes at address a into an unaligned head, 16-byte vectors and a
// tail.  The vectors start on a 128-byte boundary: a warp's load of 32
// consecutive vectors then covers four whole 128-byte lines wherever the
// bytes start (from a 16-byte boundary only, it touches five, and a counting
// loop over such vectors ran 2-3 % slower on GB300).
constexpr uint32_t kLineBytes = 128;
struct Split {
  size_t head;  // bytes before the first 128-byte boundary (<= 127; split_bytes_at: its boundary)
  size_t nvec;  // 16-byte vectors
  size_t tail;  // bytes after the vectors (<= 15)
};
// The same with the vectors from the first `align`-byte boundary (a power
// of two from 16 to 128).
__host__ __device__ __forceinline__ Split split_bytes_at(const uint8_t* a, size_t n, size_t align) {
  Split s;
  size_t h = (align - ((uintptr_t)a & (align - 1))) & (align - 1);
  s.head = h < n ? h : n;
  s.nvec = (n - s.head) / 16;
  s.tail = n - s.head - s.nvec * 16;
  return s;
}
__host__ __device__ __forceinline__ Split split_bytes(const uint8_t* a, size_t n) {
  return split_bytes_at(a, n, kLineBytes);
}

// A point at which a CTA's range cuts a buffer of memory p moves up to the
// buffer's next 32 KiB boundary (capped at the buffer's end by the caller),
// so that the CTAs' pieces start on 32 KiB boundaries: measured 1-2 % faster
// than starting them on any 128-byte line (the adaptive stream over 1 GiB,
// 6.48 -> 6.60 TB/s; the plain one 5.45 -> 5.51).  Both CTAs of a cut compute
// it from the same position, so their pieces still tile the buffer.
constexpr unsigned long long kSplitAlign = 32ull << 10;
__device__ __forceinline__ unsigned long long split_point(const uint8_t* p, unsigned long long b) {
  const unsigned long long a = (unsigned long long)(uintptr_t)p;
  return ((a + b + kSplitAlign - 1) & ~(kSplitAlign - 1)) - a;
}

// First vector of part b when nvec vectors are cut into `parts` contiguous
// ranges (b = parts gives nvec): b nvec / parts moved up to a multiple of g
// vectors, g the largest power of two up to 2048 (32 KiB) and up to 1/32 of
// a part, at least 8 (a 128-byte line).  One-shot launches over 1 GiB:
// the full table 6.61 -> 6.95 TB/s, the per-warp tables 5.44 -> 5.77 TB/s
// against equal parts cut anywhere (cuts on 128-byte lines alone gave
// 6.34 - 6.61 and 5.76).
__host__ __device__ __forceinline__ size_t part_begin(size_t nvec, size_t parts, size_t b) {
  const size_t per = nvec / parts;
  size_t g = 2048;
  while (g > 8 && g * 32 > per) g >>= 1;
  const size_t r = (nvec * b / parts + g - 1) & ~(g - 1);
  return r < nvec ? r : nvec;
}

// Count head and tail bytes of a split into the shared histogram h: thread
// t < 128 takes head byte t, thread 128 + i tail byte i (threads 0..143 of
// the CTA).
__device__ __forceinline__ void count_edges_into(const uint8_t* a, const Split& sp, uint32_t* h) {
  const int t = threadIdx.x, L = (int)kLineBytes;
  if (t < (int)sp.head) atomicAdd(&h[a[t]], 1u);
  else if (t >= L && t < L + (int)sp.tail) atomicAdd(&h[a[sp.head + sp.nvec * 16 + (t - L)]], 1u);
}

// Count head and tail bytes of a split into cs.res (threads 0..143).
__device__ __forceinline__ void count_edges(const uint8_t* a, const Split& sp, CtaShared& cs) {
  count_edges_into(a, sp, cs.res);
}

}  // namespace histdev

namespace histdev {

// ------------------------------------------------- single-warp epilogue --

// floor(a / b) for 0 < b < 2^32 and a / b < 2^20, exactly: an FP32 estimate
// (relative error below 2^-22, so within 1/4 of a quotient below 2^20)
// corrected by one integer step each way.  Other operands take the integer
// division.
__device__ __forceinline__ unsigned long long div_floor(unsigned long long a, unsigned long long b, float rb) {
  if (b < (1ull << 32) && a < (b << 20)) {
    unsigned long long q = (unsigned long long)(uint32_t)((float)a * rb);
    if (q * b > a) q -= 1;
    else if ((q + 1) * b <= a) q += 1;
    return q;
  }
  return a / b;
}

// One warp computes the degeneracy (Sec. III.C) and the binning pattern (the
// rule stated in hist.h) of the 256-bin histogram `hist`.  Lane l holds bins
// l + 32 i, i = 0..7.  Writes P (off, log2k, budget, used) and returns the
// degeneracy to every lane.
template <class T>
__device__ hist_degeneracy_result warp_epilogue(const T* hist, uint32_t budget, uint32_t theta_milli,
                                                hist_pattern& P) {
  const int lane = threadIdx.x & 31;
  unsigned long long h[8];
  unsigned long long tot = 0, mx = 0;
  int arg = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    h[i] = (unsigned long long)hist[lane + 32 * i];
    tot += h[i];
    if (h[i] > mx) {  // bins of one lane rise with i: the first maximum is the lowest
      mx = h[i];
      arg = lane + 32 * i;
    }
  }
  tot = warp_sum(tot);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, mx, o);
    const int a2 = __shfl_xor_sync(0xffffffffu, arg, o);
    if (m2 > mx || (m2 == mx && a2 < arg)) {
      mx = m2;
      arg = a2;
    }
  }
  hist_degeneracy_result r;
  r.max = mx;
  r.total = tot;
  r.maxbin = mx == 0 ? 0u : (uint32_t)arg;
  r.flag = reaches_theta(mx, tot, theta_milli) ? HIST_FLAG_ADAPTIVE : HIST_FLAG_PLAIN;

  uint32_t lk[8];
  if (tot == 0) {
#pragma unroll
    for (int i = 0; i < 8; ++i) lk[i] = default_lk(lane + 32 * i, budget);
  } else {
    const unsigned long long spare = budget - HIST_BINS;
    const float rt = 1.0f / (float)tot;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      // spare < 2^13 and h <= tot, so the quotient is below 2^13
      const unsigned long long want = 1ull + div_floor(spare * h[i], tot, rt);
      const uint32_t l0 = ilog2_u64(want);
      lk[i] = l0 > 5 ? 5 : l0;
    }
    uint32_t lf = 0;
    for (uint32_t f = 1; f <= 5; ++f) {
      unsigned long long s = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) s += 1ull << (lk[i] > f ? lk[i] : f);
      s = warp_sum(s);
      if (s <= budget) lf = f;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) lk[i] = lk[i] > lf ? lk[i] : lf;
  }
  // layout: classes of decreasing k, bins of one class in increasing index
  // (index lane + 32 i orders by i, then lane)
  uint32_t cnt[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) cnt[c] = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < 6; ++c) cnt[c] += __popc(__ballot_sync(0xffffffffu, lk[i] == (uint32_t)c));
  uint32_t base[6];
  uint32_t acc = 0;
#pragma unroll
  for (int c = 5; c >= 0; --c) {
    base[c] = acc;
    acc += cnt[c] << c;
  }
  const unsigned lt = (1u << lane) - 1u;
  uint32_t run[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) run[c] = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const unsigned m = __ballot_sync(0xffffffffu, lk[i] == (uint32_t)c);
      if (lk[i] == (uint32_t)c) {
        P.off[lane + 32 * i] = (uint16_t)(base[c] + ((run[c] + __popc(m & lt)) << c));
        P.log2k[lane + 32 * i] = (uint8_t)c;
      }
      run[c] += __popc(m);
    }
  }
  if (lane == 0) {
    P.used = acc;
    P.budget = budget;
  }
  __syncwarp();
  return r;
}

}  // namespace histdev

namespace histdev {

// Shared scratch of block_epilogue.
struct EpiShared {
  uint32_t wmax[8];     // per-warp largest count
  uint32_t warg[8];     // per-warp lowest bin holding it
  uint32_t fsum[8][5];  // per-warp sums of max(k0, 2^f), f = 1..5
  uint32_t cls[8][6];   // per-warp bins of each sub-bin class
};

// Degeneracy (Sec. III.C) and binning pattern (rule in hist.h) of the 256-bin
// histogram `hist` whose total is known to be `total`, by threads 0..255 (one
// bin each, warp reductions in hardware); all threads of the CTA call (two
// barriers).  Writes P; returns the degeneracy to threads 0..255.
static __device__ __noinline__ hist_degeneracy_result block_epilogue(const uint32_t* hist, unsigned long long total,
                                                        uint32_t budget, uint32_t theta_milli, hist_pattern& P,
                                                        EpiShared& es) {
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const bool act = t < HIST_BINS;
  const unsigned full = 0xffffffffu;
  const uint32_t h = act ? hist[t] : 0u;
  uint32_t lk0 = 0;
  if (act) {
    if (total == 0) {
      lk0 = default_lk(t, budget);
    } else {
      const unsigned long long spare = budget - HIST_BINS;
      const float rt = 1.0f / (float)total;
      const unsigned long long want = 1ull + div_floor(spare * (unsigned long long)h, total, rt);
      const uint32_t l0 = ilog2_u64(want);
      lk0 = l0 > 5 ? 5 : l0;
    }
  }
  if (w < 8) {
    const uint32_t wm = __reduce_max_sync(full, h);
    const uint32_t wa = __reduce_min_sync(full, h == wm ? (uint32_t)t : 0xffffffffu);
    uint32_t fs[5];
#pragma unroll
    for (int f = 1; f <= 5; ++f) fs[f - 1] = __reduce_add_sync(full, 1u << (lk0 > (uint32_t)f ? lk0 : (uint32_t)f));
    if (lane == 0) {
      es.wmax[w] = wm;
      es.warg[w] = wa;
#pragma unroll
      for (int f = 0; f < 5; ++f) es.fsum[w][f] = fs[f];
    }
  }
  __syncthreads();
  uint32_t lk = lk0;
  hist_degeneracy_result r;
  if (act) {
    uint32_t mx = 0, arg = 0xffffffffu;
#pragma unroll
    for (int i = 0; i < 8; ++i) mx = es.wmax[i] > mx ? es.wmax[i] : mx;
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (es.wmax[i] == mx && es.warg[i] < arg) arg = es.warg[i];
    r.max = mx;
    r.total = total;
    r.maxbin = mx == 0 ? 0u : arg;
    r.flag = reaches_theta(mx, total, theta_milli) ? HIST_FLAG_ADAPTIVE : HIST_FLAG_PLAIN;
    if (total != 0) {
      uint32_t lf = 0;
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) s += es.fsum[i][f];
        if (s <= budget) lf = (uint32_t)f + 1;
      }
      lk = lk0 > lf ? lk0 : lf;
    }
  }
  // layout: classes of decreasing k, ties by increasing bin index
  uint32_t rank = 0;
  if (w < 8) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const unsigned m = __ballot_sync(full, lk == (uint32_t)c);
      if (lk == (uint32_t)c) rank = __popc(m & ((1u << lane) - 1u));
      if (lane == 0) es.cls[w][c] = __popc(m);
    }
  }
  __syncthreads();
  if (act) {
    uint32_t base = 0, used = 0, before = 0;
#pragma unroll
    for (int c = 5; c >= 0; --c) {
      uint32_t cnt = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) cnt += es.cls[i][c];
      if ((uint32_t)c > lk) base += cnt << c;
      used += cnt << c;
    }
    for (int i = 0; i < w; ++i) before += es.cls[i][lk];
    P.off[t] = (uint16_t)(base + ((before + rank) << lk));
    P.log2k[t] = (uint8_t)lk;
    if (t == 0) {
      P.used = used;
      P.budget = budget;
    }
  }
  return r;
}

}  // namespace histdev

namespace histdev {

// ------------------------------------------------------ change detection --

// Shared scratch of change_eval.
struct ChangeShared {
  unsigned __int128 term[HIST_BINS];
  unsigned long long sa[8], sm[8];
};

// Total-variation distance between two histograms normalised to sum 1:
// D = sum_b |a_b SM - m_b SA| over 2 SA SM.  Threads 0..255 pass bin t of
// each (a, m); all threads of the CTA call (three barriers).  Thread 0 gets
// the result: the flag (1000 D >= 2 tau SA SM, exact in 128 bits while
// SA < 2^56 and SM < 2^40), floor(10^6 D / (2 SA SM)), and whether the sums
// were in that range.  Either histogram empty: distance 0.
__device__ __forceinline__ hist_change_result change_eval(unsigned long long a, unsigned long long m,
                                                          uint32_t tau_milli, ChangeShared& sh) {
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (t < HIST_BINS) {
    unsigned long long x = a, y = m;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) {
      sh.sa[w] = x;
      sh.sm[w] = y;
    }
  }
  __syncthreads();
  unsigned long long SA = 0, SM = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    SA += sh.sa[i];
    SM += sh.sm[i];
  }
  if (t < HIST_BINS) {
    const unsigned __int128 p = (unsigned __int128)a * SM, q = (unsigned __int128)m * SA;
    sh.term[t] = p > q ? p - q : q - p;
  }
  __syncthreads();
  for (int half = HIST_BINS / 2; half > 0; half >>= 1) {
    if (t < half) sh.term[t] += sh.term[t + half];
    __syncthreads();
  }
  hist_change_result r;
  r.flag = 0;
  r.in_range = (SA < (1ull << 56) && SM < (1ull << 40)) ? 1u : 0u;
  r.dist_ppm = 0;
  if (t == 0 && SA != 0 && SM != 0) {
    const unsigned __int128 D = sh.term[0];
    const unsigned __int128 den = (unsigned __int128)SA * SM * 2u;
    r.flag = (unsigned __int128)1000u * D >= den * tau_milli ? 1u : 0u;
    r.dist_ppm = (unsigned long long)((D * 1000000u) / den);
  } else if (t == 0) {
    r.flag = tau_milli == 0 ? 1u : 0u;  // distance 0 reaches only a threshold of 0
  }
  return r;
}

}  // namespace histdev
